// One level of the recursive tree contraction (paper, Section 3.2).
//
// A level is a tree (or, in batched mode, a forest) whose m_l edges are
// listed in ascending global rank with endpoints given as level vertex ids.
// Four kernels process it:
//
//   mark      min_word[x] = (rank, other end, side) of the lightest edge at
//             x (Eq. 1), by 64-bit atomicMin; the value each atomic returns
//             tells whether the edge can still be the lightest there
//   ptr_init  pointer forest: x points across its lightest edge; the two
//             endpoints of a leaf edge (lightest at both, Section 3.1) point
//             at each other and the smaller id becomes the root.  Roots get
//             dense ids (a single-pass scan) that name the supervertices of
//             the next level.  On level 0 it also writes the vertex parents
//             (Eq. 1).
//   compress  root finding with path halving: supervertex of x, packed on
//             levels >= 1 with x's chain key for the expansion.
//   compact   alpha-edges (Eq. 2: lightest at neither endpoint) are copied,
//             in rank order, to the next level with relabelled endpoints;
//             every other edge is contracted here and records the level and
//             its supervertex for the expansion.
//
// The non-alpha edges are exactly the lightest edges {P(x)}, so the components
// of the pointer forest are the components the paper contracts.  Along a
// pointer path the edge ranks strictly decrease except across a leaf edge,
// hence the forest is acyclic once each leaf edge's 2-cycle is broken.
#include "kernels.cuh"

namespace pandora {

namespace {

constexpr int LV_WARPS = LV_THREADS / 32;
static_assert(LV_ITEMS * LV_WARPS == 64, "scan helper assumes 64 (item, warp) slots");

// Exclusive ranks of the flagged elements of a striped tile (element it*256+tid),
// in element order, offset by the count of all earlier tiles (look-back).
// Returns the tile total in *tile_total.
__device__ __forceinline__ void tile_rank(const bool (&flag)[LV_ITEMS], u32 (&rank)[LV_ITEMS],
                                          u32 tile, u64 *lb, int *status, u64 *base_out,
                                          u32 *tile_total)
{
    __shared__ u32 s_cnt[LV_ITEMS * LV_WARPS];
    __shared__ u64 s_base;
    __shared__ u32 s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 ball[LV_ITEMS];
#pragma unroll
    for (int it = 0; it < LV_ITEMS; ++it) {
        ball[it] = __ballot_sync(0xFFFFFFFFu, flag[it]);
        if (lane == 0)
            s_cnt[it * LV_WARPS + warp] = __popc(ball[it]);
    }
    __syncthreads();
    if (warp == 0) {
        const u32 c0 = s_cnt[2 * lane], c1 = s_cnt[2 * lane + 1];
        const u32 sum = c0 + c1;
        u32 incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off)
                incl += y;
        }
        const u32 excl = incl - sum;
        s_cnt[2 * lane] = excl;
        s_cnt[2 * lane + 1] = excl + c0;
        const u32 total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (lane == 0) {
            s_base = lookback_exclusive(lb, tile, total, status);
            s_total = total;
        }
    }
    __syncthreads();
    const u64 base = s_base;
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < LV_ITEMS; ++it)
        rank[it] = (u32)base + s_cnt[it * LV_WARPS + warp] + __popc(ball[it] & lt);
    *base_out = base;
    *tile_total = s_total;
}

template <bool LEVEL0>
__global__ void __launch_bounds__(256) mark_kernel(const LevelParams p)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.m)
        return;
    const int2 e = p.ab[i];
    const u64 r = LEVEL0 ? (u64)i : (u64)p.er[i];
    const u64 wa = (r << 32) | ((u64)(u32)e.y << 1);        // at e.x: other end e.y, side 0
    const u64 wb = (r << 32) | ((u64)(u32)e.x << 1) | 1u;   // at e.y: other end e.x, side 1
    // A plain read first keeps hub vertices (stars) from serialising on one
    // address: the word only decreases, so a stale read may cost an unneeded
    // atomic but never a wrong skip.  The value seen (old) decides whether
    // this edge can still be the lightest at that endpoint.
    u64 old = p.min_word[e.x];
    if (old > wa)
        old = atomicMin((unsigned long long *)(p.min_word + e.x), (unsigned long long)wa);
    const bool maybe_a = old > wa;
    old = p.min_word[e.y];
    if (old > wb)
        old = atomicMin((unsigned long long *)(p.min_word + e.y), (unsigned long long)wb);
    const bool maybe_b = old > wb;
    p.maybe[i] = (unsigned char)((maybe_a ? 1 : 0) | (maybe_b ? 2 : 0));
}

template <bool LEVEL0, bool FOREST>
__global__ void __launch_bounds__(LV_THREADS) ptr_init_kernel(const LevelParams p)
{
    __shared__ u32 s_tile;
    if (threadIdx.x == 0)
        s_tile = atomicAdd(p.tile_counter, 1u);
    __syncthreads();
    const u32 tile = s_tile;
    const i64 tile_base = (i64)tile * LV_TILE;
    bool root[LV_ITEMS];
    i32 nxt[LV_ITEMS];
#pragma unroll
    for (int it = 0; it < LV_ITEMS; ++it) {
        const i64 x = tile_base + it * LV_THREADS + threadIdx.x;
        root[it] = false;
        nxt[it] = (i32)x;
        if (x >= p.n)
            continue;
        const u64 wx = p.min_word[x];
        if (wx == NO_EDGE) {
            root[it] = true;   // isolated vertex: a finished tree of a forest
        } else {
            const u32 r = (u32)(wx >> 32);
            const i32 y = (i32)((wx >> 1) & 0x7FFFFFFFu);
            if (y == (i32)x) {
                root[it] = true;   // self-loop: reported by compact on the level above
            } else {
                // a leaf edge (lightest at both ends) closes a 2-cycle; its
                // smaller endpoint becomes the root of the component
                const u64 wy = p.min_word[y];
                root[it] = ((u32)(wy >> 32) == r) && ((i32)x < y);
                nxt[it] = y;
            }
            if (LEVEL0) {
                i32 par = (i32)__ldg(p.perm + r);   // Eq. 1, caller edge id
                if (FOREST)
                    par -= (i32)__ldg(p.edge_off + tree_of_edge(p.edge_off, p.n_trees, par));
                p.vertex_parent[x] = par;
            }
        }
        if (LEVEL0 && wx == NO_EDGE)
            p.vertex_parent[x] = -1;
    }
    u32 rank[LV_ITEMS];
    u64 base;
    u32 total;
    tile_rank(root, rank, tile, p.lb, p.status, &base, &total);
#pragma unroll
    for (int it = 0; it < LV_ITEMS; ++it) {
        const i64 x = tile_base + it * LV_THREADS + threadIdx.x;
        if (x < p.n)
            p.ptr[x] = root[it] ? ~(i32)rank[it] : nxt[it];
    }
    if (threadIdx.x == 0 && tile == (u32)(level_tiles(p.n) - 1))
        *p.count_roots = base + total;
}

// Root finding with path halving.  Writes the supervertex of x; on levels
// >= 1 also the chain key 2*rank(P(x)) + side that the expansion compares
// against, packed with it.
template <bool LEVEL0>
__global__ void __launch_bounds__(256) compress_kernel(const LevelParams p)
{
    const i64 x = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= p.n)
        return;
    i32 *ptr = p.ptr;
    i32 cur = (i32)x;
    i32 res;
    i64 iter = 0;
    for (;;) {
        const i32 pc = ld_volatile(ptr + cur);
        if (pc < 0) {
            res = pc;
            break;
        }
        const i32 g = ld_volatile(ptr + pc);
        if (g < 0) {
            res = g;
            break;
        }
        st_volatile(ptr + cur, g);   // path halving: g is an ancestor of cur
        cur = g;
        if (++iter > p.n + 64) {
            set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
            res = ~0;
            break;
        }
    }
    if (LEVEL0) {
        p.vmap[x] = ~res;
    } else {
        const u64 wx = p.min_word[x];
        const u32 ck = wx == NO_EDGE ? NONE : 2u * (u32)(wx >> 32) + (u32)(wx & 1u);
        p.rec[x] = make_int2((i32)ck, ~res);
    }
    if (cur != (i32)x)
        st_volatile(ptr + x, res);     // later walks through x stop here
}

template <bool LEVEL0>
__global__ void __launch_bounds__(LV_THREADS) compact_kernel(const LevelParams p)
{
    __shared__ u32 s_tile;
    if (threadIdx.x == 0)
        s_tile = atomicAdd(p.tile_counter + 1, 1u);
    __syncthreads();
    const u32 tile = s_tile;
    const i64 tile_base = (i64)tile * LV_TILE;
    bool alpha[LV_ITEMS];
    int2 nab[LV_ITEMS];
    u32 rr[LV_ITEMS];
#pragma unroll
    for (int it = 0; it < LV_ITEMS; ++it) {
        const i64 i = tile_base + it * LV_THREADS + threadIdx.x;
        alpha[it] = false;
        if (i >= p.m)
            continue;
        const int2 e = p.ab[i];
        const u32 r = LEVEL0 ? (u32)i : p.er[i];
        const unsigned mb = p.maybe[i];
        rr[it] = r;
        // Eq. 2: an alpha-edge is the lightest incident edge of neither endpoint
        const bool a_min = (mb & 1) && (u32)(p.min_word[e.x] >> 32) == r;
        const bool b_min = (mb & 2) && (u32)(p.min_word[e.y] >> 32) == r;
        const i32 va = LEVEL0 ? p.vmap[e.x] : p.rec[e.x].y;
        if (!a_min && !b_min) {
            const i32 vb = LEVEL0 ? p.vmap[e.y] : p.rec[e.y].y;
            if (va == vb)
                set_status(p.status, PANDORA_ERR_NOT_A_TREE);   // a cycle closed up
            alpha[it] = true;
            nab[it] = make_int2(va, vb);
        } else {
            p.lev[r] = (unsigned char)p.level;
            p.start[r] = va;
        }
    }
    u32 rank[LV_ITEMS];
    u64 base;
    u32 total;
    tile_rank(alpha, rank, tile, p.lb + level_tiles(p.n) + 1, p.status, &base, &total);
#pragma unroll
    for (int it = 0; it < LV_ITEMS; ++it) {
        if (alpha[it]) {
            // a tree has at most (m - 1) / 2 alpha-edges (Section 4.2); more
            // means the input had a cycle (multi-edges): report, never overflow
            if ((i64)rank[it] < p.cap_next) {
                p.ab_next[rank[it]] = nab[it];
                p.er_next[rank[it]] = rr[it];
            } else {
                set_status(p.status, PANDORA_ERR_NOT_A_TREE);
            }
        }
    }
    if (threadIdx.x == 0 && tile == (u32)(level_tiles(p.m) - 1))
        *p.count_alpha = base + total;
}

}  // namespace

void launch_mark(const LevelParams &p, cudaStream_t s)
{
    if (p.m <= 0)
        return;
    const unsigned blocks = (unsigned)((p.m + 255) / 256);
    if (p.level == 0)
        mark_kernel<true><<<blocks, 256, 0, s>>>(p);
    else
        mark_kernel<false><<<blocks, 256, 0, s>>>(p);
}

void launch_ptr_init(const LevelParams &p, cudaStream_t s)
{
    const unsigned blocks = (unsigned)level_tiles(p.n);
    if (p.level == 0) {
        if (p.edge_off)
            ptr_init_kernel<true, true><<<blocks, LV_THREADS, 0, s>>>(p);
        else
            ptr_init_kernel<true, false><<<blocks, LV_THREADS, 0, s>>>(p);
    } else {
        ptr_init_kernel<false, false><<<blocks, LV_THREADS, 0, s>>>(p);
    }
}

void launch_compress(const LevelParams &p, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((p.n + 255) / 256);
    if (p.level == 0)
        compress_kernel<true><<<blocks, 256, 0, s>>>(p);
    else
        compress_kernel<false><<<blocks, 256, 0, s>>>(p);
}

void launch_compact(const LevelParams &p, cudaStream_t s)
{
    if (p.m <= 0)
        return;
    const unsigned blocks = (unsigned)level_tiles(p.m);
    if (p.level == 0)
        compact_kernel<true><<<blocks, LV_THREADS, 0, s>>>(p);
    else
        compact_kernel<false><<<blocks, LV_THREADS, 0, s>>>(p);
}

}  // namespace pandora

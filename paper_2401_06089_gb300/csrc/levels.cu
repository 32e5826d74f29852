// One level of the recursive tree contraction (paper, Section 3.2).
//
// A level is a tree (or, in batched mode, a forest) whose m_l edges are
// listed in ascending global rank with endpoints given as level vertex ids.
// Four kernels process it:
//
//   mark      min_inc[x] = local index of the lightest edge at x  (Eq. 1)
//   ptr_init  pointer forest: x points across its lightest edge; the two
//             endpoints of a leaf edge (lightest at both, Section 3.1) point
//             at each other and the smaller id becomes the root.  Roots get
//             dense ids (a single-pass scan) that name the supervertices of
//             the next level.  Also records the chain key of x (levels >= 1)
//             and, on level 0, the vertex parents (Eq. 1).
//   compress  root finding with path halving: vmap[x] = supervertex of x.
//   compact   alpha-edges (Eq. 2: lightest at neither endpoint) are copied,
//             in rank order, to the next level with relabelled endpoints;
//             every other edge is contracted here and records the level and
//             its supervertex for the expansion.
//
// The non-alpha edges are exactly the edges {min_inc[x]}, so the components
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

__global__ void __launch_bounds__(256) mark_kernel(const int2 *__restrict__ ab, i64 m,
                                                   u32 *__restrict__ min_inc)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m)
        return;
    const int2 e = ab[i];
    const u32 r = (u32)i;
    // Filtering by a plain read first keeps hub vertices (stars) from
    // serialising on one address: min_inc only decreases, so a stale read can
    // cause an unneeded atomic but never a wrong skip.
    if (min_inc[e.x] > r)
        atomicMin(min_inc + e.x, r);
    if (min_inc[e.y] > r)
        atomicMin(min_inc + e.y, r);
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
        const u32 i = p.min_inc[x];
        u32 ck = NONE;
        if (i == NONE) {
            root[it] = true;   // isolated vertex: a finished tree of a forest, or n = 1
        } else {
            const int2 e = __ldg(p.ab + i);
            const i32 y = e.x ^ e.y ^ (i32)x;
            if (y == (i32)x) {
                root[it] = true;   // self-loop: reported by compact on the level above
            } else {
                const u32 j = p.min_inc[y];
                root[it] = (j == i) && ((i32)x < y);
                nxt[it] = y;
            }
            if (!LEVEL0) {
                const u32 r = __ldg(p.er + i);
                ck = 2u * r + (e.y == (i32)x ? 1u : 0u);
            }
        }
        if (!LEVEL0)
            p.ck[x] = ck;
        if (LEVEL0) {
            i32 par = -1;
            if (i != NONE) {
                par = (i32)__ldg(p.perm + i);
                if (FOREST)
                    par -= (i32)__ldg(p.edge_off + tree_of_edge(p.edge_off, p.n_trees, par));
            }
            p.vertex_parent[x] = par;
        }
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

__global__ void __launch_bounds__(256) compress_kernel(i32 *ptr, i32 *__restrict__ vmap, i64 n,
                                                       int *status)
{
    const i64 x = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n)
        return;
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
        if (++iter > n + 64) {
            set_status(status, PANDORA_ERR_ITERATION_LIMIT);
            res = ~0;
            break;
        }
    }
    vmap[x] = ~res;
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
        rr[it] = r;
        const bool a_min = p.min_inc[e.x] == (u32)i;
        const bool b_min = p.min_inc[e.y] == (u32)i;
        const i32 va = p.vmap[e.x];
        if (!a_min && !b_min) {
            const i32 vb = p.vmap[e.y];
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
    mark_kernel<<<(unsigned)((p.m + 255) / 256), 256, 0, s>>>(p.ab, p.m, p.min_inc);
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
    compress_kernel<<<(unsigned)((p.n + 255) / 256), 256, 0, s>>>(p.ptr, p.vmap, p.n, p.status);
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

// One level of the recursive tree contraction (paper, Section 3.2).
//
// A level is a tree (or, in batched mode, a forest) whose m_l edges are
// listed in ascending global rank with endpoints given as level vertex ids.
// Four kernels process it:
//
//   mark      min_word[x] = (rank, other end, side) of the lightest edge at
//             x (Eq. 1), by 64-bit atomicMin after a plain read (mark.cu)
//   ptr_init  pointer forest: x points across its lightest edge; the two
//             endpoints of a leaf edge (lightest at both, Section 3.1) point
//             at each other and the smaller id becomes the root.  Roots get
//             dense ids (a single-pass scan) that name the supervertices of
//             the next level.  On level 0 it also writes the vertex parents
//             (Eq. 1).
//   compress  root finding: supervertex of x (on level 0 with edge flags
//             the tag ~supervertex in x's pointer word; without flags beside
//             the rank of x's lightest edge in x's word; on levels >= 1 in a
//             record with x's chain key, kept for the expansion).
//   compact   alpha-edges (Eq. 2: lightest at neither endpoint) are copied,
//             in rank order, to the next level with relabelled endpoints;
//             every other edge is contracted here and records the level and
//             its supervertex for the expansion.  One random read per
//             endpoint (rank and supervertex together), the second only when
//             the edge is not the lightest at the first.
//
// The non-alpha edges are exactly the lightest edges {P(x)}, so the components
// of the pointer forest are the components the paper contracts.  Along a
// pointer path the edge ranks strictly decrease except across a leaf edge,
// hence the forest is acyclic once each leaf edge's 2-cycle is broken.
#include <atomic>

#include "kernels.cuh"

// Resident blocks of 256 threads per SM the tile-ranking level kernels
// (ptr_init, compact) are compiled for (40 registers): their tiles wait on
// dependent loads and block barriers, so more resident tiles hide more of
// it.  At 10^8 edges, random recursive tree: ptr_init 1.71 -> 1.55 ms,
// compact 3.79 -> 3.38 ms against the unconstrained 48 and 63 registers
// (4 and 5 blocks resident); 5 and 8 blocks were slower than 6.
#ifndef PANDORA_LV_MINB
#define PANDORA_LV_MINB 6
#endif

namespace pandora {

namespace {

constexpr int LV_WARPS = LV_THREADS / 32;
static_assert(LV_ITEMS * LV_WARPS == 64, "scan helper assumes 64 (item, warp) slots");

// Exclusive ranks of the flagged elements of a striped tile (element it*256+tid),
// in element order, offset by the count of all earlier tiles (look-back).
// Returns the tile total in *tile_total.
__device__ __forceinline__ void tile_rank(const bool (&flag)[LV_ITEMS], u32 (&rank)[LV_ITEMS],
                                          u32 tile, u64 *lb, int *status, u64 *base_out,
                                          u32 *tile_total, u32 report)
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
            s_base = lookback_exclusive(lb, tile, total, status, report);
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

__global__ void __launch_bounds__(256) init_level_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 n = dev_count(p.d_n, p.n_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *p.d_n_deep = 0;
    for (i64 x = (i64)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (i64)gridDim.x * blockDim.x)
        p.min_word[x] = NO_EDGE;
}

__device__ __forceinline__ u32 eflag_of(const u32 *eflag, u64 r)
{
    return (__ldg(eflag + (r >> 4)) >> (2 * (u32)(r & 15))) & 3u;
}

// Claims the next tile of a dynamically scheduled kernel (tile ids are handed
// out in launch order, which keeps the look-back deadlock-free).
__device__ __forceinline__ u32 claim_tile(u32 *counter, u32 *s_tile)
{
    __syncthreads();   // everyone has read the previous tile id
    if (threadIdx.x == 0)
        *s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    return *s_tile;
}

template <bool LEVEL0, bool FOREST>
__global__ void __launch_bounds__(LV_THREADS, PANDORA_LV_MINB) ptr_init_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 n = dev_count(p.d_n, p.n_cap);
    const i64 tiles = level_tiles(n);
    __shared__ u32 s_tile;
    // persistent: a block keeps claiming tiles until the level is covered, so
    // a grid sized for the worst case costs one atomic per block, not per tile
    for (u32 tile = claim_tile(p.tile_counter, &s_tile); (i64)tile < tiles;
         tile = claim_tile(p.tile_counter, &s_tile)) {
        const i64 tile_base = (i64)tile * LV_TILE;
        bool root[LV_ITEMS];
        i32 nxt[LV_ITEMS];
#pragma unroll
        for (int it = 0; it < LV_ITEMS; ++it) {
            const i64 x = tile_base + it * LV_THREADS + threadIdx.x;
            root[it] = false;
            nxt[it] = (i32)x;
            if (x >= n)
                continue;
            const u64 wx = p.min_word[x];
            if (wx == NO_EDGE) {
                root[it] = true;   // isolated vertex: a finished tree of a forest
            } else {
                const u32 r = (u32)(wx >> 32);
                const i32 y = (i32)((wx >> 1) & 0x7FFFFFFFu);
                if (y == (i32)x || (i64)y >= n) {
                    root[it] = true;   // self-loop (reported by compact on the level above)
                } else {
                    // a leaf edge (lightest at both ends) closes a 2-cycle; its
                    // smaller endpoint becomes the root of the component
                    bool leaf;
                    if (LEVEL0 && p.eflag)
                        leaf = eflag_of(p.eflag, r) == 3u;
                    else
                        leaf = (u32)(p.min_word[y] >> 32) == r;
                    root[it] = leaf && ((i32)x < y);
                    nxt[it] = y;
                }
                if (LEVEL0 && !p.eflag) {   // with flags the flag pass wrote it
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
        tile_rank(root, rank, tile, p.lb, p.status, &base, &total, p.report_limit);
#pragma unroll
        for (int it = 0; it < LV_ITEMS; ++it) {
            const i64 x = tile_base + it * LV_THREADS + threadIdx.x;
            if (x < n)
                p.ptr[x] = root[it] ? ~(i32)rank[it] : nxt[it];
            if (LEVEL0 && FOREST && p.tree_roots) {
                // roots per tree, one atomic per tree and warp
                const i64 t = root[it] ? tree_of_vertex(p.edge_off, p.n_trees, x) : -1;
                const u32 peers = __match_any_sync(0xFFFFFFFFu, (unsigned long long)t);
                if (root[it] && (threadIdx.x & 31) == __ffs(peers) - 1) {
                    atomicAdd(p.tree_roots + t, (u32)__popc(peers));
                    p.tree_root_id[t] = (i32)rank[it];
                }
            }
        }
        if (threadIdx.x == 0 && (i64)tile == tiles - 1)
            *p.d_n_next = base + total;
    }
}

// Root finding, in two parts.
//
// 1. compress_walk: every vertex follows its pointers, read-only, for at most
//    WALK_STEPS steps.  Lightest-edge pointer forests of trees with unordered
//    weights are shallow (depth <= 7 on random recursive, caterpillar and
//    binary trees with random weights), so almost every vertex reaches a root
//    or a vertex already resolved (tagged ~dense id), records its supervertex
//    and tags itself.  A vertex still unresolved after WALK_STEPS steps is
//    appended to the deep list.
// 2. Only when the deep list is not empty (long monotone chains, e.g. a path
//    whose weights increase along it), union-find over the deep vertices:
//    uf_union hooks the representative of lower hashed priority under the
//    other (CAS, path halving) for every deep vertex and its deep pointer
//    target; the top
//    of each deep component (its pointer target is resolved) stores the dense
//    root id at the component's representative (uf_tops), and uf_finish hands
//    it to every member.  This is the union-find contraction the paper uses
//    (after Jaiganesh and Burtscher), applied where pointer chasing would cost
//    log(depth) rounds per vertex.
#ifndef PANDORA_WALK_STEPS
#define PANDORA_WALK_STEPS 8
#endif
constexpr int WALK_STEPS = PANDORA_WALK_STEPS;

// Level 0 with edge flags: compact needs only the supervertex (the flags
// tell which endpoint chose the edge), and the pointer word of every
// resolved vertex already holds ~supervertex (the walk tags it so), so the
// pointer array (4 bytes per vertex) is the supervertex array and nothing
// else is written.  Level 0 without flags keeps the supervertex in the low
// half of x's own word (the rank of x's lightest edge stays in the high
// half), so that compact learns both from one random read; higher levels
// keep {chain key, supervertex} records for the expansion, which carry the
// rank as well (chain key >> 1).
template <bool LEVEL0>
__device__ __forceinline__ void write_supervertex(const LevelParams &p, i64 x, i32 dense)
{
    if (LEVEL0 && p.eflag) {
        p.ptr[x] = ~dense;
    } else if (LEVEL0) {
        const u64 wx = p.min_word[x];
        p.min_word[x] = (wx & 0xFFFFFFFF00000000ull) | (u32)dense;
    } else {
        const u64 wx = p.min_word[x];
        const u32 ck = wx == NO_EDGE ? NONE : 2u * (u32)(wx >> 32) + (u32)(wx & 1u);
        p.rec[x] = make_int2((i32)ck, dense);
    }
}

template <bool LEVEL0>
__global__ void __launch_bounds__(256) compress_walk_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 n = dev_count(p.d_n, p.n_cap);
    const int lane = threadIdx.x & 31;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    const i64 n_round = (n + 31) & ~(i64)31;
    for (i64 x = (i64)blockIdx.x * blockDim.x + threadIdx.x; x - lane < n_round; x += stride) {
        bool deep = false;
        if (x < n) {
            i32 cur = (i32)x;
            i32 res = 0;
            bool done = false;
            for (int step = 0; step < WALK_STEPS; ++step) {
                const i32 pc = ld_volatile(p.ptr + cur);
                if (pc < 0) {
                    res = pc;
                    done = true;
                    break;
                }
                cur = pc;
            }
            if (!done) {
                // a component with the level's (or the tree's) only root: no
                // union-find needed
                if (p.n_trees == 1) {
                    if (*(const volatile u64 *)p.d_n_next == 1) {
                        res = ~0;
                        done = true;
                    }
                } else if (LEVEL0 && p.tree_roots) {
                    const i64 t = tree_of_vertex(p.edge_off, p.n_trees, x);
                    if (p.tree_roots[t] == 1u) {
                        res = ~p.tree_root_id[t];
                        done = true;
                    }
                }
                cur = -1;
            }
            if (done) {
                if (cur != (i32)x)
                    st_volatile(p.ptr + x, res);   // resolved: later walks stop here
                if (!(LEVEL0 && p.eflag))   // with flags the tag is the supervertex
                    write_supervertex<LEVEL0>(p, x, ~res);
            } else {
                deep = true;
                p.uf[x] = (i32)x;
            }
        }
        // warp-aggregated append to the deep list
        const u32 ball = __ballot_sync(0xFFFFFFFFu, deep);
        if (ball) {
            u64 base = 0;
            if (lane == __ffs(ball) - 1)
                base = atomicAdd((unsigned long long *)p.d_n_deep, (unsigned long long)__popc(ball));
            base = __shfl_sync(0xFFFFFFFFu, base, __ffs(ball) - 1);
            if (deep)
                p.deep[base + __popc(ball & lanemask_lt())] = (i32)x;
        }
    }
}

// Root of a's union-find tree with path halving.  More than `report` steps
// record PANDORA_ERR_ITERATION_LIMIT (the find goes on); more than `bound`
// steps record it and stop at the ancestor reached.
__device__ __forceinline__ i32 uf_find(i32 *uf, i32 a, int *status, i64 bound, u32 report)
{
    i64 iter = 0;
    for (;;) {
        const i32 pa = ld_volatile(uf + a);
        if (pa == a)
            return a;
        const i32 ga = ld_volatile(uf + pa);
        if (ga != pa)
            st_volatile(uf + a, ga);   // path halving (benign race: ga is an ancestor)
        a = ga;
        ++iter;
        if (iter == (i64)report + 1)
            set_status(status, PANDORA_ERR_ITERATION_LIMIT);
        if (iter > bound) {
            set_status(status, PANDORA_ERR_ITERATION_LIMIT);
            return a;
        }
    }
}

// Linking priority of a union-find representative: the lowbias32 integer
// hash (C. Wellons), a bijection of 32-bit words, so priorities are distinct.
// Hooking by a pseudo-random priority instead of by id keeps the union-find
// trees shallow whatever the labelling: with ids, a path labelled in order
// whose weights increase along it would hook every vertex under its
// neighbour at once, one chain as long as the path, which every later find
// would walk.
__device__ __forceinline__ u32 uf_priority(i32 a)
{
    u32 x = (u32)a;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ i64 deep_count(const LevelParams &p)
{
    return dev_count(p.d_n_deep, p.n_cap);
}

__global__ void __launch_bounds__(256) uf_union_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 nd = deep_count(p);
    const i64 bound = dev_count(p.d_n, p.n_cap) + 64;
    for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < nd;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 x = p.deep[k];
        const i32 y = ld_volatile(p.ptr + x);
        if (ld_volatile(p.ptr + y) < 0)
            continue;   // y is resolved: x tops its deep component
        // both deep: hook the representative of lower priority under the
        // other one (see uf_priority)
        i32 a = x, b = y;
        for (i64 iter = 0;; ++iter) {
            a = uf_find(p.uf, a, p.status, bound, p.report_limit);
            b = uf_find(p.uf, b, p.status, bound, p.report_limit);
            if (a == b)
                break;
            if (uf_priority(a) > uf_priority(b)) {
                const i32 t = a;
                a = b;
                b = t;
            }
            const i32 old = atomicCAS(p.uf + a, a, b);
            if (old == a)
                break;
            a = old;
            if (iter == (i64)p.report_limit)
                set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
            if (iter > bound) {
                set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
                break;
            }
        }
    }
}

__global__ void __launch_bounds__(256) uf_tops_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 nd = deep_count(p);
    const i64 bound = dev_count(p.d_n, p.n_cap) + 64;
    for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < nd;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 x = p.deep[k];
        const i32 y = ld_volatile(p.ptr + x);
        const i32 py = ld_volatile(p.ptr + y);
        if (py < 0)
            p.root_of[uf_find(p.uf, x, p.status, bound, p.report_limit)] = ~py;
    }
}

template <bool LEVEL0>
__global__ void __launch_bounds__(256) uf_finish_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 nd = deep_count(p);
    const i64 bound = dev_count(p.d_n, p.n_cap) + 64;
    for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < nd;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 x = p.deep[k];
        write_supervertex<LEVEL0>(p, x,
                                  p.root_of[uf_find(p.uf, x, p.status, bound, p.report_limit)]);
    }
}

// Supervertex of level-0 vertex x from its pointer word (~dense id once root
// finding is done); a word that is not a valid tag only follows an error the
// root finding reported, and is kept inside the next level.
__device__ __forceinline__ i32 sv_of(const LevelParams &p, i32 x, u64 n_next)
{
    const i32 d = ~__ldg(p.ptr + x);
    if ((u32)d >= n_next) {
        set_status(p.status, PANDORA_ERR_NOT_A_TREE);
        return 0;
    }
    return d;
}

template <bool LEVEL0>
__global__ void __launch_bounds__(LV_THREADS, PANDORA_LV_MINB) compact_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 m = dev_count(p.d_m, p.m_cap);
    const i64 tiles = level_tiles(m);
    const u64 n_next = *(const volatile u64 *)p.d_n_next;   // supervertices (roots)
    __shared__ u32 s_tile;
    for (u32 tile = claim_tile(p.tile_counter + 1, &s_tile); (i64)tile < tiles;
         tile = claim_tile(p.tile_counter + 1, &s_tile)) {
        const i64 tile_base = (i64)tile * LV_TILE;
        bool alpha[LV_ITEMS];
        int2 nab[LV_ITEMS];
        u32 rr[LV_ITEMS];
#pragma unroll
        for (int it = 0; it < LV_ITEMS; ++it) {
            const i64 i = tile_base + it * LV_THREADS + threadIdx.x;
            alpha[it] = false;
            if (i >= m)
                continue;
            const int2 e = p.ab[i];
            const u32 r = LEVEL0 ? (u32)i : p.er[i];
            rr[it] = r;
            // Eq. 2: an alpha-edge is the lightest incident edge of neither
            // endpoint.  One read per endpoint gives the rank of its lightest
            // edge and its supervertex; the second endpoint is read only when
            // the edge is not the lightest at the first.
            u32 rank_a, rank_b;
            i32 va, vb;
            if (LEVEL0 && p.eflag) {
                // the pointer word of every vertex now holds ~supervertex; a
                // contracted edge (the flags say so) reads one endpoint's
                const u32 f = eflag_of(p.eflag, r);
                if (f) {
                    p.lev[r] = (unsigned char)p.level;
                    p.start[r] = sv_of(p, (f & 1u) ? e.x : e.y, n_next);
                    continue;
                }
                va = sv_of(p, e.x, n_next);
                vb = sv_of(p, e.y, n_next);
                if (va == vb)
                    set_status(p.status, PANDORA_ERR_NOT_A_TREE);   // a cycle closed up
                alpha[it] = true;
                nab[it] = make_int2(va, vb);
                continue;
            }
            if (LEVEL0) {
                const u64 wa = p.min_word[e.x];
                rank_a = (u32)(wa >> 32);
                va = (i32)(u32)wa;
            } else {
                const int2 ra = p.rec[e.x];
                rank_a = (u32)ra.x >> 1;
                va = ra.y;
            }
            if (rank_a == r) {
                p.lev[r] = (unsigned char)p.level;
                p.start[r] = va;
                continue;
            }
            if (LEVEL0) {
                const u64 wb = p.min_word[e.y];
                rank_b = (u32)(wb >> 32);
                vb = (i32)(u32)wb;
            } else {
                const int2 rb = p.rec[e.y];
                rank_b = (u32)rb.x >> 1;
                vb = rb.y;
            }
            if (rank_b == r) {
                p.lev[r] = (unsigned char)p.level;
                p.start[r] = vb;   // the edge is contracted: same supervertex as e.x
            } else {
                if (va == vb)
                    set_status(p.status, PANDORA_ERR_NOT_A_TREE);   // a cycle closed up
                alpha[it] = true;
                nab[it] = make_int2(va, vb);
            }
        }
        u32 rank[LV_ITEMS];
        u64 base;
        u32 total;
        tile_rank(alpha, rank, tile, p.lb + level_tiles(p.n_grid) + 1, p.status, &base, &total,
                  p.report_limit);
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
        if (threadIdx.x == 0 && (i64)tile == tiles - 1) {
            const u64 n_alpha = base + total;
            *p.d_m_next = n_alpha;
            // every level of a forest of T trees has n = m + T (n_next is the
            // root count ptr_init wrote for this level)
            if (*(volatile u64 *)p.d_n_next != n_alpha + (u64)p.n_trees)
                set_status(p.status, PANDORA_ERR_NOT_A_TREE);
            if (n_alpha == 0)
                *p.d_n_levels = p.level + 1;
        }
    }
}

}  // namespace

void launch_init_level(const LevelParams &p, cudaStream_t s)
{
    i64 b = (p.n_grid + 255) / 256;
    if (b > 152 * 16)
        b = 152 * 16;
    init_level_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(p);
}

void launch_ptr_init(const LevelParams &p, cudaStream_t s)
{
    const unsigned blocks = grid_for(p.n_grid, LV_TILE);
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
    const unsigned blocks = grid_for(p.n_grid, 256);
    if (p.level == 0)
        compress_walk_kernel<true><<<blocks, 256, 0, s>>>(p);
    else
        compress_walk_kernel<false><<<blocks, 256, 0, s>>>(p);
    // the union-find part exits at once when the deep list is empty
    const unsigned uf_blocks = grid_for(p.n_grid, 256, PANDORA_UF_BPS);
    uf_union_kernel<<<uf_blocks, 256, 0, s>>>(p);
    uf_tops_kernel<<<uf_blocks, 256, 0, s>>>(p);
    if (p.level == 0)
        uf_finish_kernel<true><<<uf_blocks, 256, 0, s>>>(p);
    else
        uf_finish_kernel<false><<<uf_blocks, 256, 0, s>>>(p);
}

void launch_compact(const LevelParams &p, cudaStream_t s)
{
    const unsigned blocks = grid_for(p.m_grid, LV_TILE);
    if (p.level == 0)
        compact_kernel<true><<<blocks, LV_THREADS, 0, s>>>(p);
    else
        compact_kernel<false><<<blocks, LV_THREADS, 0, s>>>(p);
}

}  // namespace pandora

// One level of the recursive tree contraction (paper, Section 3.2).
//
// A level is a tree (or, in batched mode, a forest) whose m_l edges are
// listed in ascending global rank with endpoints given as level vertex ids.
// Four kernels process it:
//
//   mark      min_word[x] = (rank, other end, side) of the lightest edge at
//             x (Eq. 1), by 64-bit atomicMin after a plain read
//   ptr_init  pointer forest: x points across its lightest edge; the two
//             endpoints of a leaf edge (lightest at both, Section 3.1) point
//             at each other and the smaller id becomes the root.  Roots get
//             dense ids (a single-pass scan) that name the supervertices of
//             the next level.  On level 0 it also writes the vertex parents
//             (Eq. 1).
//   compress  root finding: supervertex of x, kept beside the rank of x's
//             lightest edge (in x's word on level 0; on levels >= 1 in a
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

// Level kernels run only while the loop is open: once a level without
// alpha-edges has set n_levels, kernels launched for later (bound) levels
// exit at once.
__device__ __forceinline__ bool loop_closed(const LevelParams &p)
{
    return *(const volatile int *)p.d_n_levels != 0;
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

// Blocks per SM of the mark grid.  Fewer random reads and atomics in flight
// thrash L2 less: at 10^8 edges 3-4 blocks of 256 per SM beat 16 (7.2-7.6 vs
// 9.2 ms for all levels of a random recursive tree).
#ifndef PANDORA_MARK_BPS
#define PANDORA_MARK_BPS 3
#endif
template <bool LEVEL0>
__global__ void __launch_bounds__(256) mark_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 m = dev_count(p.d_m, p.m_cap);
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (i64)gridDim.x * blockDim.x) {
        const int2 e = p.ab[i];
        const u64 r = LEVEL0 ? (u64)i : (u64)p.er[i];
        const u64 wa = (r << 32) | ((u64)(u32)e.y << 1);        // at e.x: other end e.y, side 0
        const u64 wb = (r << 32) | ((u64)(u32)e.x << 1) | 1u;   // at e.y: other end e.x, side 1
        // A plain read first keeps hub vertices (stars) from serialising on one
        // address: the word only decreases, so a stale read may cost an unneeded
        // atomic but never a wrong skip.
        const u64 oa = p.min_word[e.x], ob = p.min_word[e.y];   // both reads before the atomics
        if (oa > wa)
            atomicMin((unsigned long long *)(p.min_word + e.x), (unsigned long long)wa);
        if (ob > wb)
            atomicMin((unsigned long long *)(p.min_word + e.y), (unsigned long long)wb);
    }
}

// ---- bucketed marking ---------------------------------------------------------
// On a level whose word array is much larger than L2 every random word access
// of mark moves whole DRAM bursts and mostly misses.  Bucketed marking first
// groups the level's 2m incidences by vertex bucket (2^mark_shift vertices,
// a word range of 32 MB) -- count, bucket starts, scatter -- and then applies
// them bucket after bucket, so that the atomics of the bucket in progress hit
// a word range that stays in L2.  The minimum does not depend on the order,
// so records inside a bucket may land in any order.
#ifndef PANDORA_MB_ITEMS
#define PANDORA_MB_ITEMS 8
#endif
constexpr int MB_TILE_ITEMS = PANDORA_MB_ITEMS;
#ifndef PANDORA_MARK_APPLY_BPS
#define PANDORA_MARK_APPLY_BPS 4
#endif
constexpr int MB_TILE = 256 * MB_TILE_ITEMS;   // edges per scatter tile

__device__ __forceinline__ int mark_bucket(const LevelParams &p, i32 x)
{
    const int b = (int)((u32)x >> p.mark_shift);
    return b < p.mark_buckets ? b : p.mark_buckets - 1;
}

__global__ void __launch_bounds__(256) mark_count_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    __shared__ u32 s_cnt[MARK_MAX_BUCKETS];
    for (int b = threadIdx.x; b < p.mark_buckets; b += blockDim.x)
        s_cnt[b] = 0;
    __syncthreads();
    const i64 m = dev_count(p.d_m, p.m_cap);
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (i64)gridDim.x * blockDim.x) {
        const int2 e = p.ab[i];
        atomicAdd(&s_cnt[mark_bucket(p, e.x)], 1u);
        atomicAdd(&s_cnt[mark_bucket(p, e.y)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < p.mark_buckets; b += blockDim.x)
        if (s_cnt[b])
            atomicAdd(p.mark_count + b, s_cnt[b]);
}

// Exclusive scan of the bucket counts (one block of MARK_MAX_BUCKETS threads).
__global__ void __launch_bounds__(MARK_MAX_BUCKETS) mark_prefix_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    __shared__ u64 s[MARK_MAX_BUCKETS];
    const int b = threadIdx.x;
    s[b] = b < p.mark_buckets ? (u64)p.mark_count[b] : 0ull;
    __syncthreads();
    for (int off = 1; off < MARK_MAX_BUCKETS; off <<= 1) {
        const u64 y = b >= off ? s[b - off] : 0ull;
        __syncthreads();
        s[b] += y;
        __syncthreads();
    }
    if (b < p.mark_buckets)
        p.mark_base[b + 1] = s[b];
    if (b == 0)
        p.mark_base[0] = 0;
}

// Dynamic shared memory of a scatter tile: the tile's records staged in
// bucket order (vertex, word, bucket; on level 0 with flags also the caller
// id) so that every bucket's run is written to global memory contiguously.
constexpr size_t MB_SMEM = (size_t)2 * MB_TILE * (8 + 4 + 2);
constexpr size_t MB_SMEM_C = (size_t)2 * MB_TILE * (8 + 4 + 4 + 2);

template <bool LEVEL0>
__global__ void __launch_bounds__(256) mark_scatter_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    extern __shared__ __align__(16) unsigned char mb_smem[];
    constexpr bool CID = LEVEL0;   // records carry caller ids when p.rec_c is set
    const bool with_c = CID && p.rec_c != nullptr;
    u64 *st_w = (u64 *)mb_smem;
    u32 *st_x = (u32 *)(st_w + 2 * MB_TILE);
    u32 *st_c = st_x + 2 * MB_TILE;   // only used with_c
    unsigned short *st_b = (unsigned short *)(st_x + (with_c ? 4 : 2) * MB_TILE);
    __shared__ u32 s_cnt[MARK_MAX_BUCKETS];
    __shared__ u32 s_off[MARK_MAX_BUCKETS];
    __shared__ u64 s_gbase[MARK_MAX_BUCKETS];
    __shared__ u32 s_warp[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const i64 m = dev_count(p.d_m, p.m_cap);
    const i64 tiles = (m + MB_TILE - 1) / MB_TILE;
    const u64 cap = 2 * (u64)p.m_cap;   // record capacity (the counts never exceed it)
    for (i64 tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        for (int b = threadIdx.x; b < MARK_MAX_BUCKETS; b += blockDim.x)
            s_cnt[b] = 0;
        __syncthreads();
        int2 e[MB_TILE_ITEMS];
        u32 r[MB_TILE_ITEMS], sa[MB_TILE_ITEMS], sb[MB_TILE_ITEMS], cid[MB_TILE_ITEMS];
        const i64 t0 = tile * MB_TILE;
        const int count = (int)min((i64)MB_TILE, m - t0);
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it) {
            const int k = it * 256 + threadIdx.x;
            if (k < count) {
                e[it] = p.ab[t0 + k];
                if (with_c)
                    cid[it] = p.perm[t0 + k];
                r[it] = LEVEL0 ? (u32)(t0 + k) : p.er[t0 + k];
                sa[it] = atomicAdd(&s_cnt[mark_bucket(p, e[it].x)], 1u);
                sb[it] = atomicAdd(&s_cnt[mark_bucket(p, e[it].y)], 1u);
            }
        }
        __syncthreads();
        // exclusive scan of the bucket counts (two buckets per thread)
        const u32 c0 = s_cnt[2 * threadIdx.x], c1 = s_cnt[2 * threadIdx.x + 1];
        u32 incl = c0 + c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            s_warp[warp] = incl;
        __syncthreads();
        u32 wpre = 0;
        for (int w = 0; w < warp; ++w)
            wpre += s_warp[w];
        const u32 excl = wpre + incl - (c0 + c1);
        s_off[2 * threadIdx.x] = excl;
        s_off[2 * threadIdx.x + 1] = excl + c0;
        for (int b = threadIdx.x; b < p.mark_buckets; b += blockDim.x)
            if (s_cnt[b])
                s_gbase[b] = p.mark_base[b] + atomicAdd(p.mark_cursor + b, s_cnt[b]);
        __syncthreads();
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it) {
            const int k = it * 256 + threadIdx.x;
            if (k < count) {
                const u64 ra = (u64)r[it] << 32;
                const int ba = mark_bucket(p, e[it].x), bb = mark_bucket(p, e[it].y);
                const u32 ja = s_off[ba] + sa[it], jb = s_off[bb] + sb[it];
                st_x[ja] = (u32)e[it].x;
                st_w[ja] = ra | ((u64)(u32)e[it].y << 1);        // at e.x: side 0
                st_b[ja] = (unsigned short)ba;
                st_x[jb] = (u32)e[it].y;
                st_w[jb] = ra | ((u64)(u32)e[it].x << 1) | 1u;   // at e.y: side 1
                st_b[jb] = (unsigned short)bb;
                if (with_c) {
                    st_c[ja] = cid[it];
                    st_c[jb] = cid[it];
                }
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < 2 * count; j += blockDim.x) {
            const int b = st_b[j];
            const u64 g = s_gbase[b] + (u32)(j - (int)s_off[b]);
            if (g < cap) {
                p.rec_x[g] = st_x[j];
                p.rec_w[g] = st_w[j];
                if (with_c)
                    p.rec_c[g] = st_c[j];
            }
        }
        __syncthreads();   // staging and counters reused by the next tile
    }
}

// Applies the records in bucket order: chunks are claimed in increasing
// order, so the blocks work on one or two buckets at a time.
__global__ void __launch_bounds__(256) mark_apply_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    __shared__ u32 s_tile;
    const i64 total = min((i64)p.mark_base[p.mark_buckets], 2 * p.m_cap);
    const i64 chunks = (total + MB_TILE - 1) / MB_TILE;
    const i64 n = dev_count(p.d_n, p.n_cap);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_tile = atomicAdd(p.tile_counter + 2, 1u);
        __syncthreads();
        const i64 c = s_tile;
        if (c >= chunks)
            break;
        // all loads of the chunk first, then the atomics: an atomic between
        // two loads of the word array would order them (they may alias)
        u32 x[MB_TILE_ITEMS];
        u64 w[MB_TILE_ITEMS], old[MB_TILE_ITEMS];
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it) {
            const i64 j = c * MB_TILE + it * 256 + threadIdx.x;
            x[it] = 0xFFFFFFFFu;
            if (j < total) {
                x[it] = p.rec_x[j];
                w[it] = p.rec_w[j];
            }
        }
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it)
            old[it] = (i64)x[it] < n ? p.min_word[x[it]] : 0ull;
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it)
            if ((i64)x[it] < n && old[it] > w[it])
                atomicMin((unsigned long long *)(p.min_word + x[it]), (unsigned long long)w[it]);
    }
}

// Level 0 with flags: the records again in bucket order (the words of the
// bucket in progress stay in L2).  The record equal to its vertex's final
// word is the vertex's lightest incidence: it sets that endpoint's bit of the
// edge in eflag (2 bits per edge, a word array of m / 4 bytes that fits in
// L2) and writes the vertex's parent, the edge's caller id (Eq. 1).
template <bool FOREST>
__global__ void __launch_bounds__(256) mark_flags_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    __shared__ u32 s_tile;
    const i64 total = min((i64)p.mark_base[p.mark_buckets], 2 * p.m_cap);
    const i64 chunks = (total + MB_TILE - 1) / MB_TILE;
    const i64 n = dev_count(p.d_n, p.n_cap);
    const i64 m = dev_count(p.d_m, p.m_cap);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_tile = atomicAdd(p.tile_counter + 3, 1u);
        __syncthreads();
        const i64 c = s_tile;
        if (c >= chunks)
            break;
        u32 x[MB_TILE_ITEMS], cid[MB_TILE_ITEMS];
        u64 w[MB_TILE_ITEMS], cur[MB_TILE_ITEMS];
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it) {
            const i64 j = c * MB_TILE + it * 256 + threadIdx.x;
            x[it] = 0xFFFFFFFFu;
            if (j < total) {
                x[it] = p.rec_x[j];
                w[it] = p.rec_w[j];
                cid[it] = p.rec_c[j];
            }
        }
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it)
            cur[it] = (i64)x[it] < n ? p.min_word[x[it]] : NO_EDGE;
#pragma unroll
        for (int it = 0; it < MB_TILE_ITEMS; ++it) {
            if ((i64)x[it] >= n || cur[it] != w[it])
                continue;
            const u64 r = w[it] >> 32;
            if ((i64)r < m)
                atomicOr(p.eflag + (r >> 4), 1u << (2 * (u32)(r & 15) + (u32)(w[it] & 1u)));
            i32 par = (i32)cid[it];
            if (FOREST)
                par -= (i32)__ldg(p.edge_off + tree_of_edge(p.edge_off, p.n_trees, par));
            p.vertex_parent[x[it]] = par;
        }
    }
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
__global__ void __launch_bounds__(LV_THREADS) ptr_init_kernel(const LevelParams p)
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

// Level 0 keeps the supervertex in the low half of x's own word (the rank
// of x's lightest edge stays in the high half), so that compact learns both
// from one random read; higher levels keep {chain key, supervertex} records
// for the expansion, which carry the rank as well (chain key >> 1).
template <bool LEVEL0>
__device__ __forceinline__ void write_supervertex(const LevelParams &p, i64 x, i32 dense)
{
    if (LEVEL0) {
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
                write_supervertex<LEVEL0>(p, x, ~res);
                if (cur != (i32)x)
                    st_volatile(p.ptr + x, res);   // resolved: later walks stop here
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

template <bool LEVEL0>
__global__ void __launch_bounds__(LV_THREADS) compact_kernel(const LevelParams p)
{
    if (loop_closed(p))
        return;
    const i64 m = dev_count(p.d_m, p.m_cap);
    const i64 tiles = level_tiles(m);
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
                // the flags say which endpoint's word holds the supervertex
                const u32 f = eflag_of(p.eflag, r);
                if (f) {
                    p.lev[r] = (unsigned char)p.level;
                    p.start[r] = (i32)(u32)p.min_word[(f & 1u) ? e.x : e.y];
                    continue;
                }
                va = (i32)(u32)p.min_word[e.x];
                vb = (i32)(u32)p.min_word[e.y];
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

// Blocks for n elements at per_block each, capped at PANDORA_LV_BPS blocks
// per SM: every level kernel loops (grid-stride or over claimed tiles), so a
// grid sized for a worst-case bound does not launch idle blocks by the
// million.  The level kernels are bound by random DRAM reads: 8 blocks per SM
// measured 0.2 ms faster than 4 over all levels of a 10^8-edge random
// recursive tree, while the union-find part ran 20% faster at 4 blocks per SM
// than at 16 on a 10^8-vertex path (PANDORA_UF_BPS).
#ifndef PANDORA_LV_BPS
#define PANDORA_LV_BPS 8
#endif
#ifndef PANDORA_UF_BPS
#define PANDORA_UF_BPS 4
#endif
static unsigned grid_for(i64 n, int per_block, int bps = PANDORA_LV_BPS)
{
    i64 b = (n + per_block - 1) / per_block;
    const i64 cap = 152 * bps;
    if (b > cap)
        b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

void launch_init_level(const LevelParams &p, cudaStream_t s)
{
    i64 b = (p.n_grid + 255) / 256;
    if (b > 152 * 16)
        b = 152 * 16;
    init_level_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(p);
}

void launch_mark(const LevelParams &p, cudaStream_t s)
{
    if (p.mark_buckets > 0) {
        const unsigned cb = grid_for(p.m_grid, 256 * 8);
        mark_count_kernel<<<cb, 256, 0, s>>>(p);
        mark_prefix_kernel<<<1, MARK_MAX_BUCKETS, 0, s>>>(p);
        const unsigned sb = grid_for(p.m_grid, MB_TILE);
        static std::atomic<unsigned long long> attr_done{0};
        int dev = 0;
        cudaGetDevice(&dev);
        const unsigned long long bit = 1ull << (dev & 63);
        if (!(attr_done.load() & bit)) {
            cudaFuncSetAttribute(mark_scatter_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MB_SMEM_C);
            cudaFuncSetAttribute(mark_scatter_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MB_SMEM);
            attr_done.fetch_or(bit);
        }
        if (p.level == 0)
            mark_scatter_kernel<true><<<sb, 256, p.rec_c ? MB_SMEM_C : MB_SMEM, s>>>(p);
        else
            mark_scatter_kernel<false><<<sb, 256, MB_SMEM, s>>>(p);
        i64 ab = (2 * p.m_grid + MB_TILE - 1) / MB_TILE;
        if (ab > 152 * PANDORA_MARK_APPLY_BPS)
            ab = 152 * PANDORA_MARK_APPLY_BPS;
        const unsigned apply_blocks = (unsigned)(ab < 1 ? 1 : ab);
        mark_apply_kernel<<<apply_blocks, 256, 0, s>>>(p);
        if (p.level == 0 && p.eflag && p.rec_c) {
            if (p.edge_off)
                mark_flags_kernel<true><<<apply_blocks, 256, 0, s>>>(p);
            else
                mark_flags_kernel<false><<<apply_blocks, 256, 0, s>>>(p);
        }
        return;
    }
    i64 b = (p.m_grid + 255) / 256;
    if (b > 152 * PANDORA_MARK_BPS)
        b = 152 * PANDORA_MARK_BPS;
    const unsigned blocks = (unsigned)(b < 1 ? 1 : b);
    if (p.level == 0)
        mark_kernel<true><<<blocks, 256, 0, s>>>(p);
    else
        mark_kernel<false><<<blocks, 256, 0, s>>>(p);
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

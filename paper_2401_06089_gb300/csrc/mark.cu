// Marking, Eq. 1 (paper, Section 3.1): for every vertex x of a level,
// min_word[x] = (rank, other end, side) of the lightest edge at x, the
// minimum over x's incidences of a 64-bit word whose high half is the edge's
// rank.  Small levels take one 64-bit atomicMin per incidence (mark_kernel);
// levels whose word array is far above L2 group the incidences by vertex
// bucket first (bucketed marking), and level 0 adds a flag pass that
// classifies every edge for Eq. 2 and writes the vertex parents.
#include <atomic>

#include "kernels.cuh"

namespace pandora {

namespace {

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

}  // namespace

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

}  // namespace pandora

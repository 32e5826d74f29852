// Chain linking (paper, Section 3.3.3): after the stable sort by chain key
// (edges enter in ascending rank, so every chain leaves sorted by rank) an
// edge's parent is the next edge of its chain; the heaviest edge of a chain
// hangs from the chain's head edge p, and the heaviest edge of a root chain
// is the root (-1).  The result is scattered to the caller's edge order.
#include <algorithm>

#include "kernels.cuh"

#ifndef PANDORA_LINK_ITEMS
#define PANDORA_LINK_ITEMS 4
#endif
constexpr int LINK_ITEMS = PANDORA_LINK_ITEMS;

namespace pandora {

namespace {

// Section 3.3.3: inside a chain (sorted by rank) an edge's parent is the next
// edge; the chain's last edge hangs under the chain's head edge, or is the
// root (-1) for the root chain.  A thread takes LINK_ITEMS edges and issues
// all loads before its scattered stores, so the random reads of the chain
// heads overlap.
template <bool FOREST>
__global__ void __launch_bounds__(256) link_kernel(const LinkParams p)
{
    const i64 tile = (i64)blockIdx.x * 256 * LINK_ITEMS;
    u32 k[LINK_ITEMS], e[LINK_ITEMS], kn[LINK_ITEMS], en[LINK_ITEMS];
#pragma unroll
    for (int it = 0; it < LINK_ITEMS; ++it) {
        const i64 j = tile + it * 256 + threadIdx.x;
        k[it] = kn[it] = 0xFFFFFFFFu;
        e[it] = en[it] = 0;
        if (j < p.m) {
            k[it] = p.skeys[j];
            e[it] = p.svals[j];
            if (j + 1 < p.m) {
                kn[it] = p.skeys[j + 1];
                en[it] = p.svals[j + 1];
            }
        }
    }
    i32 par[LINK_ITEMS];
#pragma unroll
    for (int it = 0; it < LINK_ITEMS; ++it) {
        if (kn[it] == k[it])
            par[it] = (i32)en[it];
        else if (k[it] >= p.root_base)
            par[it] = -1;
        else
            par[it] = (i32)__ldg(p.perm + (k[it] >> 1));
    }
#pragma unroll
    for (int it = 0; it < LINK_ITEMS; ++it) {
        const i64 j = tile + it * 256 + threadIdx.x;
        if (j >= p.m)
            continue;
        i32 pr = par[it];
        if (FOREST && pr >= 0)
            pr -= (i32)__ldg(p.edge_off + tree_of_edge(p.edge_off, p.n_trees, (i64)e[it]));
        p.edge_parent[e[it]] = pr;
    }
}

// Bucketed link, for edge_parent arrays much larger than L2, where every
// scattered 4-byte store of link_kernel moves whole DRAM bursts.
//
// link_scatter: a block takes LB_TILE consecutive positions of the chain
// order, computes (caller edge id, parent) as link_kernel does, stages the
// pairs in shared memory grouped by caller-id bucket and writes each
// bucket's run contiguously at the bucket's cursor.
// link_apply: the pairs, read in bucket order, are stored to edge_parent;
// the stores of the buckets in progress fall in a range that stays in L2
// and every line of it is written whole.
constexpr int LB_ITEMS = 8;
constexpr int LB_TILE = 256 * LB_ITEMS;

template <bool FOREST>
__global__ void __launch_bounds__(256) link_scatter_kernel(const LinkParams p)
{
    __shared__ u32 s_e[LB_TILE];
    __shared__ i32 s_p[LB_TILE];
    __shared__ unsigned short s_b[LB_TILE];
    __shared__ u32 s_cnt[MARK_MAX_BUCKETS];
    __shared__ u32 s_off[MARK_MAX_BUCKETS];
    __shared__ i64 s_g[MARK_MAX_BUCKETS];
    __shared__ u32 s_warp[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const i64 t0 = (i64)blockIdx.x * LB_TILE;
    const int count = (int)min((i64)LB_TILE, p.m - t0);
    for (int b = threadIdx.x; b < MARK_MAX_BUCKETS; b += blockDim.x)
        s_cnt[b] = 0;
    u32 k[LB_ITEMS], e[LB_ITEMS], kn[LB_ITEMS], en[LB_ITEMS];
#pragma unroll
    for (int it = 0; it < LB_ITEMS; ++it) {
        const int j = it * 256 + threadIdx.x;
        k[it] = kn[it] = 0xFFFFFFFFu;
        e[it] = en[it] = 0;
        if (j < count) {
            k[it] = p.skeys[t0 + j];
            e[it] = p.svals[t0 + j];
            if (t0 + j + 1 < p.m) {
                kn[it] = p.skeys[t0 + j + 1];
                en[it] = p.svals[t0 + j + 1];
            }
        }
    }
    i32 par[LB_ITEMS];
#pragma unroll
    for (int it = 0; it < LB_ITEMS; ++it) {
        if (kn[it] == k[it])
            par[it] = (i32)en[it];
        else if (k[it] >= p.root_base)
            par[it] = -1;
        else
            par[it] = (i32)__ldg(p.perm + (k[it] >> 1));
    }
    __syncthreads();   // s_cnt zeroed
    u32 slot[LB_ITEMS];
    int bk[LB_ITEMS];
#pragma unroll
    for (int it = 0; it < LB_ITEMS; ++it) {
        const int j = it * 256 + threadIdx.x;
        bk[it] = 0;
        if (j < count) {
            if (FOREST && par[it] >= 0)
                par[it] -= (i32)__ldg(p.edge_off + tree_of_edge(p.edge_off, p.n_trees, (i64)e[it]));
            const int b = (int)(e[it] >> p.bucket_shift);
            bk[it] = b < p.n_buckets ? b : p.n_buckets - 1;
            slot[it] = atomicAdd(&s_cnt[bk[it]], 1u);
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
    for (int b = threadIdx.x; b < p.n_buckets; b += blockDim.x)
        if (s_cnt[b])
            s_g[b] = ((i64)b << p.bucket_shift) + atomicAdd(p.cursor + b, s_cnt[b]);
    __syncthreads();
#pragma unroll
    for (int it = 0; it < LB_ITEMS; ++it) {
        const int j = it * 256 + threadIdx.x;
        if (j < count) {
            const u32 pos = s_off[bk[it]] + slot[it];
            s_e[pos] = e[it];
            s_p[pos] = par[it];
            s_b[pos] = (unsigned short)bk[it];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < count; j += blockDim.x) {
        const int b = s_b[j];
        const i64 g = s_g[b] + (j - (i64)s_off[b]);
        // bucket b owns [b << shift, min(m, (b + 1) << shift)); the ids are a
        // permutation of [0, m), so g never leaves it (checked all the same)
        const i64 end = min(p.m, ((i64)b + 1) << p.bucket_shift);
        if (g < end)
            p.rec[g] = make_int2((i32)s_e[j], s_p[j]);
    }
}

__global__ void __launch_bounds__(256) link_apply_kernel(const LinkParams p)
{
    const i64 end = p.apply_end > 0 ? p.apply_end : p.m;
    const i64 i0 = p.apply_begin + (i64)blockIdx.x * (256 * 4) + threadIdx.x;
    int2 r[4];
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const i64 i = i0 + it * 256;
        r[it] = i < end ? p.rec[i] : make_int2(-1, 0);
    }
#pragma unroll
    for (int it = 0; it < 4; ++it)
        if (r[it].x >= 0 && (i64)r[it].x < p.m)
            p.edge_parent[r[it].x] = r[it].y;
}

}  // namespace

void launch_link(const LinkParams &p, cudaStream_t s)
{
    if (p.m <= 0)
        return;
    if (p.n_buckets > 0) {
        const unsigned sb = (unsigned)((p.m + LB_TILE - 1) / LB_TILE);
        if (p.edge_off)
            link_scatter_kernel<true><<<sb, 256, 0, s>>>(p);
        else
            link_scatter_kernel<false><<<sb, 256, 0, s>>>(p);
        if (p.apply_parts <= 1) {
            link_apply_kernel<<<(unsigned)((p.m + 1023) / 1024), 256, 0, s>>>(p);
            return;
        }
        // bucket ranges applied one launch after another, each followed by
        // its event (the caller copies that range of edge_parent out)
        const i64 per = (((i64)p.n_buckets + p.apply_parts - 1) / p.apply_parts) << p.bucket_shift;
        for (int k = 0; k < p.apply_parts; ++k) {
            LinkParams q = p;
            q.apply_begin = std::min(p.m, (i64)k * per);
            q.apply_end = std::min(p.m, (i64)(k + 1) * per);
            if (q.apply_end > q.apply_begin)
                link_apply_kernel<<<(unsigned)((q.apply_end - q.apply_begin + 1023) / 1024), 256, 0, s>>>(q);
            if (p.apply_done)
                cudaEventRecord(p.apply_done[k], s);
        }
        return;
    }
    const unsigned blocks = (unsigned)((p.m + 256 * LINK_ITEMS - 1) / (256 * LINK_ITEMS));
    if (p.edge_off)
        link_kernel<true><<<blocks, 256, 0, s>>>(p);
    else
        link_kernel<false><<<blocks, 256, 0, s>>>(p);
}

}  // namespace pandora

// Multilevel expansion and chain linking (paper, Sections 3.3.2 and 3.3.3).
//
// expand: an edge contracted on level l0 lies inside supervertex S of level
// l0 + 1.  Going up the levels k = l0+1, l0+2, ..., the edge belongs to the
// leaf chain hanging from p = P_k(S) (the lightest edge at S on level k,
// i.e. S's parent in the level-k dendrogram) as soon as it is lighter than
// p; otherwise S is replaced by its own supervertex on level k + 1.  An edge
// that no level claims is in the root chain.  The chain is named by the key
// 2 * rank(p) + side, where side tells which endpoint of p on level k the
// supervertex S is (a leaf edge heads two chains, one per side; the paper's
// "2L"/"13R").  Root chains get keys above every such key (one per tree).
//
// link: after a stable sort of the keys (edges enter in ascending rank, so
// every chain leaves sorted by rank) an edge's parent is the next edge of its
// chain; the heaviest edge of a chain hangs from the chain's head edge p, and
// the heaviest edge of a root chain is the root (-1).
#include "kernels.cuh"

#ifndef PANDORA_EXPAND_BPS
#define PANDORA_EXPAND_BPS 16
#endif
#ifndef PANDORA_LINK_ITEMS
#define PANDORA_LINK_ITEMS 4
#endif
constexpr int LINK_ITEMS = PANDORA_LINK_ITEMS;

namespace pandora {

namespace {

__global__ void __launch_bounds__(256) expand_kernel(const ExpandParams p, const LevelTable t)
{
    __shared__ u32 s_h[4 * RADIX];
    __shared__ i64 s_nv[MAX_LEVELS];   // vertices of every level, clamped to capacity
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x)
        s_h[i] = 0;
    for (int l = threadIdx.x; l < MAX_LEVELS; l += blockDim.x)
        s_nv[l] = l < p.max_levels ? dev_count(p.lvl_n + l, t.n_cap[l]) : 0;
    // levels actually run; 0 means the loop never met a level without
    // alpha-edges within the launched bound (only on invalid input)
    int n_levels = *p.d_n_levels;
    if (n_levels == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0)
            set_status(p.status, PANDORA_ERR_NOT_A_TREE);
        n_levels = p.max_levels;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    const i64 m_round = (p.m + 31) & ~(i64)31;
    for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r - lane < m_round; r += stride) {
        const bool valid = r < p.m;
        u32 key = 0;
        if (valid) {
            const int l0 = p.lev[r];
            i32 sv = p.start[r];
            key = NONE;
            for (int l = l0 + 1; l < n_levels; ++l) {
                if (sv < 0 || (i64)sv >= s_nv[l]) {   // only after an earlier error
                    set_status(p.status, PANDORA_ERR_NOT_A_TREE);
                    break;
                }
                const int2 rec = __ldg(t.rec[l] + sv);
                u32 c = (u32)rec.x;
                if ((u32)r < (c >> 1)) {   // an isolated supervertex (c = NONE) ends here too
                    if (c != NONE && (i64)(c >> 1) >= p.m) {   // only after an earlier error
                        set_status(p.status, PANDORA_ERR_NOT_A_TREE);
                        c = NONE;
                    }
                    key = c;
                    break;
                }
                sv = rec.y;
            }
            if (key == NONE) {
                u32 tree = 0;
                if (p.edge_off)
                    tree = (u32)tree_of_edge(p.edge_off, p.n_trees, (i64)__ldg(p.perm + r));
                key = p.root_base + tree;
            }
            p.keys_out[r] = key;
        }
        const u32 k0 = __shfl_sync(0xFFFFFFFFu, key, 0);
        const u32 vm = __ballot_sync(0xFFFFFFFFu, valid);
        const bool uniform = __all_sync(0xFFFFFFFFu, key == k0) && vm == 0xFFFFFFFFu;
        if (uniform) {
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    atomicAdd(&s_h[q * RADIX + ((key >> (8 * q)) & 255)], 32u);
            }
        } else if (valid) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                atomicAdd(&s_h[q * RADIX + ((key >> (8 * q)) & 255)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) {
        const u32 c = s_h[i];
        if (c)
            atomicAdd(p.hist + i, c);
    }
}

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
    const i64 i0 = (i64)blockIdx.x * (256 * 4) + threadIdx.x;
    int2 r[4];
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const i64 i = i0 + it * 256;
        r[it] = i < p.m ? p.rec[i] : make_int2(-1, 0);
    }
#pragma unroll
    for (int it = 0; it < 4; ++it)
        if (r[it].x >= 0 && (i64)r[it].x < p.m)
            p.edge_parent[r[it].x] = r[it].y;
}

__global__ void check_offsets_kernel(const i64 *off, i64 n_trees, i64 total, int *status)
{
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n_trees)
        return;
    const i64 o = off[t];
    bool bad = (t == 0 && o != 0) || (t == n_trees && o != total) || o < 0 || o > total;
    if (t > 0 && off[t - 1] > o)
        bad = true;
    if (bad)
        set_status(status, PANDORA_ERR_INVALID_ARGUMENT);
}

__global__ void set_u64_pair_kernel(u64 *a, u64 va, u64 *b, u64 vb)
{
    *a = va;
    *b = vb;
}

__global__ void fill_kernel(i32 *p, i64 n, i32 value)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        p[i] = value;
}

}  // namespace

void launch_expand(const ExpandParams &p, const LevelTable &t, cudaStream_t s)
{
    if (p.m <= 0)
        return;
    i64 blocks = (p.m + 256 * 8 - 1) / (256 * 8);
    if (blocks > 152 * PANDORA_EXPAND_BPS)
        blocks = 152 * PANDORA_EXPAND_BPS;
    expand_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, t);
}

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
        link_apply_kernel<<<(unsigned)((p.m + 1023) / 1024), 256, 0, s>>>(p);
        return;
    }
    const unsigned blocks = (unsigned)((p.m + 256 * LINK_ITEMS - 1) / (256 * LINK_ITEMS));
    if (p.edge_off)
        link_kernel<true><<<blocks, 256, 0, s>>>(p);
    else
        link_kernel<false><<<blocks, 256, 0, s>>>(p);
}

void launch_check_offsets(const i64 *off, i64 n_trees, i64 total, int *status, cudaStream_t s)
{
    check_offsets_kernel<<<(unsigned)((n_trees + 1 + 255) / 256), 256, 0, s>>>(off, n_trees, total,
                                                                              status);
}

void launch_set_u64_pair(u64 *a, u64 va, u64 *b, u64 vb, cudaStream_t s)
{
    set_u64_pair_kernel<<<1, 1, 0, s>>>(a, va, b, vb);
}

void launch_fill(i32 *p, i64 n, i32 value, cudaStream_t s)
{
    if (n <= 0)
        return;
    fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, value);
}

}  // namespace pandora

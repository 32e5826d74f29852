// Multilevel expansion (paper, Section 3.3.2), with the chain keys'
// digit histograms for the sort that precedes the linking (link.cu).
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
#include "kernels.cuh"

#ifndef PANDORA_EXPAND_BPS
#define PANDORA_EXPAND_BPS 16
#endif

namespace pandora {

namespace {

__global__ void __launch_bounds__(256) expand_kernel(const ExpandParams p, const LevelTable t)
{
    extern __shared__ u32 s_h[];       // the plan's histogram rows (dynamic size)
    __shared__ i64 s_nv[MAX_LEVELS];   // vertices of every level, clamped to capacity
    const int n_pass = p.plan.n;
    const int h_total = n_pass > 0 ? p.plan.off[n_pass - 1] + (1 << p.plan.width[n_pass - 1]) : 0;
    for (int i = threadIdx.x; i < h_total; i += blockDim.x)
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
        if (uniform ? lane == 0 : valid) {
            const u32 add = uniform ? 32u : 1u;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < n_pass)
                    atomicAdd(&s_h[p.plan.off[q] + ((key >> p.plan.shift[q]) & ((1u << p.plan.width[q]) - 1u))],
                              add);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < h_total; i += blockDim.x) {
        const u32 c = s_h[i];
        if (c)
            atomicAdd(p.hist + i, c);
    }
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
    const int n = p.plan.n;
    const size_t h_bytes = n > 0 ? (size_t)(p.plan.off[n - 1] + (1 << p.plan.width[n - 1])) * 4 : 4;
    expand_kernel<<<(unsigned)blocks, 256, h_bytes, s>>>(p, t);
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

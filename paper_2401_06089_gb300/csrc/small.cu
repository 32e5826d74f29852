// Single-CTA solver: the whole method for one small tree in shared memory.
//
// For a tree of at most SMALL_CAP edges one thread block runs every step of
// Algorithm 1 -- the (weight, index) sort (Section 3.1), the contraction levels
// (Eq. 1, Eq. 2, Section 3.2), the expansion (Section 3.3.2), the chain sort
// and the linking (Section 3.3.3) -- with __syncthreads() where the large path
// has kernel boundaries.  Every array lives in shared memory, so a small tree
// costs one launch and no DRAM traffic beyond its inputs and outputs.  In
// batched mode one block takes one tree; trees above the block's capacity (or
// the caller's cutoff) are left to the forest pipeline.
//
// With m <= 4096 every rank fits 12 bits and every vertex id 13 bits, so the
// lightest-incident-edge word packs (rank, other endpoint, side) into 32 bits
// and the sorts run on 64- and 32-bit composite keys that are unique (the
// index is part of the key), which a bitonic network sorts correctly without
// a stability requirement.  The shared-memory layout is sized by a capacity
// CAP (256, 1024 or 4096 edges: about 9, 35 and 137 KB), so that blocks of
// small trees do not hold the largest layout and several fit one SM.
#include <atomic>

#include "kernels.cuh"

namespace pandora {

namespace {

constexpr int SMALL_CAP = 4096;          // edges
constexpr u32 W_NONE = 0xFFFFFFFFu;
constexpr u32 CK_NONE = 0x3FFFu;         // chain key of a vertex without edges

template <int CAP> struct SmallSmem {
    unsigned long long sort64[CAP];        // sort 1 keys; sort 2 reuses it as u32
    unsigned short ea[CAP], eb[CAP];       // endpoints of the current level
    unsigned short er[CAP];                // global rank of each current edge
    unsigned short na[CAP / 2], nb[CAP / 2], nr[CAP / 2];  // next level
    unsigned short perm[CAP];              // rank -> caller edge index
    u32 word[CAP + 1];                     // (rank << 14 | other << 1 | side)
    short ptr[CAP + 1];                    // pointer forest; ~dense id at roots
    unsigned short vmap[CAP + 1];
    u32 rec[CAP + 64];                     // levels >= 1: ck << 13 | vmap
    unsigned short rec_off[16];
    unsigned char lev[CAP];
    unsigned short start[CAP];
    u32 warp_tot[32];
    u32 counts[4];
};

template <int T>
__device__ __forceinline__ void bitonic_sort_u64(unsigned long long *a, int n_pow2)
{
    for (int k = 2; k <= n_pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pow2; i += T) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <int T>
__device__ __forceinline__ void bitonic_sort_u32(u32 *a, int n_pow2)
{
    for (int k = 2; k <= n_pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pow2; i += T) {
                const int l = i ^ j;
                if (l > i) {
                    const u32 x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Exclusive ranks of flagged items 0..n-1 in index order.  Thread t owns the
// contiguous items [t*per, (t+1)*per); returns the rank of its first item and
// the total (in s->counts[slot]).
template <int T, class S>
__device__ __forceinline__ u32 block_rank_start(S *s, u32 local, int slot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off)
            incl += y;
    }
    if (lane == 31)
        s->warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const u32 own = lane < T / 32 ? s->warp_tot[lane] : 0u;
        u32 t = own;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const u32 y = __shfl_up_sync(0xFFFFFFFFu, t, off);
            if (lane >= off)
                t += y;
        }
        if (lane < T / 32)
            s->warp_tot[lane] = t - own;
        if (lane == 31)
            s->counts[slot] = t;
    }
    __syncthreads();
    return s->warp_tot[warp] + incl - local;
}

template <int T, int CAP>
__global__ void __launch_bounds__(T) small_tree_kernel(const SmallParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem<CAP> *s = (SmallSmem<CAP> *)smem_raw;
    const int tid = threadIdx.x;

    // ---- which tree --------------------------------------------------------
    i64 e0 = 0, m64 = p.m;
    i64 t = 0;
    if (p.edge_off) {
        t = p.tree_list ? p.tree_list[blockIdx.x] : (i64)blockIdx.x;
        if (t < 0 || t >= p.n_trees)
            return;   // only after a plan mismatch, which is reported
        e0 = p.edge_off[t];
        m64 = p.edge_off[t + 1] - e0;
        if (e0 < 0 || m64 < 0 || e0 + m64 > p.total_edges) {
            if (tid == 0)
                set_status(p.status, PANDORA_ERR_INVALID_ARGUMENT);
            return;
        }
    }
    if (m64 > p.cutoff || m64 > CAP) {
        // the host sends only trees within both bounds
        if (tid == 0)
            set_status(p.status, PANDORA_ERR_INVALID_ARGUMENT);
        return;
    }
    const int m = (int)m64;
    const int n = m + 1;
    const i32 *u = p.u + e0;
    const i32 *v = p.v + e0;
    const float *w = p.w + e0;
    i32 *ep = p.edge_parent + e0;
    i32 *vp = p.vertex_parent + e0 + t;
    if (m == 0) {
        if (tid == 0)
            vp[0] = -1;
        return;
    }
    int P = 1;
    while (P < m)
        P <<= 1;

    // ---- 1. sort by (weight, index), Section 3.1 ------------------------------
    bool bad_nan = false, bad_range = false, bad_loop = false;
    for (int e = tid; e < P; e += T) {
        if (e < m) {
            const float x = w[e];
            bad_nan |= (x != x);
            const i32 a = u[e], b = v[e];
            bad_range |= (a < 0 || a >= n || b < 0 || b >= n);
            bad_loop |= (a == b);
            s->ea[e] = (unsigned short)(a < 0 || a >= n ? 0 : a);
            s->eb[e] = (unsigned short)(b < 0 || b >= n ? 0 : b);
            s->sort64[e] = ((unsigned long long)weight_key(x) << 32) | (u32)e;
        } else {
            s->sort64[e] = ~0ull;
        }
    }
    if (bad_nan)
        set_status(p.status, PANDORA_ERR_NAN_WEIGHT);
    if (bad_range)
        set_status(p.status, PANDORA_ERR_VERTEX_OUT_OF_RANGE);
    if (bad_loop && !bad_range)
        set_status(p.status, PANDORA_ERR_SELF_LOOP);
    __syncthreads();
    bitonic_sort_u64<T>(s->sort64, P);
    // endpoints into rank order (through registers: caller order -> rank order)
    {
        constexpr int PER = (CAP + T - 1) / T;
        unsigned short ra[PER], rb[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int r = k * T + tid;
            if (r < m) {
                const int e = (int)(u32)s->sort64[r];
                ra[k] = s->ea[e];
                rb[k] = s->eb[e];
                s->perm[r] = (unsigned short)e;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int r = k * T + tid;
            if (r < m) {
                s->ea[r] = ra[k];
                s->eb[r] = rb[k];
                s->er[r] = (unsigned short)r;
            }
        }
    }
    __syncthreads();

    // ---- 2. contraction levels, Section 3.2 ----------------------------------
    int ml = m, nl = n, level = 0, n_levels = 0, rec_used = 0;
    for (;;) {
        if (level >= 15) {
            set_status(p.status, PANDORA_ERR_NOT_A_TREE);
            return;
        }
        // Eq. 1: lightest incident edge word of every vertex
        for (int x = tid; x < nl; x += T)
            s->word[x] = W_NONE;
        __syncthreads();
        for (int i = tid; i < ml; i += T) {
            const u32 r = s->er[i], a = s->ea[i], b = s->eb[i];
            atomicMin(&s->word[a], (r << 14) | (b << 1));
            atomicMin(&s->word[b], (r << 14) | (a << 1) | 1u);
        }
        __syncthreads();
        // pointer forest; roots = smaller endpoint of each leaf edge
        const int vper = (nl + T - 1) / T;
        const int v0 = tid * vper;
        u32 local = 0;
        for (int x = v0; x < v0 + vper && x < nl; ++x) {
            const u32 wx = s->word[x];
            bool root;
            if (wx == W_NONE) {
                root = true;
            } else {
                const u32 y = (wx >> 1) & 0x1FFFu;
                root = ((s->word[y] >> 14) == (wx >> 14)) && ((u32)x < y);
                if (level == 0)
                    vp[x] = (i32)s->perm[wx >> 14];   // Eq. 1, caller edge index
            }
            local += root ? 1u : 0u;
        }
        u32 rank = block_rank_start<T>(s, local, 0);
        const int n_next = (int)s->counts[0];
        for (int x = v0; x < v0 + vper && x < nl; ++x) {
            const u32 wx = s->word[x];
            const u32 y = (wx >> 1) & 0x1FFFu;
            const bool root = wx == W_NONE ||
                              (((s->word[y] >> 14) == (wx >> 14)) && ((u32)x < y));
            s->ptr[x] = root ? (short)~(int)rank++ : (short)y;
        }
        __syncthreads();
        // root finding (path halving; every wait is bounded by the level size)
        for (int x = tid; x < nl; x += T) {
            int cur = x, res = ~0;
            volatile short *vptr = s->ptr;
            for (int it = 0; it <= nl; ++it) {
                const int pc = vptr[cur];
                if (pc < 0) {
                    res = pc;
                    break;
                }
                const int g = vptr[pc];
                if (g < 0) {
                    res = g;
                    break;
                }
                vptr[cur] = (short)g;   // path halving: g is an ancestor of cur
                cur = g;
            }
            s->vmap[x] = (unsigned short)~res;
        }
        __syncthreads();
        if (level > 0) {
            for (int x = tid; x < nl; x += T) {
                const u32 wx = s->word[x];
                const u32 ck = wx == W_NONE ? CK_NONE : 2u * (wx >> 14) + (wx & 1u);
                s->rec[rec_used + x] = (ck << 13) | s->vmap[x];
            }
            if (tid == 0)
                s->rec_off[level] = (unsigned short)rec_used;
            rec_used += nl;
        }
        // Eq. 2: alpha-edges go to the next level, the others are contracted here
        const int eper = (ml + T - 1) / T;
        const int i0 = tid * eper;
        local = 0;
        for (int i = i0; i < i0 + eper && i < ml; ++i) {
            const u32 r = s->er[i];
            const bool alpha = (s->word[s->ea[i]] >> 14) != r && (s->word[s->eb[i]] >> 14) != r;
            local += alpha ? 1u : 0u;
        }
        rank = block_rank_start<T>(s, local, 1);
        const int m_next = (int)s->counts[1];
        for (int i = i0; i < i0 + eper && i < ml; ++i) {
            const u32 r = s->er[i];
            const int a = s->ea[i], b = s->eb[i];
            const bool alpha = (s->word[a] >> 14) != r && (s->word[b] >> 14) != r;
            if (alpha) {
                if (s->vmap[a] == s->vmap[b])
                    set_status(p.status, PANDORA_ERR_NOT_A_TREE);
                if (rank < CAP / 2) {
                    s->na[rank] = s->vmap[a];
                    s->nb[rank] = s->vmap[b];
                    s->nr[rank] = (unsigned short)r;
                }
                ++rank;
            } else {
                s->lev[r] = (unsigned char)level;
                s->start[r] = s->vmap[a];
            }
        }
        __syncthreads();
        n_levels = level + 1;
        if (n_next != m_next + 1 || m_next > CAP / 2 || rec_used + n_next > CAP + 64) {
            set_status(p.status, PANDORA_ERR_NOT_A_TREE);
            return;
        }
        if (m_next == 0)
            break;
        for (int i = tid; i < m_next; i += T) {
            s->ea[i] = s->na[i];
            s->eb[i] = s->nb[i];
            s->er[i] = s->nr[i];
        }
        __syncthreads();
        ml = m_next;
        nl = n_next;
        ++level;
    }

    // ---- 3. expansion, Section 3.3.2: chain key of every edge ------------------
    u32 *sort32 = (u32 *)s->sort64;
    const u32 root_key = 2u * (u32)m;
    for (int r = tid; r < P; r += T) {
        u32 key = root_key;
        if (r < m) {
            int sv = s->start[r];
            for (int l = s->lev[r] + 1; l < n_levels; ++l) {
                const u32 rc = s->rec[s->rec_off[l] + sv];
                const u32 c = rc >> 13;
                if ((u32)r < (c >> 1)) {   // an isolated supervertex ends here too
                    if ((c >> 1) < (u32)m)
                        key = c;
                    else if (c != CK_NONE)   // only after an earlier error
                        set_status(p.status, PANDORA_ERR_NOT_A_TREE);
                    break;
                }
                sv = (int)(rc & 0x1FFFu);
            }
            sort32[r] = (key << 12) | (u32)r;
        } else {
            sort32[r] = ~0u;
        }
    }
    __syncthreads();

    // ---- 4. chains sorted, linked and stitched, Section 3.3.3 ----------------
    bitonic_sort_u32<T>(sort32, P);
    for (int j = tid; j < m; j += T) {
        const u32 c = sort32[j];
        const u32 key = c >> 12;
        const int e = s->perm[c & 0xFFFu];
        i32 par;
        if (j + 1 < m && (sort32[j + 1] >> 12) == key)
            par = (i32)s->perm[sort32[j + 1] & 0xFFFu];
        else if (key == root_key)
            par = -1;
        else
            par = (i32)s->perm[key >> 1];
        ep[e] = par;
    }
}

// The opt-in to more than 48 KB of dynamic shared memory is per device; a
// bit mask remembers the devices done.
template <int T, int CAP>
void launch_small_t(const SmallParams &p, unsigned blocks, cudaStream_t s)
{
    const int bytes = (int)sizeof(SmallSmem<CAP>);
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        cudaFuncSetAttribute(small_tree_kernel<T, CAP>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        done.fetch_or(bit);
    }
    small_tree_kernel<T, CAP><<<blocks, T, bytes, s>>>(p);
}

template <int CAP>
void launch_small_cap(const SmallParams &p, int threads, unsigned blocks, cudaStream_t s)
{
    switch (threads) {
    case 256: launch_small_t<256, CAP>(p, blocks, s); break;
    case 1024: launch_small_t<1024, CAP>(p, blocks, s); break;
    default: launch_small_t<512, CAP>(p, blocks, s); break;
    }
}

// ---- the last levels of a single tree in one block ---------------------------
struct TailSmem {
    unsigned short ea[TAIL_CAP], eb[TAIL_CAP];   // endpoints (level ids < n <= TAIL_CAP + 1)
    u32 er[TAIL_CAP];                            // global ranks
    unsigned short na[TAIL_CAP / 2], nb[TAIL_CAP / 2];
    u32 nr[TAIL_CAP / 2];
    u32 word[TAIL_CAP + 1];                      // (local index << 14 | other << 1 | side)
    short ptr[TAIL_CAP + 1];
    unsigned short vmap[TAIL_CAP + 1];
    u32 warp_tot[32];
    u32 counts[4];
};

// Edges of a level are listed in ascending global rank, so a local index
// orders them as the rank does and the lightest-edge word fits 32 bits.
__global__ void __launch_bounds__(1024) tail_levels_kernel(const TailParams p)
{
    constexpr int T = 1024;
    if (*(const volatile int *)p.d_n_levels != 0)
        return;   // the loop ended on an earlier level
    extern __shared__ __align__(16) unsigned char tail_raw[];
    TailSmem *s = (TailSmem *)tail_raw;
    const int tid = threadIdx.x;
    const i64 m64 = (i64)p.d_m[p.level];
    if (m64 > TAIL_CAP || m64 < 0 || m64 > p.ab_cap) {
        if (tid == 0)
            set_status(p.status, PANDORA_ERR_NOT_A_TREE);   // more than the bound allows
        return;
    }
    int ml = (int)m64, nl = ml + 1;
    for (int i = tid; i < ml; i += T) {
        const int2 e = p.ab[i];
        const bool ok = e.x >= 0 && e.x < nl && e.y >= 0 && e.y < nl;
        s->ea[i] = (unsigned short)(ok ? e.x : 0);
        s->eb[i] = (unsigned short)(ok ? e.y : 0);
        s->er[i] = p.er[i];
        if (!ok)
            set_status(p.status, PANDORA_ERR_NOT_A_TREE);
    }
    __syncthreads();
    for (int k = 0;; ++k) {
        const int level = p.level + k;
        if (k >= TAIL_MAX_LEVELS || level >= p.max_levels || (i64)nl > p.rec_cap[k]) {
            if (tid == 0)
                set_status(p.status, PANDORA_ERR_NOT_A_TREE);   // beyond Section 4.2's bound
            return;
        }
        if (tid == 0) {
            p.lvl_m[level] = (u64)ml;
            p.lvl_n[level] = (u64)nl;
        }
        // Eq. 1
        for (int x = tid; x < nl; x += T)
            s->word[x] = W_NONE;
        __syncthreads();
        for (int i = tid; i < ml; i += T) {
            const u32 a = s->ea[i], b = s->eb[i];
            atomicMin(&s->word[a], ((u32)i << 14) | (b << 1));
            atomicMin(&s->word[b], ((u32)i << 14) | (a << 1) | 1u);
        }
        __syncthreads();
        // pointer forest, roots with dense ids in vertex order
        const int vper = (nl + T - 1) / T;
        const int v0 = tid * vper;
        u32 local = 0;
        for (int x = v0; x < v0 + vper && x < nl; ++x) {
            const u32 wx = s->word[x];
            const u32 y = (wx >> 1) & 0x1FFFu;
            const bool root = wx == W_NONE || (((s->word[y] >> 14) == (wx >> 14)) && ((u32)x < y));
            local += root ? 1u : 0u;
        }
        u32 rank = block_rank_start<T>(s, local, 0);
        const int n_next = (int)s->counts[0];
        for (int x = v0; x < v0 + vper && x < nl; ++x) {
            const u32 wx = s->word[x];
            const u32 y = (wx >> 1) & 0x1FFFu;
            const bool root = wx == W_NONE || (((s->word[y] >> 14) == (wx >> 14)) && ((u32)x < y));
            s->ptr[x] = root ? (short)~(int)rank++ : (short)y;
        }
        __syncthreads();
        for (int x = tid; x < nl; x += T) {
            int cur = x, res = ~0;
            volatile short *vptr = s->ptr;
            for (int it = 0; it <= nl; ++it) {
                const int pc = vptr[cur];
                if (pc < 0) {
                    res = pc;
                    break;
                }
                const int g = vptr[pc];
                if (g < 0) {
                    res = g;
                    break;
                }
                vptr[cur] = (short)g;
                cur = g;
            }
            s->vmap[x] = (unsigned short)~res;
        }
        __syncthreads();
        // the records the expansion walks: {2 * rank + side of x's lightest
        // edge, x's supervertex on the next level}
        for (int x = tid; x < nl; x += T) {
            const u32 wx = s->word[x];
            const u32 ck = wx == W_NONE ? NONE : 2u * s->er[wx >> 14] + (wx & 1u);
            p.rec[k][x] = make_int2((i32)ck, (i32)s->vmap[x]);
        }
        // Eq. 2: alpha-edges go on, the others are contracted on this level
        const int eper = (ml + T - 1) / T;
        const int i0 = tid * eper;
        local = 0;
        for (int i = i0; i < i0 + eper && i < ml; ++i) {
            const bool alpha = (s->word[s->ea[i]] >> 14) != (u32)i &&
                               (s->word[s->eb[i]] >> 14) != (u32)i;
            local += alpha ? 1u : 0u;
        }
        rank = block_rank_start<T>(s, local, 1);
        const int m_next = (int)s->counts[1];
        for (int i = i0; i < i0 + eper && i < ml; ++i) {
            const int a = s->ea[i], b = s->eb[i];
            const bool alpha = (s->word[a] >> 14) != (u32)i && (s->word[b] >> 14) != (u32)i;
            if (alpha) {
                if (s->vmap[a] == s->vmap[b])
                    set_status(p.status, PANDORA_ERR_NOT_A_TREE);
                if (rank < TAIL_CAP / 2) {
                    s->na[rank] = s->vmap[a];
                    s->nb[rank] = s->vmap[b];
                    s->nr[rank] = s->er[i];
                }
                ++rank;
            } else {
                p.lev[s->er[i]] = (unsigned char)level;
                p.start[s->er[i]] = (i32)s->vmap[a];
            }
        }
        __syncthreads();
        if (n_next != m_next + 1 || m_next > TAIL_CAP / 2) {
            if (tid == 0)
                set_status(p.status, PANDORA_ERR_NOT_A_TREE);
            return;
        }
        if (m_next == 0) {
            if (tid == 0) {
                p.lvl_m[level + 1] = 0;
                p.lvl_n[level + 1] = 1;
                *p.d_n_levels = level + 1;
            }
            return;
        }
        for (int i = tid; i < m_next; i += T) {
            s->ea[i] = s->na[i];
            s->eb[i] = s->nb[i];
            s->er[i] = s->nr[i];
        }
        __syncthreads();
        ml = m_next;
        nl = n_next;
    }
}

// Copies the edges of the trees in `list` into a packed forest (offsets
// `coff`): one thread per packed edge (a binary search over coff finds its
// tree), so a few large trees still spread over the whole GPU.
__global__ void __launch_bounds__(256) gather_trees_kernel(const i32 *u, const i32 *v, const float *w,
                                                           const i64 *off, i64 n_trees, i64 total,
                                                           const i32 *list, const i64 *coff,
                                                           i64 n_list, i64 packed_total, i32 *cu,
                                                           i32 *cv, float *cw)
{
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < packed_total;
         j += (i64)gridDim.x * blockDim.x) {
        const i64 k = tree_of_edge(coff, n_list, j);
        const i64 t = list[k];
        if (t < 0 || t >= n_trees)
            continue;   // only after a plan mismatch, which is reported
        const i64 e0 = off[t], m = off[t + 1] - e0, c0 = coff[k];
        const i64 i = j - c0;
        if (e0 < 0 || m < 0 || e0 + m > total || i < 0 || i >= m)
            continue;
        cu[j] = u[e0 + i];
        cv[j] = v[e0 + i];
        cw[j] = w[e0 + i];
    }
}

// Copies the packed forest's outputs back to the trees' own positions (ids are
// tree-local on both sides): one thread per packed edge for edge_parent, one
// per packed vertex for vertex_parent (packed tree k has vertices
// [coff[k] + k, coff[k+1] + k + 1)).
__global__ void __launch_bounds__(256) scatter_trees_kernel(const i32 *cep, const i32 *cvp,
                                                            const i64 *off, i64 n_trees, i64 total,
                                                            const i32 *list, const i64 *coff,
                                                            i64 n_list, i64 packed_total, i32 *ep,
                                                            i32 *vp)
{
    const i64 stride = (i64)gridDim.x * blockDim.x;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < packed_total; j += stride) {
        const i64 k = tree_of_edge(coff, n_list, j);
        const i64 t = list[k];
        if (t < 0 || t >= n_trees)
            continue;
        const i64 e0 = off[t], m = off[t + 1] - e0, i = j - coff[k];
        if (e0 < 0 || m < 0 || e0 + m > total || i < 0 || i >= m)
            continue;
        ep[e0 + i] = cep[j];
    }
    for (i64 x = (i64)blockIdx.x * blockDim.x + threadIdx.x; x < packed_total + n_list;
         x += stride) {
        // tree k holds x when coff[k] + k <= x < coff[k + 1] + k + 1
        i64 lo = 0, hi = n_list - 1;
        while (lo < hi) {
            const i64 mid = (lo + hi + 1) >> 1;
            if (__ldg(coff + mid) + mid <= x)
                lo = mid;
            else
                hi = mid - 1;
        }
        const i64 k = lo;
        const i64 t = list[k];
        if (t < 0 || t >= n_trees)
            continue;
        const i64 e0 = off[t], m = off[t + 1] - e0, i = x - (coff[k] + k);
        if (e0 < 0 || m < 0 || e0 + m > total || i < 0 || i > m)
            continue;
        vp[e0 + t + i] = cvp[x];
    }
}

// One block of 1024 threads walks the trees in order, 1024 at a time: per
// class a warp ballot ranks the trees of the chunk, so every class list keeps
// tree order (stable), and a warp scan over the large trees' sizes gives
// their packed offsets.
__global__ void __launch_bounds__(1024) plan_kernel(const PlanParams p)
{
    __shared__ u32 s_cnt[32][N_CLASSES];
    __shared__ u32 s_tot[N_CLASSES];
    __shared__ i64 s_run[N_CLASSES];
    __shared__ i64 s_wm[32];
    __shared__ i64 s_edges, s_chunk_edges;
    __shared__ int s_bad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < N_CLASSES)
        s_run[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_edges = 0;
        s_bad = 0;
    }
    __syncthreads();
    for (i64 c0 = 0; c0 < p.n_trees; c0 += 1024) {
        const i64 t = c0 + threadIdx.x;
        int cls = -1;
        i64 m = 0;
        if (t < p.n_trees) {
            m = p.off[t + 1] - p.off[t];
            cls = size_class(m < 0 ? p.total_edges + 1 : m, p.cutoff);
        }
        u32 my_rank = 0;
#pragma unroll
        for (int c = 0; c < N_CLASSES; ++c) {
            const u32 mask = __ballot_sync(0xFFFFFFFFu, cls == c);
            if (cls == c)
                my_rank = __popc(mask & lanemask_lt());
            if (lane == 0)
                s_cnt[warp][c] = __popc(mask);
        }
        const i64 em = cls == CLASS_LARGE ? m : 0;
        i64 incl = em;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const i64 y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            s_wm[warp] = incl;
        __syncthreads();
        if (threadIdx.x < N_CLASSES) {
            u32 acc = 0;
            for (int w = 0; w < 32; ++w) {
                const u32 x = s_cnt[w][threadIdx.x];
                s_cnt[w][threadIdx.x] = acc;
                acc += x;
            }
            s_tot[threadIdx.x] = acc;
        } else if (threadIdx.x == 32) {
            i64 acc = 0;
            for (int w = 0; w < 32; ++w) {
                const i64 x = s_wm[w];
                s_wm[w] = acc;
                acc += x;
            }
            s_chunk_edges = acc;
        }
        __syncthreads();
        if (cls >= 0) {
            const i64 pos = s_run[cls] + s_cnt[warp][cls] + my_rank;
            if (pos < p.count[cls]) {
                p.lists[p.base[cls] + pos] = (i32)t;
                if (cls == CLASS_LARGE)
                    p.coff[pos] = s_edges + s_wm[warp] + incl - em;
            } else {
                s_bad = 1;
            }
        }
        __syncthreads();
        if (threadIdx.x < N_CLASSES)
            s_run[threadIdx.x] += s_tot[threadIdx.x];
        else if (threadIdx.x == 32)
            s_edges += s_chunk_edges;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bool bad = s_bad != 0 || s_edges != p.m_large;
        for (int c = 0; c < N_CLASSES; ++c)
            bad = bad || s_run[c] != p.count[c];
        if (bad)   // list slots not written keep the host's fill (-1: no tree)
            set_status(p.status, PANDORA_ERR_INVALID_ARGUMENT);
        p.coff[p.count[CLASS_LARGE]] = p.m_large;
    }
}

// A plan error overrides what the kernels found after it: those ran on a
// plan the device offsets do not follow.
__global__ void merge_status_kernel(const int *from, int *to)
{
    if (threadIdx.x == 0 && *from != 0)
        *to = *from;
}

}  // namespace

int small_tree_capacity() { return SMALL_CAP; }

int small_layout_capacity(i64 max_edges)
{
    return max_edges < 256 ? 256 : max_edges < 1024 ? 1024 : SMALL_CAP;
}

void launch_tail(const TailParams &p, cudaStream_t s)
{
    const int bytes = (int)sizeof(TailSmem);
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        cudaFuncSetAttribute(tail_levels_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
        done.fetch_or(bit);
    }
    tail_levels_kernel<<<1, 1024, bytes, s>>>(p);
}

void launch_plan(const PlanParams &p, cudaStream_t s)
{
    plan_kernel<<<1, 1024, 0, s>>>(p);
}

void launch_merge_status(const int *from, int *to, cudaStream_t s)
{
    merge_status_kernel<<<1, 32, 0, s>>>(from, to);
}

void launch_gather_trees(const i32 *u, const i32 *v, const float *w, const i64 *off, i64 n_trees,
                         i64 total, const i32 *list, const i64 *coff, i64 n_list, i64 packed_total,
                         i32 *cu, i32 *cv, float *cw, cudaStream_t s)
{
    if (n_list <= 0)
        return;
    const i64 b = (packed_total + 255) / 256;
    const unsigned blocks = (unsigned)(b < 1 ? 1 : b < 152 * 16 ? b : 152 * 16);
    gather_trees_kernel<<<blocks, 256, 0, s>>>(u, v, w, off, n_trees, total, list, coff, n_list,
                                               packed_total, cu, cv, cw);
}

void launch_scatter_trees(const i32 *cep, const i32 *cvp, const i64 *off, i64 n_trees, i64 total,
                          const i32 *list, const i64 *coff, i64 n_list, i64 packed_total, i32 *ep,
                          i32 *vp, cudaStream_t s)
{
    if (n_list <= 0)
        return;
    const i64 b = (packed_total + n_list + 255) / 256;
    const unsigned blocks = (unsigned)(b < 1 ? 1 : b < 152 * 16 ? b : 152 * 16);
    scatter_trees_kernel<<<blocks, 256, 0, s>>>(cep, cvp, off, n_trees, total, list, coff, n_list,
                                                packed_total, ep, vp);
}

void launch_small(const SmallParams &p, int threads, i64 max_edges, unsigned blocks,
                  cudaStream_t s)
{
    if (blocks == 0)
        return;
    switch (small_layout_capacity(max_edges)) {
    case 256: launch_small_cap<256>(p, threads, blocks, s); break;
    case 1024: launch_small_cap<1024>(p, threads, blocks, s); break;
    default: launch_small_cap<SMALL_CAP>(p, threads, blocks, s); break;
    }
}

}  // namespace pandora

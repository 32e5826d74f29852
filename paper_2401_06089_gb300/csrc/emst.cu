// Mutual-reachability minimum spanning tree of 3-D points
// (include/pandora_emst.h; the step before the dendrogram in the HDBSCAN*
// pipeline of the paper, Section 6.5).
//
//   1. bounding box, 30-bit Morton codes, sort of (code, point id) with the
//      library's onesweep radix sort
//   2. linear BVH over the sorted points (Karras 2012): internal node i
//      spans the key range whose longest common prefix it owns; equal codes
//      are told apart by their position
//   3. bottom-up refit: every internal node keeps, for each of its two
//      children, the box, the least core2 below it and the component of
//      its points when they all share one (else -1), so that a traversal
//      step reads one 64-byte record and needs no point record for a leaf
//   4. core2 of every point: k nearest points by a best-first traversal with
//      the k smallest squared distances in a sorted list
//   5. Boruvka rounds: every point finds its least edge, in the (mr2, smaller
//      id, larger id) order, to a point of another component, skipping
//      subtrees of its own component and subtrees whose lower bound is above
//      the component's least edge found so far; each component keeps its
//      least edge (two atomic minima: weight, then the id pair), links to the
//      component across it, and pointer jumping relabels the points
//
// Every lower bound is computed with the same float32 operations, in the
// same order, as the distances it bounds, so rounding can never make a bound
// exceed a distance it stands for (round-to-nearest is monotone): the result
// is the exact minimum spanning tree of the float32 reading.
#include <algorithm>
#include <vector>

#include "kernels.cuh"
#include "../../include/pandora_emst.h"

namespace pandora {

cudaMemPool_t flat_pool(int dev);   // the library's stream-ordered pool

namespace {

constexpr int EM_K_MAX = PANDORA_EMST_MAX_MIN_PTS;
constexpr int EM_STACK = 64;
constexpr int EM_MAX_ROUNDS = 64;
constexpr int EM_REFIT_DEPTH = 256;
constexpr u32 INF_BITS = 0x7F800000u;

struct EmCtrl {
    int status;
    int changed;           // pointer jumping: a parent moved in the last pass
    u64 n_edges;           // tree edges found so far
    u32 lo_key[3];         // bounding box as order-preserving keys
    u32 hi_key[3];
    u32 hist[4][RADIX];
    u32 base[4][RADIX];
    u32 tile_counter;
};

__device__ __forceinline__ float key_to_float(u32 k)
{
    const u32 b = k ^ ((k & 0x80000000u) ? 0x80000000u : 0xFFFFFFFFu);
    return __uint_as_float(b);
}

// d2 of the float32 reading: ((dx*dx + dy*dy) + dz*dz), no contraction
__device__ __forceinline__ float em_d2(float4 a, float4 b)
{
    const float dx = __fsub_rn(b.x, a.x), dy = __fsub_rn(b.y, a.y), dz = __fsub_rn(b.z, a.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Lower bound of em_d2(q, p) over the points p of a box: the per-axis gap is
// a float32 difference with the box face, which by monotone rounding is at
// most the difference with any point inside; the squares and sums follow the
// distance's own order.
__device__ __forceinline__ float em_box_d2(float4 q, float4 lo, float4 hi)
{
    const float gx = q.x < lo.x ? __fsub_rn(lo.x, q.x) : (q.x > hi.x ? __fsub_rn(q.x, hi.x) : 0.f);
    const float gy = q.y < lo.y ? __fsub_rn(lo.y, q.y) : (q.y > hi.y ? __fsub_rn(q.y, hi.y) : 0.f);
    const float gz = q.z < lo.z ? __fsub_rn(lo.z, q.z) : (q.z > hi.z ? __fsub_rn(q.z, hi.z) : 0.f);
    return __fadd_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)), __fmul_rn(gz, gz));
}

__device__ __forceinline__ u32 spread10(u32 x)
{
    x &= 1023u;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// ---- 1. box, Morton codes, Morton-ordered points -----------------------------
__global__ void __launch_bounds__(256) em_bbox_kernel(const float *__restrict__ pts, i64 n,
                                                      EmCtrl *c)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (i64)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float x = pts[3 * i + d];
            bad |= !isfinite(x);
            lo[d] = fminf(lo[d], x);
            hi[d] = fmaxf(hi[d], x);
        }
    }
    if (bad)
        set_status(&c->status, PANDORA_ERR_BAD_POINT);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xFFFFFFFFu, lo[d], o));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xFFFFFFFFu, hi[d], o));
        }
        if ((threadIdx.x & 31) == 0 && lo[d] <= hi[d]) {
            atomicMin(&c->lo_key[d], weight_key(lo[d]));
            atomicMax(&c->hi_key[d], weight_key(hi[d]));
        }
    }
}

__global__ void __launch_bounds__(256) em_morton_kernel(const float *__restrict__ pts, i64 n,
                                                        const EmCtrl *c, u32 *codes, u32 *ids)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    u32 code = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float lo = key_to_float(c->lo_key[d]), hi = key_to_float(c->hi_key[d]);
        const float ext = hi - lo;
        float t = ext > 0.f ? (pts[3 * i + d] - lo) / ext * 1024.f : 0.f;
        t = fminf(fmaxf(t, 0.f), 1023.f);
        code |= spread10((u32)t) << (2 - d);
    }
    codes[i] = code;
    ids[i] = (u32)i;
}

__global__ void __launch_bounds__(256) em_gather_kernel(const float *__restrict__ pts, i64 n,
                                                        const u32 *ids, float4 *P4, i32 *pos_of,
                                                        i32 *comp)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const u32 id = ids[i];
    P4[i] = make_float4(pts[3 * (i64)id], pts[3 * (i64)id + 1], pts[3 * (i64)id + 2], 0.f);
    pos_of[id] = (i32)i;
    comp[i] = (i32)i;
}

// ---- 2. linear BVH (Karras 2012) ----------------------------------------------
// Node ids: internal nodes 0 .. n-2 (0 is the root), leaf j is n - 1 + j.
__device__ __forceinline__ int em_delta(const u32 *__restrict__ k, i64 n, i64 i, i64 j)
{
    if (j < 0 || j >= n)
        return -1;
    const u32 a = k[i], b = k[j];
    if (a != b)
        return __clz(a ^ b);
    return 32 + __clz((u32)i ^ (u32)j);
}

__global__ void __launch_bounds__(256) em_build_kernel(const u32 *__restrict__ k, i64 n,
                                                       int2 *kids, int *parent)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1)
        return;
    const int d = (em_delta(k, n, i, i + 1) - em_delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = em_delta(k, n, i, i - d);
    i64 lmax = 2;
    while (em_delta(k, n, i, i + lmax * d) > dmin)   // ends: out of range gives -1
        lmax <<= 1;
    i64 l = 0;
    for (i64 t = lmax >> 1; t >= 1; t >>= 1)
        if (em_delta(k, n, i, i + (l + t) * d) > dmin)
            l += t;
    const i64 j = i + l * d;
    const int dnode = em_delta(k, n, i, j);
    i64 s = 0;
    for (i64 div = 2;; div <<= 1) {
        const i64 t = (l + div - 1) / div;
        if (em_delta(k, n, i, i + (s + t) * d) > dnode)
            s += t;
        if (t <= 1)
            break;
    }
    const i64 gamma = i + s * d + (d < 0 ? -1 : 0);
    const i64 lo = i < j ? i : j, hi = i < j ? j : i;
    const int lc = (int)(lo == gamma ? (n - 1) + gamma : gamma);
    const int rc = (int)(hi == gamma + 1 ? (n - 1) + gamma + 1 : gamma + 1);
    kids[i] = make_int2(lc, rc);
    parent[lc] = (int)i;
    parent[rc] = (int)i;
    if (i == 0)
        parent[0] = -1;
}

// ---- 3. bottom-up refit ------------------------------------------------------------
// Every internal node keeps the boxes of both its children (wide node): lo =
// (box lo, least core2 below), hi = (box hi, component of all points below
// as int bits, or -1).  A leaf child's box is its point (xyz, core2) with the
// point's component, so a traversal reads one 64-byte record per visited
// node and no point record at all for a leaf child.
struct WideNode {
    float4 lo[2];
    float4 hi[2];
};

// Box of node c (leaf: its point), from data written earlier in this launch
// by other threads (read past L1).
__device__ __forceinline__ void em_box_of(i64 n, int c, const float4 *P4, const i32 *comp,
                                          const WideNode *wn, float4 &lo, float4 &hi)
{
    if (c >= n - 1) {
        const float4 p = __ldcg(P4 + (c - (n - 1)));
        lo = p;
        hi = make_float4(p.x, p.y, p.z, __int_as_float(__ldcg(comp + (c - (n - 1)))));
    } else {
        const float4 a0 = __ldcg(&wn[c].lo[0]), a1 = __ldcg(&wn[c].lo[1]);
        const float4 b0 = __ldcg(&wn[c].hi[0]), b1 = __ldcg(&wn[c].hi[1]);
        const int c0 = __float_as_int(b0.w), c1 = __float_as_int(b1.w);
        lo = make_float4(fminf(a0.x, a1.x), fminf(a0.y, a1.y), fminf(a0.z, a1.z), fminf(a0.w, a1.w));
        hi = make_float4(fmaxf(b0.x, b1.x), fmaxf(b0.y, b1.y), fmaxf(b0.z, b1.z),
                         __int_as_float(c0 == c1 ? c0 : -1));
    }
}

__global__ void __launch_bounds__(256) em_refit_kernel(i64 n, const float4 *P4, const i32 *comp,
                                                       const int2 *kids, const int *parent,
                                                       WideNode *wn, int *flags, int *status)
{
    const i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n)
        return;
    int node = parent[(n - 1) + j];
    for (int depth = 0; node >= 0; ++depth) {
        if (depth >= EM_REFIT_DEPTH) {
            set_status(status, PANDORA_ERR_ITERATION_LIMIT);
            return;
        }
        __threadfence();
        if (atomicAdd(flags + node, 1) == 0)
            return;   // the other child is not done yet; its thread goes on
        __threadfence();
        const int2 ch = kids[node];
        float4 l0, h0, l1, h1;
        em_box_of(n, ch.x, P4, comp, wn, l0, h0);
        em_box_of(n, ch.y, P4, comp, wn, l1, h1);
        wn[node].lo[0] = l0;
        wn[node].hi[0] = h0;
        wn[node].lo[1] = l1;
        wn[node].hi[1] = h1;
        node = parent[node];
    }
}

// ---- 4. core distances ----------------------------------------------------------------
// The k smallest squared distances, ascending, in registers (KCAP slots, of
// which the first k are used): an insertion is one compare-and-shift pass
// with static indices.
template <int KCAP>
struct TopK {
    float v[KCAP];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int t = 0; t < KCAP; ++t)
            v[t] = INFINITY;
    }
    __device__ __forceinline__ float kth(int k) const
    {
        float r = INFINITY;
#pragma unroll
        for (int t = 0; t < KCAP; ++t)
            if (t == k - 1)
                r = v[t];
        return r;
    }
    // insert d2 keeping v ascending; entries past slot k - 1 are dropped
    __device__ __forceinline__ void insert(float d2, int k)
    {
        float x = d2;
#pragma unroll
        for (int t = 0; t < KCAP; ++t) {
            if (t < k && x < v[t]) {
                const float y = v[t];
                v[t] = x;
                x = y;
            }
        }
    }
};

// Every point first takes the points within k positions of it in Morton
// order (itself included), which gives a tight k-th distance before the
// traversal; the traversal then skips those leaves.
#ifndef PANDORA_EM_KNN_MINB
#define PANDORA_EM_KNN_MINB 1
#endif
template <int KCAP>
__global__ void __launch_bounds__(128, PANDORA_EM_KNN_MINB) em_knn_kernel(i64 n, int k, const float4 *__restrict__ P4,
                                                     const int2 *__restrict__ kids,
                                                     const WideNode *__restrict__ wn, float *core2,
                                                     int *status)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 q = P4[i];
    TopK<KCAP> best;
    best.init();
    // a distance at or above the k-th smallest so far cannot enter the
    // first k slots (the insertion is strict), so only smaller ones are
    // inserted
    const i64 w0 = i - k < 0 ? 0 : i - k, w1 = i + k >= n ? n - 1 : i + k;
    float kth = INFINITY;
    for (i64 j = w0; j <= w1; ++j) {
        const float d2 = em_d2(q, P4[j]);
        if (d2 < kth) {
            best.insert(d2, k);
            kth = best.kth(k);
        }
    }
    if (n == 1) {
        core2[i] = kth;
        return;
    }
    // a node goes on the stack with its box's lower bound, taken again
    // against the k-th distance when it is popped
    int stack[EM_STACK];
    float slb[EM_STACK];
    int sp = 0;
    stack[0] = 0;
    slb[0] = 0.f;
    sp = 1;
    while (sp > 0) {
        --sp;
        if (slb[sp] >= kth)
            continue;
        const int node = stack[sp];
        const int2 kc = kids[node];
        const int ch[2] = {kc.x, kc.y};
        float lb[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float4 clo = wn[node].lo[c];
            lb[c] = INFINITY;
            if (ch[c] >= n - 1) {
                const i64 j = ch[c] - (n - 1);
                if (j < w0 || j > w1) {   // the window's points are counted already
                    const float d2 = em_d2(q, clo);
                    if (d2 < kth) {
                        best.insert(d2, k);
                        kth = best.kth(k);
                    }
                }
            } else {
                lb[c] = em_box_d2(q, clo, wn[node].hi[c]);
            }
        }
        // push the farther child first so that the nearer one is visited next
        const int first = lb[0] <= lb[1] ? 1 : 0;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int c = t == 0 ? first : 1 - first;
            if (ch[c] < n - 1 && lb[c] < kth) {   // internal nodes only
                if (sp >= EM_STACK) {
                    set_status(status, PANDORA_ERR_ITERATION_LIMIT);
                    sp = 0;
                    break;
                }
                stack[sp] = ch[c];
                slb[sp] = lb[c];
                ++sp;
            }
        }
    }
    core2[i] = kth;
}

__global__ void __launch_bounds__(256) em_set_core_kernel(i64 n, float4 *P4, const float *core2)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        P4[i].w = core2[i];
}

// ---- 5. Boruvka rounds ------------------------------------------------------------------
__device__ __forceinline__ bool em_less(float w, u32 lo, u32 hi, float bw, u32 blo, u32 bhi)
{
    return w < bw || (w == bw && (lo < blo || (lo == blo && hi < bhi)));
}

__device__ __forceinline__ float em_comp_bound(const u32 *cbest_w, int c)
{
    return __uint_as_float(*(const volatile u32 *)(cbest_w + c));
}

// A point's least edge of the previous round (weight pw, id pair lo < hi,
// one of them the point's own id oq) is still an edge to another component
// when its far end has not joined the point's component since: components
// only merge, so it stays a candidate and bounds the point's least edge
// from above.
__device__ __forceinline__ bool em_prev_valid(float pw, u32 lo, u32 hi, u32 oq, int cq,
                                              const i32 *comp, const i32 *pos_of)
{
    if (!(pw < INFINITY))
        return false;
    const u32 other = lo == oq ? hi : lo;
    return comp[pos_of[other]] != cq;
}

#ifndef PANDORA_EM_QUERY_MINB
#define PANDORA_EM_QUERY_MINB 1
#endif
__global__ void __launch_bounds__(128, PANDORA_EM_QUERY_MINB) em_query_kernel(i64 n, const float4 *__restrict__ P4,
                                                       const i32 *__restrict__ comp,
                                                       const u32 *__restrict__ orig,
                                                       const int2 *__restrict__ kids,
                                                       const WideNode *__restrict__ wn,
                                                       const i32 *__restrict__ pos_of,
                                                       u32 *cbest_w, float *qbw, u32 *qlo,
                                                       u32 *qhi, int *status)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 q = P4[i];
    const int cq = comp[i];
    const u32 oq = orig[i];
    float bw = INFINITY;
    u32 blo = 0xFFFFFFFFu, bhi = 0xFFFFFFFFu;
    {
        const float pw = qbw[i];
        const u32 plo = qlo[i], phi = qhi[i];
        if (em_prev_valid(pw, plo, phi, oq, cq, comp, pos_of)) {
            bw = pw;
            blo = plo;
            bhi = phi;
        }
    }
    float cw = em_comp_bound(cbest_w, cq);
    // every edge of q weighs at least core2(q): above the component's least
    // edge found so far, q cannot supply it
    if (!(q.w > cw)) {
        // a node goes on the stack with the lower bound of its box (no subtree
        // wholly in q's component is pushed), taken again against the bound
        // when it is popped
        int stack[EM_STACK];
        float slb[EM_STACK];
        stack[0] = 0;
        slb[0] = 0.f;
        int sp = 1;
        int pops = 0;
        while (sp > 0) {
            --sp;
            if ((++pops & 15) == 0)
                cw = em_comp_bound(cbest_w, cq);
            if (slb[sp] > fminf(bw, cw))
                continue;
            const int node = stack[sp];
            const int2 kc = kids[node];
            const int ch[2] = {kc.x, kc.y};
            float lb[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                lb[c] = INFINITY;
                const float4 clo = wn[node].lo[c], chi = wn[node].hi[c];
                if (__float_as_int(chi.w) == cq)
                    continue;   // all of its points are in q's component
                if (ch[c] >= n - 1) {
                    // a point of another component: clo = (x, y, z, core2)
                    const float w2 = fmaxf(fmaxf(q.w, clo.w), em_d2(q, clo));
                    if (w2 <= bw) {
                        const u32 oj = orig[ch[c] - (n - 1)];
                        const u32 lo_id = oq < oj ? oq : oj, hi_id = oq < oj ? oj : oq;
                        if (em_less(w2, lo_id, hi_id, bw, blo, bhi)) {
                            bw = w2;
                            blo = lo_id;
                            bhi = hi_id;
                        }
                    }
                } else {
                    lb[c] = fmaxf(fmaxf(q.w, clo.w), em_box_d2(q, clo, chi));
                }
            }
            const float bound2 = fminf(bw, cw);
            const int first = lb[0] <= lb[1] ? 1 : 0;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int c = t == 0 ? first : 1 - first;
                // only internal nodes go on the stack (a leaf child was
                // handled above; its lb stays infinite, and so can the bound)
                if (ch[c] < n - 1 && lb[c] <= bound2) {
                    if (sp >= EM_STACK) {
                        set_status(status, PANDORA_ERR_ITERATION_LIMIT);
                        sp = 0;
                        break;
                    }
                    stack[sp] = ch[c];
                    slb[sp] = lb[c];
                    ++sp;
                }
            }
        }
    }
    qbw[i] = bw;
    qlo[i] = blo;
    qhi[i] = bhi;
    if (bw < INFINITY)
        atomicMin(cbest_w + cq, __float_as_uint(bw));
}

// Before the traversals of a round: every point offers the lightest edge to
// its Morton-order neighbours (within EM_SEED positions) in another
// component as an upper bound of its component's least edge, so that the
// traversals start with a tight bound.  Only a bound: the traversal finds
// the least edge itself.
constexpr int EM_SEED = 8;
__global__ void __launch_bounds__(256) em_seed_kernel(i64 n, const float4 *__restrict__ P4,
                                                      const i32 *__restrict__ comp,
                                                      const u32 *__restrict__ orig,
                                                      const i32 *__restrict__ pos_of,
                                                      const float *__restrict__ qbw,
                                                      const u32 *__restrict__ qlo,
                                                      const u32 *__restrict__ qhi, u32 *cbest_w)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float4 q = P4[i];
    const int cq = comp[i];
    float bw = INFINITY;
    const i64 w0 = i - EM_SEED < 0 ? 0 : i - EM_SEED, w1 = i + EM_SEED >= n ? n - 1 : i + EM_SEED;
    for (i64 j = w0; j <= w1; ++j) {
        if (comp[j] == cq)
            continue;
        const float4 p = P4[j];
        bw = fminf(bw, fmaxf(fmaxf(q.w, p.w), em_d2(q, p)));
    }
    // and the point's least edge of the previous round, if still valid
    const float pw = qbw[i];
    if (pw < bw && em_prev_valid(pw, qlo[i], qhi[i], orig[i], cq, comp, pos_of))
        bw = pw;
    if (bw < INFINITY && __float_as_uint(bw) < *(const volatile u32 *)(cbest_w + cq))
        atomicMin(cbest_w + cq, __float_as_uint(bw));
}

// Among the points whose least edge has the component's least weight, the
// least id pair.
__global__ void __launch_bounds__(256) em_choose_kernel(i64 n, const i32 *comp, const u32 *cbest_w,
                                                        const float *qbw, const u32 *qlo,
                                                        const u32 *qhi, u64 *cbest_e)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const int c = comp[i];
    const float bw = qbw[i];
    if (bw < INFINITY && __float_as_uint(bw) == cbest_w[c])
        atomicMin((unsigned long long *)(cbest_e + c), ((u64)qlo[i] << 32) | qhi[i]);
}

// Every component (its representative is the point r with comp[r] == r)
// links to the component across its least edge; of two components that chose
// the same edge the one with the smaller representative becomes the root and
// the edge is recorded once.
__global__ void __launch_bounds__(256) em_link_kernel(i64 n, const i32 *comp, const i32 *pos_of,
                                                      const u32 *cbest_w, const u64 *cbest_e,
                                                      i32 *parent, EmCtrl *ctrl, u32 *eu,
                                                      u32 *ev, float *ew2)
{
    const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n || comp[r] != (i32)r)
        return;
    const u64 e = cbest_e[r];
    if (e == ~0ull) {   // no edge leaves: the last component
        parent[r] = (i32)r;
        return;
    }
    const u32 lo = (u32)(e >> 32), hi = (u32)e;
    if ((i64)lo >= n || (i64)hi >= n) {
        set_status(&ctrl->status, PANDORA_ERR_ITERATION_LIMIT);
        parent[r] = (i32)r;
        return;
    }
    const i32 ca = comp[pos_of[lo]], cb = comp[pos_of[hi]];
    const i32 other = ca == (i32)r ? cb : ca;
    if (other == (i32)r || (ca != (i32)r && cb != (i32)r)) {   // never on a valid state
        set_status(&ctrl->status, PANDORA_ERR_ITERATION_LIMIT);
        parent[r] = (i32)r;
        return;
    }
    const bool mutual = cbest_e[other] == e;
    if (mutual && (i32)r < other) {
        parent[r] = (i32)r;
        return;
    }
    parent[r] = other;
    const u64 slot = atomicAdd((unsigned long long *)&ctrl->n_edges, 1ull);
    if ((i64)slot < n - 1) {
        eu[slot] = lo;
        ev[slot] = hi;
        ew2[slot] = __uint_as_float(cbest_w[r]);
    } else {
        set_status(&ctrl->status, PANDORA_ERR_ITERATION_LIMIT);
    }
}

__global__ void __launch_bounds__(256) em_jump_kernel(i64 n, const i32 *comp, i32 *parent,
                                                      EmCtrl *ctrl)
{
    const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n || comp[r] != (i32)r)
        return;
    const i32 p = parent[r];
    const i32 pp = parent[p];
    if (pp != p) {
        parent[r] = pp;
        ctrl->changed = 1;
    }
}

__global__ void __launch_bounds__(256) em_relabel_kernel(i64 n, i32 *comp, const i32 *parent,
                                                         u32 *cbest_w, u64 *cbest_e)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    comp[i] = parent[comp[i]];
    cbest_w[i] = INF_BITS;   // reset for the next round
    cbest_e[i] = ~0ull;
}

__global__ void __launch_bounds__(256) em_output_kernel(i64 n, const u32 *eu, const u32 *ev,
                                                        const float *ew2, i32 *u, i32 *v,
                                                        float *w, const float *core2,
                                                        const u32 *orig, float *core_out)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n - 1) {
        u[i] = (i32)eu[i];
        v[i] = (i32)ev[i];
        w[i] = __fsqrt_rn(ew2[i]);
    }
    if (core_out && i < n)
        core_out[orig[i]] = core2[i];
}

__global__ void em_fill_kernel(u32 *a, u64 *b, float *qbw, i64 n)
{
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        a[i] = INF_BITS;
        b[i] = ~0ull;
        qbw[i] = INFINITY;
    }
}

inline unsigned blocks_for(i64 n, int t) { return (unsigned)std::max<i64>(1, (n + t - 1) / t); }

struct EmLayout {
    size_t ctrl, codesA, codesB, idsA, idsB, lb, P4, pos_of, comp, parentc, cbest_w, cbest_e;
    size_t qbw, qlo, qhi, eu, ev, ew2, core2, kids, nparent, wn, flags, total;
};

EmLayout em_layout(i64 n)
{
    EmLayout L{};
    size_t off = 0;
    auto take = [&](i64 bytes) {
        const size_t o = off;
        off = (off + (size_t)std::max<i64>(bytes, 0) + 255) & ~size_t(255);
        return o;
    };
    const i64 ni = std::max<i64>(n - 1, 1);
    L.ctrl = take(sizeof(EmCtrl));
    L.codesA = take(n * 4);
    L.codesB = take(n * 4);
    L.idsA = take(n * 4);
    L.idsB = take(n * 4);
    L.lb = take(onesweep_tiles(n) * RADIX * 8);
    L.P4 = take(n * 16);
    L.pos_of = take(n * 4);
    L.comp = take(n * 4);
    L.parentc = take(n * 4);
    L.cbest_w = take(n * 4);
    L.cbest_e = take(n * 8);
    L.qbw = take(n * 4);
    L.qlo = take(n * 4);
    L.qhi = take(n * 4);
    L.eu = take(n * 4);
    L.ev = take(n * 4);
    L.ew2 = take(n * 4);
    L.core2 = take(n * 4);
    L.kids = take(ni * 8);
    L.nparent = take((2 * n) * 4);
    L.wn = take(ni * sizeof(WideNode));
    L.flags = take(ni * 4);
    L.total = off;
    return L;
}

#define EM_CUDA(call)                      \
    do {                                   \
        if ((call) != cudaSuccess)         \
            return PANDORA_ERR_CUDA;       \
    } while (0)

int em_read(const EmCtrl *c, EmCtrl *h, cudaStream_t s)
{
    EM_CUDA(cudaMemcpyAsync(h, c, offsetof(EmCtrl, hist), cudaMemcpyDeviceToHost, s));
    EM_CUDA(cudaStreamSynchronize(s));
    return PANDORA_OK;
}

int em_run(const float *pts, i64 n, int k, i32 *u, i32 *v, float *w, float *core_out, char *base,
           cudaStream_t s)
{
    const EmLayout L = em_layout(n);
    EmCtrl *ctrl = (EmCtrl *)(base + L.ctrl);
    u32 *codesA = (u32 *)(base + L.codesA), *codesB = (u32 *)(base + L.codesB);
    u32 *idsA = (u32 *)(base + L.idsA), *idsB = (u32 *)(base + L.idsB);
    u64 *lb = (u64 *)(base + L.lb);
    float4 *P4 = (float4 *)(base + L.P4);
    i32 *pos_of = (i32 *)(base + L.pos_of), *comp = (i32 *)(base + L.comp);
    i32 *parentc = (i32 *)(base + L.parentc);
    u32 *cbest_w = (u32 *)(base + L.cbest_w);
    u64 *cbest_e = (u64 *)(base + L.cbest_e);
    float *qbw = (float *)(base + L.qbw);
    u32 *qlo = (u32 *)(base + L.qlo), *qhi = (u32 *)(base + L.qhi);
    u32 *eu = (u32 *)(base + L.eu), *ev = (u32 *)(base + L.ev);
    float *ew2 = (float *)(base + L.ew2), *core2 = (float *)(base + L.core2);
    int2 *kids = (int2 *)(base + L.kids);
    int *nparent = (int *)(base + L.nparent);
    WideNode *wn = (WideNode *)(base + L.wn);
    int *flags = (int *)(base + L.flags);
    EmCtrl h{};

    EM_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(EmCtrl), s));
    EM_CUDA(cudaMemsetAsync(ctrl->lo_key, 0xFF, sizeof(ctrl->lo_key), s));
    em_bbox_kernel<<<blocks_for(n, 256 * 16) > 1216 ? 1216 : blocks_for(n, 256 * 16), 256, 0, s>>>(
        pts, n, ctrl);
    em_morton_kernel<<<blocks_for(n, 256), 256, 0, s>>>(pts, n, ctrl, codesA, idsA);
    launch_hist_keys(codesA, n, &ctrl->hist[0][0], s);
    launch_hist_scan(&ctrl->hist[0][0], &ctrl->base[0][0], 4, s);
    static thread_local u32 hh[4][RADIX];
    EM_CUDA(cudaMemcpyAsync(hh, ctrl->hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
    if (int e = em_read(ctrl, &h, s))
        return e;
    if (h.status)
        return h.status;
    // stable LSD sort of (Morton code, point id); passes whose digit is the
    // same for every code are skipped
    const u32 *ck = codesA, *cv = idsA;
    for (int p = 0; p < 4; ++p) {
        bool trivial = false;
        for (int d = 0; d < RADIX; ++d)
            if ((i64)hh[p][d] == n)
                trivial = true;
        if (trivial)
            continue;
        OnesweepParams P{};
        P.n = n;
        P.shift = 8 * p;
        P.hist = ctrl->hist[p];
        P.bin_base = ctrl->base[p];
        P.lb = lb;
        P.tile_counter = &ctrl->tile_counter;
        P.status = &ctrl->status;
        P.keys_in = ck;
        P.vals_in = cv;
        P.keys_out = ck == codesA ? codesB : codesA;
        P.vals_out = cv == idsA ? idsB : idsA;
        EM_CUDA(cudaMemsetAsync(lb, 0, (size_t)onesweep_tiles(n) * RADIX * 8, s));
        EM_CUDA(cudaMemsetAsync(&ctrl->tile_counter, 0, 4, s));
        launch_onesweep(OS_WRITE_KEYS, P, s);
        ck = P.keys_out;
        cv = P.vals_out;
    }
    em_gather_kernel<<<blocks_for(n, 256), 256, 0, s>>>(pts, n, cv, P4, pos_of, comp);
    const u32 *orig = cv;
    if (n > 1) {
        em_build_kernel<<<blocks_for(n - 1, 256), 256, 0, s>>>(ck, n, kids, nparent);
        EM_CUDA(cudaMemsetAsync(flags, 0, (size_t)(n - 1) * 4, s));
        em_refit_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, P4, comp, kids, nparent, wn, flags,
                                                           &ctrl->status);
    }
    if (k <= 8)
        em_knn_kernel<8><<<blocks_for(n, 128), 128, 0, s>>>(n, k, P4, kids, wn, core2, &ctrl->status);
    else if (k <= 16)
        em_knn_kernel<16><<<blocks_for(n, 128), 128, 0, s>>>(n, k, P4, kids, wn, core2, &ctrl->status);
    else
        em_knn_kernel<EM_K_MAX><<<blocks_for(n, 128), 128, 0, s>>>(n, k, P4, kids, wn, core2,
                                                                   &ctrl->status);
    em_set_core_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, P4, core2);
    em_fill_kernel<<<blocks_for(n, 256), 256, 0, s>>>(cbest_w, cbest_e, qbw, n);
    EM_CUDA(cudaGetLastError());
    for (int round = 0; n > 1; ++round) {
        if (round >= EM_MAX_ROUNDS)
            return PANDORA_ERR_ITERATION_LIMIT;
        EM_CUDA(cudaMemsetAsync(flags, 0, (size_t)(n - 1) * 4, s));
        em_refit_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, P4, comp, kids, nparent, wn, flags,
                                                           &ctrl->status);
        em_seed_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, P4, comp, orig, pos_of, qbw, qlo,
                                                          qhi, cbest_w);
        em_query_kernel<<<blocks_for(n, 128), 128, 0, s>>>(n, P4, comp, orig, kids, wn, pos_of,
                                                           cbest_w, qbw, qlo, qhi, &ctrl->status);
        em_choose_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, comp, cbest_w, qbw, qlo, qhi,
                                                            cbest_e);
        em_link_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, comp, pos_of, cbest_w, cbest_e,
                                                          parentc, ctrl, eu, ev, ew2);
        // pointer jumping to the roots, checked every few passes
        for (int pass = 0;; pass += 4) {
            if (pass > 2 * 64)
                return PANDORA_ERR_ITERATION_LIMIT;
            EM_CUDA(cudaMemsetAsync(&ctrl->changed, 0, 4, s));
            for (int t = 0; t < 4; ++t)
                em_jump_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, comp, parentc, ctrl);
            if (int e = em_read(ctrl, &h, s))
                return e;
            if (h.status)
                return h.status;
            if (!h.changed)
                break;
        }
        em_relabel_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, comp, parentc, cbest_w, cbest_e);
        EM_CUDA(cudaGetLastError());
        if (int e = em_read(ctrl, &h, s))
            return e;
        if (h.status)
            return h.status;
        if ((i64)h.n_edges >= n - 1)
            break;
    }
    em_output_kernel<<<blocks_for(n, 256), 256, 0, s>>>(n, eu, ev, ew2, u, v, w, core2, orig,
                                                        core_out);
    EM_CUDA(cudaGetLastError());
    if (int e = em_read(ctrl, &h, s))
        return e;
    return h.status;
}

}  // namespace
}  // namespace pandora

extern "C" int pandora_mr_emst(const float *points, int64_t n_points, int32_t min_pts, int32_t *u,
                               int32_t *v, float *w, float *core_sq, void *stream)
{
    using namespace pandora;
    if (!points || n_points < 1 || min_pts < 1 || min_pts > PANDORA_EMST_MAX_MIN_PTS ||
        (i64)min_pts > n_points)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (n_points > PANDORA_EMST_MAX_POINTS)
        return PANDORA_ERR_SIZE_LIMIT;
    if (n_points > 1 && (!u || !v || !w))
        return PANDORA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    cudaMemPool_t pool = flat_pool(dev);
    if (!pool)
        return PANDORA_ERR_CUDA;
    const size_t bytes = em_layout(n_points).total + 256;
    void *ws = nullptr;
    if (cudaMallocFromPoolAsync(&ws, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return PANDORA_ERR_OUT_OF_MEMORY;
    }
    char *base = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    const int st = em_run(points, n_points, min_pts, u, v, w, core_sq, base, s);
    cudaFreeAsync(ws, s);
    cudaStreamSynchronize(s);
    return st;
}

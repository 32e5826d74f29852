// HDBSCAN* flat clusters from a single-linkage dendrogram
// (pandora_hdbscan_labels, include/pandora.h).
//
// The optional last step of the HDBSCAN* pipeline (Section 6.5): the flat
// clustering of Campello et al.  As edges are removed from the heaviest down
// (lambda = 1/w grows), a cluster is a part of the tree that stays at least
// min_cluster_size (mcs) points large; it ends where it splits into two such
// parts, and points leave it where they fall off in smaller parts.  Clusters
// are scored by their stability and the non-overlapping set of largest total
// stability is kept (excess of mass, the whole data set excluded).
//
// Nodes: edge e is node e, vertex x is node m + x; the parent of a node is
// edge_parent / vertex_parent.  Every step is a data-parallel kernel:
//
//  1. parents, child slots and validation (binary tree, one root, every
//     parent later than its child in (weight, index) order, weights > 0);
//  2. leaf counts: Euler tour of the dendrogram (down/up arc per edge, one
//     arc per leaf), suffix sums by list ranking over a sparse ruling set;
//  3. big = leaf count >= mcs; cluster starts (the root, and both children
//     of an edge whose children are both big); the start above every big
//     edge (the big edges of a cluster form one upward path: a second ruling
//     set); for every vertex, the top t of the small subtree it falls off in
//     (t has a big parent p; p gives the leave lambda and, through its start,
//     the cluster), found by a fill-forward scan over the leaf indices of the
//     tour, since each such subtree holds consecutive leaves;
//  4. stabilities: every term (a leaving point's fl(lambda - birth), and
//     size(D) copies of a child cluster's fl(birth(D) - birth(C))) is a
//     multiple of 2^-180 below 2^181 (lambda = 1/w of a float32 w lies in
//     (2^-128, 2^149]), so it is added exactly into a fixed-point accumulator
//     of 32-bit digits with integer atomics; the exact sum is rounded once to
//     float64 (round to nearest, ties to even).  The result does not depend on
//     the order of the additions;
//  5. excess of mass over the binary cluster tree, exactly (children's best
//     totals are exact sums of float64 stabilities), by parallel tree
//     contraction (rake rounds, then the rakes replayed in reverse);
//  6. labels: the topmost selected cluster above a vertex's cluster (pointer
//     jumping over the cluster tree), numbered by smallest member (two scans).
#include <cfloat>
#include <cstdint>
#include <cstring>

#include "common.cuh"

namespace pandora {
cudaMemPool_t flat_pool(int dev);
}

namespace {

using namespace pandora;

constexpr int FT = 256;            // threads per block of the element-wise kernels
constexpr int NL = 14;             // 32-bit digits of a stability accumulator (448 bits)
constexpr int FIX_EXP = 180;       // accumulator unit: 2^-180
constexpr u32 FULL = 0xFFFFFFFFu;

struct FlatCtrl {
    int status;
    int n_roots;
    int root;          // root edge
    int n_starts;      // clusters (start edges), from the scan
    int root_cid;      // cluster id of the root
    int n_selected;    // selected clusters, from the scan
    int n_leaves;      // leaf clusters, from the scan
    u32 rs_count;      // splitters of the list ranking
    u32 bp_count;      // splitters of the path heads
    u32 unresolved;    // segments still without their start (per round)
};

__device__ __forceinline__ bool failed(const FlatCtrl *c)
{
    return *(const volatile int *)&c->status != 0;
}

// Slot in a list appended to by many threads: one atomic per warp on the
// shared counter (a counter hit by every thread serialises in L2).
__device__ __forceinline__ u32 warp_append(u32 *counter, bool want)
{
    const u32 active = __activemask();
    const u32 mask = __ballot_sync(active, want);
    if (!want)
        return 0;
    const int leader = __ffs(mask) - 1;
    const int lane = threadIdx.x & 31;
    u32 base = 0;
    if (lane == leader)
        base = atomicAdd(counter, (u32)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + (u32)__popc(mask & ((1u << lane) - 1));
}

__device__ __forceinline__ i32 enter_arc(i32 node, i32 m)
{
    return node < m ? 2 * node : 2 * m + (node - m);
}

// Arc after the last arc of node c's subtree walk.
__device__ __forceinline__ i32 after_arc(i32 c, i32 m, const i32 *par, const i32 *kids)
{
    const i32 p = par[c];
    if (p < 0)
        return -1;
    if (kids[2 * (i64)p] == c)
        return enter_arc(kids[2 * (i64)p + 1], m);
    return par[p] < 0 ? -1 : 2 * p + 1;
}

// ---- 1. parents and validation --------------------------------------------
// Children of edge p: the smaller node id in kids[2p], the larger in
// kids[2p + 1] (any fixed order serves the tour).  Three 32-bit reductions per
// child (count, min, max) measured faster than one 64-bit add carrying the
// count and the id sum plus a min (79.6 vs 86.4 ms at 10^8 points).
__global__ void flat_parents_kernel(const i32 *ep, const i32 *vp, const float *w, i32 m, i32 n,
                                    i32 *par, i32 *cnt, i32 *kids, FlatCtrl *c)
{
    const i64 N = (i64)m + n;
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < N;
         i += (i64)gridDim.x * blockDim.x) {
        i32 p;
        if (i < m) {
            const float we = w[i];
            if (!(we > 0.f && we <= FLT_MAX))
                set_status(&c->status, PANDORA_ERR_BAD_WEIGHT);
            p = ep[i];
            if (p == -1) {
                atomicAdd(&c->n_roots, 1);
                c->root = (i32)i;
                par[i] = -1;
                continue;
            }
        } else {
            p = vp[i - m];
        }
        if (p < 0 || p >= m) {
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
            par[i] = -1;
            continue;
        }
        par[i] = p;
        // no return values: the three updates issue as reductions
        atomicAdd(&cnt[p], 1);
        atomicMin(&kids[2 * (i64)p], (i32)i);
        atomicMax(&kids[2 * (i64)p + 1], (i32)i);
    }
}

// kids[2e] = INT32_MAX and kids[2e + 1] = -1 (for the min / max above), cnt = 0.
__global__ void kids_init_kernel(i32 m, i32 *kids, i32 *cnt)
{
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x) {
        reinterpret_cast<int2 *>(kids)[e] = make_int2(INT32_MAX, -1);
        cnt[e] = 0;
    }
}

// Two children per edge, one root, and every parent after its child in the
// (weight, index) order (which also rules out cycles).
__global__ void flat_check_kernel(const float *w, i32 m, const i32 *par, const i32 *cnt,
                                  FlatCtrl *c)
{
    if (blockIdx.x == 0 && threadIdx.x == 0 && c->n_roots != 1)
        set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x) {
        bool ok = cnt[e] == 2;
        const i32 p = par[e];
        if (p >= 0) {
            const float wp = w[p], we = w[e];
            ok = ok && (wp > we || (wp == we && p > e));
        }
        if (!ok)
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
    }
}

// ---- 2. leaf counts ----------------------------------------------------------
// Arc word: next arc (high 32 bits, -1 at the end) | leaf count (low 32 bits).
__global__ void tour_init_kernel(i32 m, i32 n, const i32 *par, const i32 *kids, u64 *arc,
                                 const FlatCtrl *c)
{
    if (failed(c))
        return;
    const i64 L = 2 * (i64)m + n;
    for (i64 a = blockIdx.x * (i64)blockDim.x + threadIdx.x; a < L;
         a += (i64)gridDim.x * blockDim.x) {
        i32 next;
        u32 val = 0;
        if (a < 2 * (i64)m) {
            const i32 e = (i32)(a >> 1);
            next = (a & 1) ? after_arc(e, m, par, kids) : enter_arc(kids[2 * (i64)e], m);
        } else {
            next = after_arc(m + (i32)(a - 2 * (i64)m), m, par, kids);
            val = 1;
        }
        arc[a] = ((u64)(u32)next << 32) | val;
    }
}

__global__ void rank_step_kernel(const u64 *in, u64 *out, i64 L, const FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 a = blockIdx.x * (i64)blockDim.x + threadIdx.x; a < L;
         a += (i64)gridDim.x * blockDim.x) {
        const u64 r = in[a];
        const i32 nx = (i32)(r >> 32);
        if (nx >= 0) {
            const u64 q = in[nx];
            out[a] = (q & 0xFFFFFFFF00000000ull) | (u32)((u32)r + (u32)q);
        } else {
            out[a] = r;
        }
    }
}

// Suffix sums by a sparse ruling set: about one arc in 64 (by a hash of its
// id, plus the head and the root's unused up arc) is a splitter; one thread
// per splitter walks its segment up to the next splitter, recording for every
// arc its segment and the sum before it; the short list of segments is
// ranked by pointer jumping; then suffix(a) = suffix(segment) - (sum before a).
// O(L) work instead of the O(L log L) of jumping on the whole list.
constexpr u32 RS_MASK = 63;

__device__ __forceinline__ bool rs_splitter(i64 a, i64 head)
{
    u32 h = (u32)a * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    return a == head || a == head + 1 || (h & RS_MASK) == 0;
}

inline i64 rs_capacity(i64 L) { return L / 48 + 4096; }

__global__ void rs_pick_kernel(i64 L, i32 *sid_of, i32 *spl, i64 cap, FlatCtrl *c)
{
    if (failed(c))
        return;
    const i64 head = 2 * (i64)c->root;
    for (i64 a = blockIdx.x * (i64)blockDim.x + threadIdx.x; a < L;
         a += (i64)gridDim.x * blockDim.x) {
        const bool pick = rs_splitter(a, head);
        const u32 id = warp_append(&c->rs_count, pick);
        if (!pick)
            continue;
        if ((i64)id < cap) {
            spl[id] = (i32)a;
            sid_of[a] = (i32)id;
        } else {
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
        }
    }
}

// seg[i]: next segment (high 32 bits, -1 at the end) | sum of the segment.
// Records (segment, sum before it) for every arc in owner_loc.  (Writing it
// over the arc word just read, in place, measured six times slower.)
__global__ void rs_walk_kernel(const u64 *arc, u64 *owner_loc, const i32 *sid_of,
                               const i32 *spl, i64 cap, i64 L, u64 *seg, FlatCtrl *c)
{
    if (failed(c))
        return;
    const i64 head = 2 * (i64)c->root;
    const i64 cnt = (i64)c->rs_count < cap ? (i64)c->rs_count : cap;
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < cnt;
         i += (i64)gridDim.x * blockDim.x) {
        i64 a = spl[i];
        u32 sum = 0;
        u32 next_seg = 0xFFFFFFFFu;
        for (i64 steps = 0;; ++steps) {
            if (steps > L) {
                set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
                break;
            }
            const u64 w = arc[a];
            owner_loc[a] = ((u64)i << 32) | sum;
            sum += (u32)w;
            const i32 nx = (i32)(w >> 32);
            if (nx < 0)
                break;
            if (rs_splitter(nx, head)) {
                next_seg = (u32)sid_of[nx];
                break;
            }
            a = nx;
        }
        seg[i] = ((u64)next_seg << 32) | sum;
    }
}

// (segment, sum before) -> suffix sum, into the arc array.
__global__ void rs_final_kernel(const u64 *owner_loc, const u64 *seg_suf, i64 cap, i64 L,
                                u64 *arc, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 a = blockIdx.x * (i64)blockDim.x + threadIdx.x; a < L;
         a += (i64)gridDim.x * blockDim.x) {
        const u64 ol = owner_loc[a];
        const i64 own = (i64)(ol >> 32);
        if (own >= cap) {
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
            continue;
        }
        arc[a] = (u32)seg_suf[own] - (u32)ol;
    }
}

// size(e) = suffix(down(e)) - suffix(up(e)); the root holds all n leaves.
__global__ void sizes_kernel(const u64 *suf, i32 m, i32 n, i32 *size, FlatCtrl *c)
{
    if (failed(c))
        return;
    const i32 root = c->root;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (u32)suf[2 * (i64)root] != (u32)n)
        set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x)
        size[e] = e == root ? n : (i32)((u32)suf[2 * e] - (u32)suf[2 * e + 1]);
}

// ---- 3. cluster starts, the start above every big edge ---------------------------
__device__ __forceinline__ i32 node_size(i32 node, i32 m, const i32 *size)
{
    return node < m ? size[node] : 1;
}

// start(e): the root, or a big edge whose sibling is big too (both children of
// a split start clusters).  head(e) = e for a start, -1 until resolved.
__global__ void start_kernel(i32 m, i32 mcs, const i32 *par, const i32 *kids, const i32 *size,
                             i32 *start, i32 *head, const FlatCtrl *c)
{
    if (failed(c))
        return;
    const i32 root = c->root;
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x) {
        bool st = e == root;
        if (!st && size[e] >= mcs) {
            const i32 p = par[e];
            const i32 k0 = kids[2 * (i64)p];
            const i32 sib = k0 == (i32)e ? kids[2 * (i64)p + 1] : k0;
            st = node_size(sib, m, size) >= mcs;
        }
        start[e] = st;
        head[e] = st ? (i32)e : -1;
    }
}

// The big edges of one cluster form a path going up to its start (a big edge
// with one big child continues its parent's cluster), so the start above
// every big edge is the head of its path: list ranking again, by a ruling
// set.  Splitters: the bottom of every path (a big non-start edge with zero
// or two big children) and about one other big edge in 64; one thread per
// splitter walks up to the next splitter or to the start; the short lists
// of segments are resolved by pointer jumping.
__device__ __forceinline__ bool path_hash_pick(i64 e)
{
    u32 h = (u32)e * 0x9E3779B1u;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    return (h & 63u) == 0;
}

__global__ void path_pick_kernel(i32 m, i32 mcs, const i32 *kids, const i32 *size,
                                 const i32 *start, i32 *bsid, i32 *spl, i64 cap, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x) {
        i32 id = -1;
        bool pick = false;
        if (size[e] >= mcs && !start[e]) {
            const int nbig = (node_size(kids[2 * e], m, size) >= mcs) +
                             (node_size(kids[2 * e + 1], m, size) >= mcs);
            pick = nbig != 1 || path_hash_pick(e);
        }
        const u32 t = warp_append(&c->bp_count, pick);
        if (pick) {
            if ((i64)t < cap) {
                id = (i32)t;
                spl[t] = (i32)e;
            } else {
                set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
            }
        }
        bsid[e] = id;
    }
}

__global__ void path_walk_kernel(i32 m, const i32 *par, const i32 *start, const i32 *bsid,
                                 const i32 *spl, i64 cap, i32 *seg_of, i32 *seg_next,
                                 i32 *seg_head, FlatCtrl *c)
{
    if (failed(c))
        return;
    const i64 cnt = (i64)c->bp_count < cap ? (i64)c->bp_count : cap;
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < cnt;
         i += (i64)gridDim.x * blockDim.x) {
        i32 cur = spl[i];
        for (i64 steps = 0;; ++steps) {
            seg_of[cur] = (i32)i;
            const i32 nx = par[cur];
            if (nx < 0 || steps > m) {             // a big non-start edge has a parent
                set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
                break;
            }
            if (start[nx]) {
                seg_next[i] = -1;
                seg_head[i] = nx;
                break;
            }
            const i32 sb = bsid[nx];
            if (sb >= 0) {
                seg_next[i] = sb;
                seg_head[i] = -1;
                break;
            }
            cur = nx;
        }
    }
}

// (next, head): head is valid once next = -1.
__global__ void seg_jump_kernel(i64 cnt, const i32 *nxA, const i32 *hdA, i32 *nxB, i32 *hdB,
                                u32 *unresolved, const FlatCtrl *c)
{
    if (failed(c))
        return;
    u32 open = 0;
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < cnt;
         i += (i64)gridDim.x * blockDim.x) {
        const i32 j = nxA[i];
        if (j >= 0) {
            const i32 jj = nxA[j];
            nxB[i] = jj;
            hdB[i] = hdA[j];
            open += jj >= 0;
        } else {
            nxB[i] = -1;
            hdB[i] = hdA[i];
        }
    }
    open = __reduce_add_sync(__activemask(), open);
    if ((threadIdx.x & 31) == 0 && open)
        atomicAdd(unresolved, open);
}

__global__ void path_final_kernel(i32 m, i32 mcs, const i32 *size, const i32 *start,
                                  const i32 *seg_of, const i32 *hd, i64 cap, i32 *head,
                                  FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x) {
        if (size[e] < mcs || start[e])
            continue;
        const i32 sg = seg_of[e];
        const i32 h = (sg >= 0 && sg < cap) ? hd[sg] : -1;
        if (h < 0)
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
        else
            head[e] = h;
    }
}

// Every leaf leaves its cluster inside the small subtree whose top t has a
// big parent p: at lambda(p), from the cluster of p.  Those subtrees hold
// consecutive leaves of the tour, so the record (cluster of p, p) is written
// at the index of t's first leaf (leaves before it = n - suffix(first arc))
// and filled forward over the leaf indices.
constexpr u64 NO_RECORD = ~0ull;

__global__ void anchor_mark_kernel(i32 m, i32 n, i32 mcs, const i32 *par, const i32 *size,
                                   const i32 *head, const i32 *cid, const u64 *suf, u64 *rec,
                                   FlatCtrl *c)
{
    if (failed(c))
        return;
    const i64 N = (i64)m + n;
    for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < N;
         t += (i64)gridDim.x * blockDim.x) {
        if (t < m && size[t] >= mcs)
            continue;                              // big
        const i32 p = par[t];
        if (p < 0 || size[p] < mcs)
            continue;                              // not the top of a small subtree
        const i32 h = head[p];
        const u32 key = (u32)n - (u32)suf[t < m ? 2 * t : 2 * (i64)m + (t - m)];
        if (h < 0 || key >= (u32)n) {
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
            continue;
        }
        rec[key] = ((u64)(u32)cid[h] << 32) | (u32)p;
    }
}

// ---- exclusive scan of int32 flags (3 kernels) --------------------------------
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = FT * SC_ITEMS;

__device__ __forceinline__ i32 block_exclusive_scan(i32 v, i32 *sm, i32 *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    i32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const i32 y = __shfl_up_sync(FULL, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        i32 s = lane < nw ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const i32 y = __shfl_up_sync(FULL, s, o);
            if (lane >= o)
                s += y;
        }
        sm[lane] = s;
    }
    __syncthreads();
    const i32 before = warp ? sm[warp - 1] : 0;
    *total = sm[nw - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void scan_reduce_kernel(const i32 *in, i64 len, i32 *bsum)
{
    __shared__ i32 sm[32];
    const i64 base = blockIdx.x * (i64)SC_TILE + threadIdx.x * (i64)SC_ITEMS;
    i32 s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k)
        if (base + k < len)
            s += in[base + k];
    i32 total;
    block_exclusive_scan(s, sm, &total);
    if (threadIdx.x == 0)
        bsum[blockIdx.x] = total;
}

// One block: bsum[0..nb) becomes its exclusive scan; *total gets the sum.
__global__ void scan_top_kernel(i32 *bsum, i64 nb, i32 *total)
{
    __shared__ i32 sm[32];
    const i64 per = (nb + blockDim.x - 1) / blockDim.x;
    const i64 lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    i32 s = 0;
    for (i64 i = lo; i < hi; ++i)
        s += bsum[i];
    i32 tot;
    i32 run = block_exclusive_scan(s, sm, &tot);
    for (i64 i = lo; i < hi; ++i) {
        const i32 v = bsum[i];
        bsum[i] = run;
        run += v;
    }
    if (threadIdx.x == 0)
        *total = tot;
}

__global__ void scan_down_kernel(const i32 *in, i64 len, const i32 *bsum, i32 *out)
{
    __shared__ i32 sm[32];
    const i64 base = blockIdx.x * (i64)SC_TILE + threadIdx.x * (i64)SC_ITEMS;
    i32 v[SC_ITEMS];
    i32 s = 0;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        v[k] = base + k < len ? in[base + k] : 0;
        s += v[k];
    }
    i32 total;
    i32 run = bsum[blockIdx.x] + block_exclusive_scan(s, sm, &total);
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        if (base + k < len)
            out[base + k] = run;
        run += v[k];
    }
}

// ---- fill-forward scan of u64 records (3 kernels) ---------------------------------
// out[i] = the last record at or before i that is not NO_RECORD.
__device__ __forceinline__ u64 fill_op(u64 earlier, u64 later)
{
    return later != NO_RECORD ? later : earlier;
}

__device__ __forceinline__ u64 block_exclusive_fill(u64 v, u64 *sm, u64 *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(FULL, x, o);
        if (lane >= o)
            x = fill_op(y, x);
    }
    u64 before = __shfl_up_sync(FULL, x, 1);
    if (lane == 0)
        before = NO_RECORD;
    if (lane == 31)
        sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        u64 t = lane < nw ? sm[lane] : NO_RECORD;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(FULL, t, o);
            if (lane >= o)
                t = fill_op(y, t);
        }
        sm[lane] = t;
    }
    __syncthreads();
    const u64 warp_before = warp ? sm[warp - 1] : NO_RECORD;
    *total = sm[nw - 1];
    __syncthreads();
    return fill_op(warp_before, before);
}

__global__ void fill_reduce_kernel(const u64 *in, i64 len, u64 *bagg)
{
    __shared__ u64 sm[32];
    const i64 base = blockIdx.x * (i64)SC_TILE + threadIdx.x * (i64)SC_ITEMS;
    u64 a = NO_RECORD;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k)
        if (base + k < len)
            a = fill_op(a, in[base + k]);
    u64 total;
    block_exclusive_fill(a, sm, &total);
    if (threadIdx.x == 0)
        bagg[blockIdx.x] = total;
}

// One block: bagg[b] becomes the record carried into tile b.
__global__ void fill_top_kernel(u64 *bagg, i64 nb)
{
    __shared__ u64 sm[32];
    const i64 per = (nb + blockDim.x - 1) / blockDim.x;
    const i64 lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    u64 a = NO_RECORD;
    for (i64 i = lo; i < hi; ++i)
        a = fill_op(a, bagg[i]);
    u64 total;
    u64 run = block_exclusive_fill(a, sm, &total);
    for (i64 i = lo; i < hi; ++i) {
        const u64 v = bagg[i];
        bagg[i] = run;
        run = fill_op(run, v);
    }
}

__global__ void fill_down_kernel(u64 *data, i64 len, const u64 *bagg)
{
    __shared__ u64 sm[32];
    const i64 base = blockIdx.x * (i64)SC_TILE + threadIdx.x * (i64)SC_ITEMS;
    u64 v[SC_ITEMS];
    u64 a = NO_RECORD;
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        v[k] = base + k < len ? data[base + k] : NO_RECORD;
        a = fill_op(a, v[k]);
    }
    u64 total;
    u64 run = fill_op(bagg[blockIdx.x], block_exclusive_fill(a, sm, &total));
#pragma unroll
    for (int k = 0; k < SC_ITEMS; ++k) {
        run = fill_op(run, v[k]);
        if (base + k < len)
            data[base + k] = run;
    }
}

// ---- 4. exact stability sums ---------------------------------------------------
// (host-callable too, so that the arithmetic can be checked without a GPU)
__host__ __device__ __forceinline__ u64 double_bits(double t)
{
#ifdef __CUDA_ARCH__
    return (u64)__double_as_longlong(t);
#else
    u64 b;
    memcpy(&b, &t, sizeof b);
    return b;
#endif
}

__host__ __device__ __forceinline__ double bits_double(u64 b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double t;
    memcpy(&t, &b, sizeof t);
    return t;
#endif
}

__host__ __device__ __forceinline__ int leading_zeros(u32 x)
{
#ifdef __CUDA_ARCH__
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// Splits a non-negative double t that is a multiple of 2^-FIX_EXP into digits
// d[0..2] with t * 2^FIX_EXP = (d0 + d1 * 2^32 + d2 * 2^64) * 2^(32 * j0).
// Returns false for t == 0; a value outside that form sets *bad.
__host__ __device__ __forceinline__ bool split_digits(double t, int &j0, u32 &d0, u32 &d1,
                                                      u32 &d2, bool &bad)
{
    const u64 bits = double_bits(t);
    if ((bits << 1) == 0)
        return false;
    const int ex = (int)(bits >> 52);          // sign bit included: negative -> >= 2048
    if (ex == 0 || ex >= 2047) {
        bad = true;
        return false;
    }
    u64 M = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    int s = ex - 1075 + FIX_EXP;               // t * 2^FIX_EXP = M * 2^s
    if (s < 0) {
        const int sh = -s;
        if (sh >= 53 || (M & ((1ull << sh) - 1))) {
            bad = true;
            return false;
        }
        M >>= sh;
        s = 0;
    }
    j0 = s >> 5;
    const int r = s & 31;
    if (j0 + 2 >= NL) {
        bad = true;
        return false;
    }
    d0 = (u32)(M << r);
    const u64 t1 = M >> (32 - r);
    d1 = (u32)t1;
    d2 = (u32)(t1 >> 32);
    return true;
}

__global__ void cluster_init_kernel(i32 m, i64 Kmax, const i32 *start, const i32 *cid,
                                    const i32 *par, const i32 *head, const i32 *size,
                                    const float *w, i32 *cpar, i32 *ckids, i32 *ccnt, i32 *csize,
                                    i32 *cedge, double *birth, FlatCtrl *c)
{
    if (failed(c))
        return;
    const i32 root = c->root;
    for (i64 e = blockIdx.x * (i64)blockDim.x + threadIdx.x; e < m;
         e += (i64)gridDim.x * blockDim.x) {
        if (!start[e])
            continue;
        const i32 k = cid[e];
        const i32 hp = e == root ? -1 : head[par[e]];
        const i32 pk = e == root ? -1 : (hp >= 0 ? cid[hp] : (i32)Kmax);
        if (k >= Kmax || pk >= Kmax) {           // more clusters than n / mcs allows
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
            continue;
        }
        csize[k] = size[e];
        cedge[k] = (i32)e;
        if (e == root) {
            cpar[k] = -1;
            birth[k] = 0.0;
            c->root_cid = k;
            continue;
        }
        birth[k] = 1.0 / (double)w[par[e]];
        cpar[k] = pk;
        const i32 slot = atomicAdd(&ccnt[pk], 1);
        if (slot < 2)
            ckids[2 * (i64)pk + slot] = k;
        else
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
    }
}

// size(D) copies of fl(birth(D) - birth(C)), added to C's accumulator.
__global__ void child_terms_kernel(i32 K, const i32 *cpar, const i32 *csize,
                                   const double *birth, u64 *acc, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 pk = cpar[k];
        if (pk < 0)
            continue;
        const double d = birth[k] - birth[pk];
        int j0;
        u32 dg[3];
        bool bad = false;
        if (split_digits(d, j0, dg[0], dg[1], dg[2], bad)) {
            const u64 mult = (u64)(u32)csize[k];
            for (int q = 0; q < 3; ++q)
                if (dg[q])
                    atomicAdd((unsigned long long *)&acc[(i64)pk * NL + j0 + q],
                              (unsigned long long)(dg[q] * mult));
        }
        if (bad)
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
    }
}

// Every vertex: its cluster, and fl(lambda_leave - birth) into that cluster's
// accumulator.  Lanes of a warp with the same (cluster, digit position) add
// their digits first (16-bit halves, so the 32-lane sums cannot overflow),
// then one lane per group issues the atomics.
__global__ void leaf_terms_kernel(i32 m, i32 n, const u64 *suf, const u64 *rec, const float *w,
                                  const double *birth, u64 *acc, i32 *lcl, FlatCtrl *c)
{
    if (failed(c))
        return;
    const int lane = threadIdx.x & 31;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    for (i64 base = (blockIdx.x * (i64)blockDim.x + threadIdx.x) & ~(i64)31; base < n;
         base += stride) {
        const i64 x = base + lane;
        u64 key = (1ull << 63) | (u64)lane;    // unique: contributes nothing
        u32 dg[3] = {0, 0, 0};
        int j0 = 0;
        i32 k = 0;
        bool bad = false;
        if (x < n) {
            const u32 idx = (u32)n - (u32)suf[2 * (i64)m + x];
            const u64 r = idx < (u32)n ? rec[idx] : NO_RECORD;
            k = (i32)(r >> 32);
            const i32 p = (i32)(u32)r;
            if (r == NO_RECORD) {
                bad = true;
                k = 0;
            }
            lcl[x] = k;
            if (!bad) {
                const double t = 1.0 / (double)w[p] - birth[k];
                if (split_digits(t, j0, dg[0], dg[1], dg[2], bad))
                    key = ((u64)(u32)k << 4) | (u64)j0;
            }
        }
        if (bad)
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
        const u32 grp = __match_any_sync(FULL, key);
        u64 sum[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const u32 lo = __reduce_add_sync(grp, dg[q] & 0xFFFFu);
            const u32 hi = __reduce_add_sync(grp, dg[q] >> 16);
            sum[q] = (u64)lo + ((u64)hi << 16);
        }
        if (!(key >> 63) && lane == __ffs(grp) - 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (sum[q])
                    atomicAdd((unsigned long long *)&acc[(i64)k * NL + j0 + q],
                              (unsigned long long)sum[q]);
        }
    }
}

// Bits [pos, pos + cnt) (cnt <= 64) of the number held in 32-bit digits D.
__host__ __device__ __forceinline__ u64 digit_bits(const u32 *D, int pos, int cnt)
{
    if (pos < 0 || cnt <= 0)
        return 0;
    const int i = pos >> 5, off = pos & 31;
    auto dig = [&](int j) -> u64 { return j < NL ? (u64)D[j] : 0ull; };
    const u64 lo = dig(i) | (dig(i + 1) << 32);
    const u64 hi = dig(i + 2) | (dig(i + 3) << 32);
    const u64 v = off ? (lo >> off) | (hi << (64 - off)) : lo;
    return cnt == 64 ? v : v & ((1ull << cnt) - 1);
}

// The number held in NL 32-bit digits times 2^-FIX_EXP, rounded to the
// nearest double (ties to even).
__host__ __device__ __forceinline__ double round_fixed(const u32 *D)
{
    int top = -1;
    for (int j = NL - 1; j >= 0; --j)
        if (D[j]) {
            top = 32 * j + 31 - leading_zeros(D[j]);
            break;
        }
    if (top < 0)
        return 0.0;
    u64 mant;
    int e2 = top - FIX_EXP;                        // value in [2^e2, 2^(e2+1))
    if (top <= 52) {
        mant = digit_bits(D, 0, top + 1) << (52 - top);
    } else {
        const int sh = top - 52;
        mant = digit_bits(D, sh, 53);
        const bool guard = digit_bits(D, sh - 1, 1) != 0;
        bool sticky = false;
        const int below = sh - 1;                  // bits [0, below) break ties
        for (int j = 0; j < NL && 32 * j < below; ++j) {
            const int hi_bit = below - 32 * j;
            const u32 part = hi_bit >= 32 ? D[j] : (D[j] & ((1u << hi_bit) - 1));
            if (part) {
                sticky = true;
                break;
            }
        }
        if (guard && (sticky || (mant & 1))) {
            ++mant;
            if (mant == (1ull << 53)) {
                mant >>= 1;
                ++e2;
            }
        }
    }
    return bits_double(((u64)(e2 + 1023) << 52) | (mant & ((1ull << 52) - 1)));
}

// Carries between the 64-bit accumulator words, then round_fixed.
__global__ void finalize_kernel(i32 K, const u64 *acc, double *stab, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        u32 D[NL];
        u64 carry = 0;
        for (int j = 0; j < NL; ++j) {
            const u64 v = acc[k * NL + j] + carry;
            D[j] = (u32)v;
            carry = v >> 32;
        }
        if (carry) {
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
            continue;
        }
        stab[k] = round_fixed(D);
    }
}

// ---- 5. excess of mass -----------------------------------------------------------
// best(C) = max(stab(C), best(D1) + best(D2)) over the binary cluster tree,
// with exact sums (448-bit fixed point, unit 2^-FIX_EXP: stabilities are
// float64 multiples of 2^-180 below 2^213, and sums of at most 2^30 of them
// stay below 2^243).  The tree can be as deep as it is large (a caterpillar
// shedding one small cluster per level), so it is contracted in O(log K)
// rounds: leaves are numbered left to right in the dendrogram's tour order
// (the first and last leaf left out), and each round rakes the odd-numbered
// leaves that are left children, then those that are right children, then
// halves the numbers -- the classical schedule under which no two
// simultaneous rakes touch the same nodes.  Raking leaf l removes l and its
// parent p and hangs l's sibling s from p's parent; the edge above s carries
// f(x) = max(a, x + b) (a may be -inf), and such functions compose exactly:
//     f_s <- f_p o (x -> max(stab(p), k + f_s(x))),   k = f_l(best(l)).
// Replaying the rakes in reverse then gives every best(p) =
// max(stab(p), k + f_s(best(s))) from values already known.
struct __align__(8) Big {
    u32 d[NL];
};

__device__ __forceinline__ Big big_add(const Big &a, const Big &b)
{
    Big r;
    u64 c = 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        const u64 t = (u64)a.d[j] + b.d[j] + c;
        r.d[j] = (u32)t;
        c = t >> 32;
    }
    return r;
}

__device__ __forceinline__ bool big_less(const Big &a, const Big &b)
{
#pragma unroll
    for (int j = NL - 1; j >= 0; --j)
        if (a.d[j] != b.d[j])
            return a.d[j] < b.d[j];
    return false;
}

__device__ __forceinline__ Big big_from_double(double t, bool &bad)
{
    Big r;
#pragma unroll
    for (int j = 0; j < NL; ++j)
        r.d[j] = 0;
    int j0;
    u32 d0, d1, d2;
    if (split_digits(t, j0, d0, d1, d2, bad)) {
        r.d[j0] = d0;
        r.d[j0 + 1] = d1;
        r.d[j0 + 2] = d2;
    }
    return r;
}

// Per-cluster arrays of the contraction.
struct Eom {
    i32 *cur_par, *cur_kid, *leafnum, *rake_step, *rk_s, *a_inf, *rk_as_inf;
    Big *a, *b, *bstab, *best, *rk_k, *rk_as, *rk_bs;
};

constexpr i32 LEAF_INTERNAL = -1, LEAF_RAKED = -2;

// Orientation of the children (left = first in the tour, i.e. the larger
// suffix leaf count), identity edge functions, exact stabilities, and a flag
// at every leaf cluster's tour position (number of leaves before it).
__global__ void eom_prep_kernel(i32 K, i32 n, const i32 *cedge, const u64 *suf, const i32 *ckids,
                                const i32 *ccnt, const i32 *cpar, const double *stab, Eom E,
                                i32 *posflag, FlatCtrl *c)
{
    if (failed(c))
        return;
    const i32 root_cid = c->root_cid;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        bool bad = false;
        const Big bs = big_from_double(stab[k], bad);
        if (bad)
            set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
        E.bstab[k] = bs;
        E.cur_par[k] = cpar[k];
        E.a_inf[k] = 1;
        Big z;
#pragma unroll
        for (int j = 0; j < NL; ++j)
            z.d[j] = 0;
        E.b[k] = z;
        E.rake_step[k] = -1;
        if (ccnt[k] == 2) {
            i32 x = ckids[2 * k], y = ckids[2 * k + 1];
            if ((u32)suf[2 * (i64)cedge[x]] < (u32)suf[2 * (i64)cedge[y]]) {
                const i32 t = x;
                x = y;
                y = t;
            }
            E.cur_kid[2 * k] = x;
            E.cur_kid[2 * k + 1] = y;
            E.leafnum[k] = LEAF_INTERNAL;
        } else {
            E.leafnum[k] = 0;
            E.best[k] = bs;
            if (k != root_cid)
                posflag[n - (u32)suf[2 * (i64)cedge[k]]] = 1;
        }
    }
}

// Leaves get their left-to-right rank; the first and the last stay 0.
__global__ void eom_number_kernel(i32 K, i32 n, i32 n_leaves, const i32 *cedge, const u64 *suf,
                                  const i32 *rank, Eom E, FlatCtrl *c)
{
    if (failed(c))
        return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && c->n_leaves != n_leaves)
        set_status(&c->status, PANDORA_ERR_NOT_A_DENDROGRAM);
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        if (E.leafnum[k] != 0 || k == c->root_cid)
            continue;
        const i32 r = rank[n - (u32)suf[2 * (i64)cedge[k]]];
        E.leafnum[k] = (r >= 1 && r <= n_leaves - 2) ? r : 0;
    }
}

__global__ void rake_kernel(i32 K, int side, i32 step, Eom E, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 l = blockIdx.x * (i64)blockDim.x + threadIdx.x; l < K;
         l += (i64)gridDim.x * blockDim.x) {
        const i32 num = E.leafnum[l];
        if (num <= 0 || !(num & 1))
            continue;
        const i32 p = E.cur_par[l];
        const int sd = E.cur_kid[2 * (i64)p] == (i32)l ? 0 : 1;
        if (sd != side)
            continue;
        const i32 sb = E.cur_kid[2 * (i64)p + 1 - sd];
        const i32 g = E.cur_par[p];
        if (g < 0) {                               // never under this schedule
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
            continue;
        }
        // k = f_l(best(l)); l is a leaf of the original tree, best = stab
        Big kv = big_add(E.bstab[l], E.b[l]);
        if (!E.a_inf[l] && big_less(kv, E.a[l]))
            kv = E.a[l];
        const int as_inf = E.a_inf[sb];
        const Big as = E.a[sb], bs = E.b[sb];
        E.rk_s[p] = sb;
        E.rk_k[p] = kv;
        E.rk_as_inf[p] = as_inf;
        E.rk_as[p] = as;
        E.rk_bs[p] = bs;
        E.rake_step[p] = step;
        // h(x) = max(A, x + B): A = max(stab(p), k + a_s), B = k + b_s
        Big A = E.bstab[p];
        if (!as_inf) {
            const Big t = big_add(kv, as);
            if (big_less(A, t))
                A = t;
        }
        const Big Bv = big_add(kv, bs);
        // f_p o h = max(max(a_p, A + b_p), x + B + b_p)
        const Big bp = E.b[p];
        Big a2 = big_add(A, bp);
        if (!E.a_inf[p] && big_less(a2, E.a[p]))
            a2 = E.a[p];
        E.a[sb] = a2;
        E.a_inf[sb] = 0;
        E.b[sb] = big_add(Bv, bp);
        E.cur_par[sb] = g;
        const int gs = E.cur_kid[2 * (i64)g] == p ? 0 : 1;
        E.cur_kid[2 * (i64)g + gs] = sb;
        E.leafnum[l] = LEAF_RAKED;
    }
}

__global__ void renumber_kernel(i32 K, Eom E, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 num = E.leafnum[k];
        if (num <= 0)
            continue;
        if (num & 1)                               // an odd leaf that was not raked
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
        else
            E.leafnum[k] = num >> 1;
    }
}

// Every internal cluster but the root must have been raked.
__global__ void rake_check_kernel(i32 K, Eom E, FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x)
        if (E.leafnum[k] == LEAF_INTERNAL && k != c->root_cid && E.rake_step[k] < 0)
            set_status(&c->status, PANDORA_ERR_ITERATION_LIMIT);
}

__global__ void expand_step_kernel(i32 K, i32 step, Eom E, const FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 p = blockIdx.x * (i64)blockDim.x + threadIdx.x; p < K;
         p += (i64)gridDim.x * blockDim.x) {
        if (E.rake_step[p] != step)
            continue;
        Big v = big_add(E.best[E.rk_s[p]], E.rk_bs[p]);   // f_s(best(s)) at rake time
        if (!E.rk_as_inf[p] && big_less(v, E.rk_as[p]))
            v = E.rk_as[p];
        Big t = big_add(E.rk_k[p], v);
        if (big_less(t, E.bstab[p]))
            t = E.bstab[p];
        E.best[p] = t;
    }
}

// Keep C (for now) when stab(C) >= best(D1) + best(D2), exactly; a cluster
// without children is kept; the root is not a candidate.
__global__ void decide_kernel(i32 K, const i32 *ckids, const i32 *ccnt, Eom E, i32 *sel,
                              const FlatCtrl *c)
{
    if (failed(c))
        return;
    const i32 root_cid = c->root_cid;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        if (k == root_cid) {
            sel[k] = 0;
            continue;
        }
        if (ccnt[k] == 0) {
            sel[k] = 1;
            continue;
        }
        const Big kids = big_add(E.best[ckids[2 * k]], E.best[ckids[2 * k + 1]]);
        sel[k] = !big_less(E.bstab[k], kids);
    }
}

// ---- 6. labels --------------------------------------------------------------------
__global__ void top_init_kernel(i32 K, const i32 *cpar, const i32 *sel, i32 *up, i32 *val,
                                const FlatCtrl *c)
{
    if (failed(c))
        return;
    const i32 root_cid = c->root_cid;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 p = cpar[k];
        up[k] = (k == root_cid || p == root_cid) ? -1 : p;
        val[k] = (k != root_cid && sel[k]) ? (i32)k : -1;
    }
}

// val: the topmost selected cluster among k and its 2^r nearest ancestors.
__global__ void top_step_kernel(i32 K, const i32 *up, const i32 *val, i32 *up2, i32 *val2,
                                const FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 k = blockIdx.x * (i64)blockDim.x + threadIdx.x; k < K;
         k += (i64)gridDim.x * blockDim.x) {
        const i32 a = up[k];
        if (a >= 0) {
            const i32 va = val[a];
            val2[k] = va >= 0 ? va : val[k];
            up2[k] = up[a];
        } else {
            val2[k] = val[k];
            up2[k] = -1;
        }
    }
}

__global__ void label_raw_kernel(i32 n, const i32 *lcl, const i32 *val, i32 *lab, i32 *first,
                                 const FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < n;
         x += (i64)gridDim.x * blockDim.x) {
        const i32 L = val[lcl[x]];
        lab[x] = L;
        if (L >= 0)
            atomicMin(&first[L], (i32)x);
    }
}

__global__ void first_flag_kernel(i32 n, const i32 *lab, const i32 *first, i32 *flag,
                                  const FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < n;
         x += (i64)gridDim.x * blockDim.x) {
        const i32 L = lab[x];
        flag[x] = L >= 0 && first[L] == (i32)x;
    }
}

__global__ void label_final_kernel(i32 n, const i32 *lab, const i32 *first, const i32 *rank,
                                   const double *stab, i32 *labels, double *stab_out,
                                   const FlatCtrl *c)
{
    if (failed(c))
        return;
    for (i64 x = blockIdx.x * (i64)blockDim.x + threadIdx.x; x < n;
         x += (i64)gridDim.x * blockDim.x) {
        const i32 L = lab[x];
        if (L < 0) {
            labels[x] = -1;
            continue;
        }
        const i32 f = first[L];
        const i32 r = rank[f];
        labels[x] = r;
        if (stab_out && f == (i32)x)
            stab_out[r] = stab[L];
    }
}

// ---- host side ------------------------------------------------------------------------
int ceil_log2(i64 v)
{
    int r = 0;
    while (((i64)1 << r) < v)
        ++r;
    return r;
}

struct Carve {
    char *p;
    size_t off = 0;
    template <class T>
    T *take(i64 count)
    {
        off = (off + 255) & ~(size_t)255;
        T *r = reinterpret_cast<T *>(p + off);
        off += (size_t)(count > 0 ? count : 1) * sizeof(T);
        return r;
    }
};

struct FlatLayout {
    FlatCtrl *ctrl;
    i32 *par, *cnt, *kids, *size, *head, *start, *cid, *bsum, *lcl, *lab, *flag, *rank;
    u64 *arcA, *arcB;       // tour words, then suffix sums (A); (segment, offset) (B)
    i32 *sid_of, *spl;      // ruling set: splitter id per arc, splitter arcs
    u64 *segA, *segB;       // ruling set: segment words
    i64 rs_cap;
    i32 *bsid, *bspl, *seg_of, *nxA, *nxB, *hdA, *hdB;   // path heads (ruling set)
    i64 bp_cap;
    u64 *rec, *bagg;        // leaf records and their fill scan
    i32 *first, *cpar, *ckids, *ccnt, *csize, *cedge, *sel, *upA, *upB, *valA, *valB;
    double *birth, *stab;
    u64 *acc;
    Eom eom;
    size_t bytes;
};

FlatLayout flat_layout(char *base, i64 n, i64 Kmax)
{
    const i64 m = n - 1, N = m + n, L = 2 * m + n;
    const i64 nb = (N + SC_TILE - 1) / SC_TILE;
    Carve cv{base};
    FlatLayout l;
    l.ctrl = cv.take<FlatCtrl>(1);
    l.par = cv.take<i32>(N);
    l.cnt = cv.take<i32>(m);
    l.kids = cv.take<i32>(2 * m);
    l.size = cv.take<i32>(m);
    l.head = cv.take<i32>(m);
    l.start = cv.take<i32>(m);
    l.cid = cv.take<i32>(m);
    l.bsum = cv.take<i32>(nb);
    l.lcl = cv.take<i32>(n);
    l.lab = cv.take<i32>(n);
    l.flag = cv.take<i32>(n);
    l.rank = cv.take<i32>(n);
    l.arcA = cv.take<u64>(L);
    l.arcB = cv.take<u64>(L);
    l.rs_cap = rs_capacity(L);
    l.sid_of = cv.take<i32>(L);
    l.spl = cv.take<i32>(l.rs_cap);
    l.segA = cv.take<u64>(l.rs_cap);
    l.segB = cv.take<u64>(l.rs_cap);
    l.bp_cap = m / 48 + 4096 + 2 * Kmax;
    l.bsid = cv.take<i32>(m);
    l.seg_of = cv.take<i32>(m);
    l.bspl = cv.take<i32>(l.bp_cap);
    l.nxA = cv.take<i32>(l.bp_cap);
    l.nxB = cv.take<i32>(l.bp_cap);
    l.hdA = cv.take<i32>(l.bp_cap);
    l.hdB = cv.take<i32>(l.bp_cap);
    l.rec = cv.take<u64>(n);
    l.bagg = cv.take<u64>(nb);
    l.bytes = cv.off + 256;
    return l;
}

// The per-cluster arrays (about 600 bytes per cluster, most of it the tree
// contraction's 448-bit edge functions), carved from a second block once the
// cluster count K is known.
size_t cluster_layout(FlatLayout &l, char *base, i64 Kmax)
{
    Carve cv{base};
    l.first = cv.take<i32>(Kmax);
    l.cpar = cv.take<i32>(Kmax);
    l.ckids = cv.take<i32>(2 * Kmax);
    l.ccnt = cv.take<i32>(Kmax);
    l.csize = cv.take<i32>(Kmax);
    l.cedge = cv.take<i32>(Kmax);
    l.sel = cv.take<i32>(Kmax);
    l.upA = cv.take<i32>(Kmax);
    l.upB = cv.take<i32>(Kmax);
    l.valA = cv.take<i32>(Kmax);
    l.valB = cv.take<i32>(Kmax);
    l.birth = cv.take<double>(Kmax);
    l.stab = cv.take<double>(Kmax);
    l.acc = cv.take<u64>(Kmax * NL);
    Eom &E = l.eom;
    E.cur_par = cv.take<i32>(Kmax);
    E.cur_kid = cv.take<i32>(2 * Kmax);
    E.leafnum = cv.take<i32>(Kmax);
    E.rake_step = cv.take<i32>(Kmax);
    E.rk_s = cv.take<i32>(Kmax);
    E.a_inf = cv.take<i32>(Kmax);
    E.rk_as_inf = cv.take<i32>(Kmax);
    E.a = cv.take<Big>(Kmax);
    E.b = cv.take<Big>(Kmax);
    E.bstab = cv.take<Big>(Kmax);
    E.best = cv.take<Big>(Kmax);
    E.rk_k = cv.take<Big>(Kmax);
    E.rk_as = cv.take<Big>(Kmax);
    E.rk_bs = cv.take<Big>(Kmax);
    return cv.off + 256;
}

// Grid of a grid-stride kernel: one block per FT items, at most 8 blocks per
// SM of the device current at the first call (thread-safe initialisation).
int grid_for(i64 count)
{
    static const int sms = [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        return n;
    }();
    const i64 want = (count + FT - 1) / FT;
    const i64 cap = (i64)sms * 8;
    return (int)(want < 1 ? 1 : want < cap ? want : cap);
}

void scan_flags(const i32 *in, i64 len, i32 *bsum, i32 *out, i32 *total, cudaStream_t s)
{
    const i64 nb = (len + SC_TILE - 1) / SC_TILE;
    if (nb == 0)
        return;
    scan_reduce_kernel<<<(unsigned)nb, FT, 0, s>>>(in, len, bsum);
    scan_top_kernel<<<1, 1024, 0, s>>>(bsum, nb, total);
    scan_down_kernel<<<(unsigned)nb, FT, 0, s>>>(in, len, bsum, out);
}

// Launches every step on s; returns after reading the status.  The only
// host synchronisation inside is the read of the cluster count.
void fill_records(u64 *data, i64 len, u64 *bagg, cudaStream_t s)
{
    const i64 nb = (len + SC_TILE - 1) / SC_TILE;
    if (nb == 0)
        return;
    fill_reduce_kernel<<<(unsigned)nb, FT, 0, s>>>(data, len, bagg);
    fill_top_kernel<<<1, 1024, 0, s>>>(bagg, nb);
    fill_down_kernel<<<(unsigned)nb, FT, 0, s>>>(data, len, bagg);
}

int run_flat_on(FlatLayout &l, const i32 *ep, const i32 *vp, const float *w, i64 n, i32 mcs,
                i64 Kmax, i32 *labels, double *stab_out, i64 *n_clusters, cudaMemPool_t pool,
                void **cluster_ws, cudaStream_t s)
{
    const i64 m = n - 1, N = m + n, L = 2 * m + n;
    FlatCtrl *c = l.ctrl;
    const i32 mi = (i32)m, ni = (i32)n;
    cudaMemsetAsync(c, 0, sizeof(FlatCtrl), s);
    kids_init_kernel<<<grid_for(m), FT, 0, s>>>(mi, l.kids, l.cnt);

    // 1. parents and validation
    flat_parents_kernel<<<grid_for(N), FT, 0, s>>>(ep, vp, w, mi, ni, l.par, l.cnt, l.kids, c);
    flat_check_kernel<<<grid_for(m), FT, 0, s>>>(w, mi, l.par, l.cnt, c);
    if (n >= mcs) {
        // 2. leaf counts
        tour_init_kernel<<<grid_for(L), FT, 0, s>>>(mi, ni, l.par, l.kids, l.arcA, c);
        cudaMemsetAsync(l.segA, 0xFF, sizeof(u64) * l.rs_cap, s);   // unused: next = -1
        rs_pick_kernel<<<grid_for(L), FT, 0, s>>>(L, l.sid_of, l.spl, l.rs_cap, c);
        rs_walk_kernel<<<grid_for(l.rs_cap), FT, 0, s>>>(l.arcA, l.arcB, l.sid_of, l.spl,
                                                         l.rs_cap, L, l.segA, c);
        u64 *in = l.segA, *out = l.segB;
        for (int r = ceil_log2(l.rs_cap); r > 0; --r) {
            rank_step_kernel<<<grid_for(l.rs_cap), FT, 0, s>>>(in, out, l.rs_cap, c);
            u64 *t = in;
            in = out;
            out = t;
        }
        rs_final_kernel<<<grid_for(L), FT, 0, s>>>(l.arcB, in, l.rs_cap, L, l.arcA, c);
        const u64 *suf = l.arcA;
        sizes_kernel<<<grid_for(m), FT, 0, s>>>(suf, mi, ni, l.size, c);
        // 3. starts, the start above every big edge, cluster ids, leaf records
        start_kernel<<<grid_for(m), FT, 0, s>>>(mi, mcs, l.par, l.kids, l.size, l.start, l.head,
                                                c);
        cudaMemsetAsync(l.seg_of, 0xFF, sizeof(i32) * m, s);
        cudaMemsetAsync(l.nxA, 0xFF, sizeof(i32) * l.bp_cap, s);
        cudaMemsetAsync(l.hdA, 0xFF, sizeof(i32) * l.bp_cap, s);
        path_pick_kernel<<<grid_for(m), FT, 0, s>>>(mi, mcs, l.kids, l.size, l.start, l.bsid,
                                                    l.bspl, l.bp_cap, c);
        path_walk_kernel<<<grid_for(l.bp_cap), FT, 0, s>>>(mi, l.par, l.start, l.bsid, l.bspl,
                                                           l.bp_cap, l.seg_of, l.nxA, l.hdA, c);
        {
            // pointer jumping over the segments until every one has its start
            // (a path of q segments needs ceil(log2 q) rounds; paths are short)
            FlatCtrl h{};
            if (cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return PANDORA_ERR_CUDA;
            if (h.status)
                return h.status;
            const i64 cnt = (i64)h.bp_count < l.bp_cap ? (i64)h.bp_count : l.bp_cap;
            i32 *na = l.nxA, *ha = l.hdA, *nb = l.nxB, *hb = l.hdB;
            for (int r = ceil_log2(cnt) + 1; r > 0 && cnt > 0; --r) {
                cudaMemsetAsync(&c->unresolved, 0, sizeof(u32), s);
                seg_jump_kernel<<<grid_for(cnt), FT, 0, s>>>(cnt, na, ha, nb, hb, &c->unresolved,
                                                             c);
                i32 *t = na;
                na = nb;
                nb = t;
                t = ha;
                ha = hb;
                hb = t;
                u32 open = 0;
                if (cudaMemcpyAsync(&open, &c->unresolved, sizeof(u32), cudaMemcpyDeviceToHost,
                                    s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return PANDORA_ERR_CUDA;
                if (open == 0)
                    break;
            }
            path_final_kernel<<<grid_for(m), FT, 0, s>>>(mi, mcs, l.size, l.start, l.seg_of, ha,
                                                         l.bp_cap, l.head, c);
        }
        scan_flags(l.start, m, l.bsum, l.cid, &c->n_starts, s);
        cudaMemsetAsync(l.rec, 0xFF, sizeof(u64) * n, s);
        anchor_mark_kernel<<<grid_for(N), FT, 0, s>>>(mi, ni, mcs, l.par, l.size, l.head, l.cid,
                                                      suf, l.rec, c);
        fill_records(l.rec, n, l.bagg, s);
        {
            // the cluster count is known now: size the per-cluster arrays by it
            FlatCtrl h{};
            if (cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return PANDORA_ERR_CUDA;
            if (h.status)
                return h.status;
            if (h.n_starts < 1 || (i64)h.n_starts > Kmax)
                return PANDORA_ERR_NOT_A_DENDROGRAM;   // more clusters than n / mcs allows
            Kmax = h.n_starts;
            const size_t cbytes = cluster_layout(l, nullptr, Kmax);
            if (cudaMallocFromPoolAsync(cluster_ws, cbytes, pool, s) != cudaSuccess) {
                cudaGetLastError();
                *cluster_ws = nullptr;
                return PANDORA_ERR_OUT_OF_MEMORY;
            }
            cluster_layout(l, (char *)(((uintptr_t)*cluster_ws + 255) & ~(uintptr_t)255), Kmax);
        }
        cudaMemsetAsync(l.ccnt, 0, sizeof(i32) * Kmax, s);
        cudaMemsetAsync(l.sel, 0, sizeof(i32) * Kmax, s);
        cudaMemsetAsync(l.acc, 0, sizeof(u64) * Kmax * NL, s);
        cudaMemsetAsync(l.first, 0x7F, sizeof(i32) * Kmax, s);
        cluster_init_kernel<<<grid_for(m), FT, 0, s>>>(mi, Kmax, l.start, l.cid, l.par, l.head,
                                                       l.size, w, l.cpar, l.ckids, l.ccnt,
                                                       l.csize, l.cedge, l.birth, c);
        FlatCtrl h{};
        if (cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PANDORA_ERR_CUDA;
        if (h.status)
            return h.status;
        const i32 K = h.n_starts;
        if (K < 1 || K > Kmax)
            return PANDORA_ERR_NOT_A_DENDROGRAM;
        // 4. stabilities
        child_terms_kernel<<<grid_for(K), FT, 0, s>>>(K, l.cpar, l.csize, l.birth, l.acc, c);
        leaf_terms_kernel<<<grid_for(n), FT, 0, s>>>(mi, ni, suf, l.rec, w, l.birth, l.acc,
                                                     l.lcl, c);
        finalize_kernel<<<grid_for(K), FT, 0, s>>>(K, l.acc, l.stab, c);
        // 5. excess of mass (K == 1: no candidate, nothing kept)
        if (K >= 3) {
            const Eom &E = l.eom;
            const i32 n_leaves = (K + 1) / 2;
            cudaMemsetAsync(l.flag, 0, sizeof(i32) * n, s);
            eom_prep_kernel<<<grid_for(K), FT, 0, s>>>(K, ni, l.cedge, suf, l.ckids, l.ccnt,
                                                       l.cpar, l.stab, E, l.flag, c);
            scan_flags(l.flag, n, l.bsum, l.rank, &c->n_leaves, s);
            eom_number_kernel<<<grid_for(K), FT, 0, s>>>(K, ni, n_leaves, l.cedge, suf, l.rank,
                                                         E, c);
            const int rounds = ceil_log2(n_leaves) + 1;
            for (int r = 0; r < rounds; ++r) {
                rake_kernel<<<grid_for(K), FT, 0, s>>>(K, 0, 2 * r, E, c);
                rake_kernel<<<grid_for(K), FT, 0, s>>>(K, 1, 2 * r + 1, E, c);
                renumber_kernel<<<grid_for(K), FT, 0, s>>>(K, E, c);
            }
            rake_check_kernel<<<grid_for(K), FT, 0, s>>>(K, E, c);
            for (int t = 2 * rounds - 1; t >= 0; --t)
                expand_step_kernel<<<grid_for(K), FT, 0, s>>>(K, t, E, c);
            decide_kernel<<<grid_for(K), FT, 0, s>>>(K, l.ckids, l.ccnt, E, l.sel, c);
        }
        // 6. labels
        top_init_kernel<<<grid_for(K), FT, 0, s>>>(K, l.cpar, l.sel, l.upA, l.valA, c);
        i32 *ua = l.upA, *va = l.valA, *ub = l.upB, *vb = l.valB;
        for (int r = ceil_log2(K) + 1; r > 0; --r) {
            top_step_kernel<<<grid_for(K), FT, 0, s>>>(K, ua, va, ub, vb, c);
            i32 *t = ua;
            ua = ub;
            ub = t;
            t = va;
            va = vb;
            vb = t;
        }
        label_raw_kernel<<<grid_for(n), FT, 0, s>>>(ni, l.lcl, va, l.lab, l.first, c);
        first_flag_kernel<<<grid_for(n), FT, 0, s>>>(ni, l.lab, l.first, l.flag, c);
        scan_flags(l.flag, n, l.bsum, l.rank, &c->n_selected, s);
        label_final_kernel<<<grid_for(n), FT, 0, s>>>(ni, l.lab, l.first, l.rank, l.stab, labels,
                                                      stab_out, c);
    } else {
        cudaMemsetAsync(labels, 0xFF, sizeof(i32) * n, s);   // too few points: all noise
    }
    if (cudaGetLastError() != cudaSuccess)
        return PANDORA_ERR_CUDA;
    FlatCtrl h{};
    if (cudaMemcpyAsync(&h, c, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    if (h.status)
        return h.status;
    if (n_clusters)
        *n_clusters = n >= mcs ? h.n_selected : 0;
    return PANDORA_OK;
}

int run_flat(const i32 *ep, const i32 *vp, const float *w, i64 n, i32 mcs, i32 *labels,
             double *stab_out, i64 *n_clusters, cudaStream_t s)
{
    const i64 Kmax = 2 * (n / mcs) + 1;
    const size_t bytes = flat_layout(nullptr, n, Kmax).bytes;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    cudaMemPool_t pool = flat_pool(dev);
    if (!pool)
        return PANDORA_ERR_CUDA;
    void *ws = nullptr, *cws = nullptr;
    if (cudaMallocFromPoolAsync(&ws, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return PANDORA_ERR_OUT_OF_MEMORY;
    }
    FlatLayout l = flat_layout((char *)ws, n, Kmax);
    const int st = run_flat_on(l, ep, vp, w, n, mcs, Kmax, labels, stab_out, n_clusters, pool,
                               &cws, s);
    if (cws)
        cudaFreeAsync(cws, s);
    cudaFreeAsync(ws, s);
    if (st != PANDORA_OK)
        cudaStreamSynchronize(s);
    return st;
}

}  // namespace

extern "C" int pandora_hdbscan_labels(const int32_t *edge_parent, const int32_t *vertex_parent,
                                      const float *w, int64_t n_vertices,
                                      int32_t min_cluster_size, int32_t *labels,
                                      double *cluster_stability, int64_t *n_clusters,
                                      void *stream)
{
    if (n_vertices < 0 || min_cluster_size < 2)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (n_vertices > PANDORA_FLAT_MAX_VERTICES)
        return PANDORA_ERR_SIZE_LIMIT;
    if (n_vertices > 0 && (!labels || !vertex_parent))
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (n_vertices > 1 && (!edge_parent || !w))
        return PANDORA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_vertices <= 1) {
        if (n_vertices == 1 && cudaMemsetAsync(labels, 0xFF, sizeof(int32_t), s) != cudaSuccess)
            return PANDORA_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess)
            return PANDORA_ERR_CUDA;
        if (n_clusters)
            *n_clusters = 0;
        return PANDORA_OK;
    }
    return run_flat(edge_parent, vertex_parent, w, n_vertices, min_cluster_size, labels,
                    cluster_stability, n_clusters, s);
}

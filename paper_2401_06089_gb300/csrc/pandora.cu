// Host orchestration and C ABI of the dendrogram library (include/pandora.h).
//
// Algorithm 1 of the paper, one tree or a forest of trees at once:
//   1. sort the edges by (weight, index)              sort.cu   (Section 3.1)
//   2. contraction levels until no alpha-edge is left levels.cu (Section 3.2)
//   3. chain key of every edge                        expand.cu (Section 3.3.2)
//   4. sort by chain key, link each chain             sort.cu, expand.cu (3.3.3)
// Between levels the host reads back two counters (the next level's edges and
// vertices) to size the next launches; nothing else leaves the device.
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace pandora {
namespace {


// ---- optional instrumentation (pandora_profile_*) -------------------------
enum Slot : int {
    K_HIST_WEIGHTS, K_SORT_WEIGHTS, K_MARK, K_PTR_INIT, K_COMPRESS, K_COMPACT, K_EXPAND,
    K_SORT_CHAINS, K_LINK, K_CHECK_OFFSETS, K_FILL, K_INIT_LEVEL, K_SMALL, K_GATHER, K_TAIL,
    K_SLOTS
};
static_assert(K_SLOTS <= PANDORA_PROFILE_SLOTS, "profile slots");
const char *const kSlotNames[K_SLOTS] = {
    "hist_weights", "onesweep_weights", "mark", "ptr_init", "compress", "compact", "expand",
    "onesweep_chains", "link", "check_offsets", "fill", "init_level", "small_tree",
    "gather_scatter", "tail_levels"};

struct Profiler {
    std::mutex mu;
    bool timing = false;
    i64 launches[K_SLOTS] = {};
    i64 kernels[K_SLOTS] = {};
    i64 elements[K_SLOTS] = {};
    double ms[K_SLOTS] = {};
    std::vector<cudaEvent_t> free_events;
};
Profiler &profiler()
{
    static Profiler p;
    return p;
}

// Counts every launch of one call; with timing on, brackets each launch with
// a CUDA event pair on the launching stream and adds the elapsed times to the
// process-wide totals once the call's work is complete.
class CallTimer {
  public:
    // Timing needs a host synchronisation at the end of the call, so it is
    // only done for blocking calls; asynchronous calls only count launches.
    CallTimer(cudaStream_t s, bool blocking) : s_(s)
    {
        Profiler &p = profiler();
        std::lock_guard<std::mutex> lock(p.mu);
        timing_ = p.timing && blocking;
    }
    ~CallTimer() { flush(); }

    template <class F> void launch(int slot, i64 elements, F &&f) { launch(slot, elements, 1, f); }

    // `kernels`: CUDA kernels the step launches
    template <class F> void launch(int slot, i64 elements, int kernels, F &&f)
    {
        cudaEvent_t a = nullptr, b = nullptr;
        if (timing_) {
            a = get();
            b = get();
            if (a)
                cudaEventRecord(a, s_);
        }
        f();
        if (timing_ && b)
            cudaEventRecord(b, s_);
        recs_.push_back({slot, elements, kernels, a, b});
    }

  private:
    struct Rec {
        int slot;
        i64 elements;
        int kernels;
        cudaEvent_t a, b;
    };
    cudaEvent_t get()
    {
        Profiler &p = profiler();
        {
            std::lock_guard<std::mutex> lock(p.mu);
            if (!p.free_events.empty()) {
                cudaEvent_t e = p.free_events.back();
                p.free_events.pop_back();
                return e;
            }
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess)
            return nullptr;
        return e;
    }
    void flush()
    {
        if (recs_.empty())
            return;
        if (timing_)
            cudaStreamSynchronize(s_);
        Profiler &p = profiler();
        std::lock_guard<std::mutex> lock(p.mu);
        for (const Rec &r : recs_) {
            p.launches[r.slot] += 1;
            p.kernels[r.slot] += r.kernels;
            p.elements[r.slot] += r.elements;
            if (r.a && r.b) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
                    p.ms[r.slot] += ms;
            }
            if (r.a)
                p.free_events.push_back(r.a);
            if (r.b)
                p.free_events.push_back(r.b);
        }
        recs_.clear();
        cudaGetLastError();
    }
    cudaStream_t s_;
    bool timing_ = false;
    std::vector<Rec> recs_;
};

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Levels with more vertices than this (a word array above 256 MB, twice L2)
// mark by buckets of 2^MARK_BUCKET_SHIFT vertices (16 MB of words each;
// 21 measured 0.13 ms faster than 22 on all levels of a 10^8-edge tree).
// Measured on the 10^8-vertex random recursive tree: level 0 (10^8 vertices)
// 6.4 -> 4.3 ms with buckets; level 1 (2.6*10^7 vertices) is faster direct
// (1.0 vs 1.1 ms).
#ifndef PANDORA_MARK_DIRECT_MAX
#define PANDORA_MARK_DIRECT_MAX (i64(1) << 25)
#endif
#ifndef PANDORA_MARK_BUCKET_SHIFT
#define PANDORA_MARK_BUCKET_SHIFT 21
#endif
constexpr i64 MARK_DIRECT_MAX_VERTICES = PANDORA_MARK_DIRECT_MAX;
// Level 0 goes bucketed from a lower size: there the bucketed form also runs
// the flag pass, which removes two random reads per vertex from ptr_init and
// one per contracted edge from compact.  Random recursive trees, ms per
// dendrogram, direct / bucketed level 0: 3.2*10^7 edges 8.86 / 8.26,
// 2.4*10^7 6.33 / 6.15, 1.2*10^7 3.32 / 3.47, 6*10^6 2.10 / 2.26.
#ifndef PANDORA_MARK_DIRECT_MAX0
#define PANDORA_MARK_DIRECT_MAX0 (i64(1) << 24)
#endif
constexpr i64 MARK_DIRECT_MAX0_VERTICES = PANDORA_MARK_DIRECT_MAX0;
// Link stores edge_parent by caller-id buckets of 2^LINK_BUCKET_SHIFT ids
// (8 MB of edge_parent each; 21 measured 0.07 ms faster than 22 at 10^8
// edges) above LINK_BUCKET_MIN_EDGES edges.
#ifndef PANDORA_LINK_BUCKET_MIN
#define PANDORA_LINK_BUCKET_MIN (i64(1) << 25)
#endif
#ifndef PANDORA_LINK_BUCKET_SHIFT
#define PANDORA_LINK_BUCKET_SHIFT 21
#endif
constexpr i64 LINK_BUCKET_MIN_EDGES = PANDORA_LINK_BUCKET_MIN;
constexpr int LINK_BUCKET_SHIFT = PANDORA_LINK_BUCKET_SHIFT;
constexpr int MARK_BUCKET_SHIFT = PANDORA_MARK_BUCKET_SHIFT;

// Digit plan of the chain-key sort: keys are 2 * rank + side below 2M and
// root keys 2M .. 2M + T - 1, so the plan follows the bits of 2M + T - 1.
// PANDORA_CHAIN_WIDE_DIGITS=0 keeps 8-bit digits at every key width.
#ifndef PANDORA_CHAIN_WIDE_DIGITS
#define PANDORA_CHAIN_WIDE_DIGITS 1
#endif
DigitPlan chain_digit_plan(i64 M, i64 T)
{
    const u64 max_key = (u64)(2 * M) + (u64)T - 1;
    int bits = 0;
    while (bits < 32 && (max_key >> bits) != 0)
        ++bits;
    if (!PANDORA_CHAIN_WIDE_DIGITS && bits > 24 && bits <= 27)
        bits = 31;   // four 8-bit passes
    return digit_plan(bits);
}

struct Layout {
    size_t ctrl, keysA, keysB, valsA, valsB, perm, ab0, lb, min_word, ptr;
    size_t deep, uf, root_of;
    size_t kept_rec, abX, erX, abY, erY, lev, start, eflag, troots, total;
    i64 kept_cap, half_cap, lb_words;
};

Layout make_layout(i64 M, i64 T)
{
    const i64 N = M + T;
    Layout L{};
    size_t off = 0;
    auto take = [&](i64 bytes) {
        const size_t o = off;
        off = align_up(off + (size_t)std::max<i64>(bytes, 0));
        return o;
    };
    L.ctrl = take(sizeof(Ctrl));
    L.keysA = take(M * 4);
    L.keysB = take(M * 4);
    L.valsA = take(M * 4);
    L.valsB = take(M * 4);
    L.perm = take(M * 4);
    L.ab0 = take(M * 8);
    // look-back words of the widest pass (the chain sort may use 9- or 10-bit digits)
    const DigitPlan cpl = chain_digit_plan(M, T);
    int widest = 8;
    for (int q = 0; q < cpl.n; ++q)
        widest = std::max(widest, cpl.width[q]);
    const i64 os_words = onesweep_tiles(M) * ((i64)1 << widest);
    const i64 lv_words = level_tiles(N) + 1 + level_tiles(M) + 1;
    L.lb_words = std::max(os_words, lv_words);
    L.lb = take(L.lb_words * 8);
    L.min_word = take(N * 8);
    L.ptr = take(N * 4);
    L.deep = take(N * 4);
    L.uf = take(N * 4);
    L.root_of = take(N * 4);
    // vertices of all levels >= 1: n_l = m_l + T and sum_{l>=1} m_l <= M
    L.kept_cap = M + (i64)MAX_LEVELS * T + 64;
    L.kept_rec = take(L.kept_cap * 8);
    // edges of levels >= 1 (ping-pong): m_1 <= M / 2 and m_{l+1} <= m_l / 2
    L.half_cap = M / 2 + 1;
    L.abX = take(L.half_cap * 8);
    L.erX = take(L.half_cap * 4);
    L.abY = take(L.half_cap * 8);
    L.erY = take(L.half_cap * 4);
    L.lev = take(M);
    L.start = take(M * 4);
    L.eflag = take(eflag_words(M) * 4);
    L.troots = take(T * 8);   // tree_roots, tree_root_id (forests)
    L.total = off + 256;   // slack for aligning an unaligned base
    return L;
}

#define PANDORA_CUDA(call)                 \
    do {                                   \
        if ((call) != cudaSuccess)         \
            return PANDORA_ERR_CUDA;       \
    } while (0)

// Host copy of the head of the control block (status, level count, level sizes).
struct HostCounters {
    int status;
    int n_levels;
    u64 lvl_m[MAX_LEVELS + 1];
    u64 lvl_n[MAX_LEVELS + 1];
};
static_assert(offsetof(Ctrl, lvl_n) + sizeof(u64) * (MAX_LEVELS + 1) == sizeof(HostCounters),
              "HostCounters mirrors the head of Ctrl");

int read_counters(const Ctrl *ctrl, HostCounters *h, cudaStream_t s)
{
    PANDORA_CUDA(cudaMemcpyAsync(h, ctrl, sizeof(HostCounters), cudaMemcpyDeviceToHost, s));
    PANDORA_CUDA(cudaStreamSynchronize(s));
    return PANDORA_OK;
}

// Passes of an 8-bit LSD sort that actually move keys (a pass whose digit is
// the same for every key is the identity and is skipped).
std::vector<int> useful_passes(const u32 (*hist)[RADIX], int n_passes, i64 m)
{
    std::vector<int> out;
    for (int p = 0; p < n_passes; ++p) {
        bool trivial = false;
        for (int d = 0; d < RADIX; ++d)
            if ((i64)hist[p][d] == m)
                trivial = true;
        if (!trivial)
            out.push_back(p);
    }
    return out;
}

// Worst-case number of contraction levels: a tree of m edges has at most
// (m - 1) / 2 alpha-edges (Section 4.2), a forest at most m / 2, so level l
// has at most floor(M / 2^l) edges and the loop ends within
// ceil(log2(M + 1)) levels.
int level_bound(i64 M)
{
    int L = 0;
    while (L < MAX_LEVELS && (M >> L) > 0)
        ++L;
    return L;
}

// The whole pipeline on one workspace.
//   blocking: the host reads the level sizes after every level (exact launch
//             sizes, loop ends at the first level without alpha-edges, trivial
//             sort passes skipped) and returns the device status;
//   !blocking: everything is enqueued for the worst case (level_bound levels,
//             every sort pass) with no host synchronisation and no allocation,
//             so the call can be captured in a CUDA graph; kernels of levels
//             past the last one exit at once.  The device status stays in the
//             workspace (pandora_workspace_status).
pandora_tuning tuning_snapshot();

// Hooks of the host-buffer entry point: the stream waits for uv_ready (the
// endpoints' host-to-device copy) only before the first sort pass, which is
// the first step that reads them; vp_done is recorded once level 0 has
// written vertex_parent, so its device-to-host copy overlaps the rest.
constexpr int UV_CHUNKS = 8;
constexpr int EP_PARTS = 8;
struct Overlap {
    cudaEvent_t uv_ready = nullptr;
    // endpoints arriving in chunks of uv_chunk_tiles sort tiles: the first
    // sort pass runs chunk by chunk, chunk k after uv_chunk[k]
    int n_uv_chunks = 0;
    i64 uv_chunk_tiles = 0;
    const cudaEvent_t *uv_chunk = nullptr;
    // edge_parent back to ep_host on vp_stream in EP_PARTS ranges of whole
    // link buckets, each after its part of the link's apply pass (only where
    // the link is bucketed; *ep_copied then tells the caller)
    i32 *ep_host = nullptr;
    cudaEvent_t *ep_done = nullptr;
    bool *ep_copied = nullptr;
    cudaEvent_t vp_done = nullptr;
    cudaStream_t vp_stream = nullptr;   // copies vertex_parent to vp_host after vp_done
    i32 *vp_host = nullptr;
};

// Enqueues the copy of vertex_parent (N entries) to the host once it is final.
int overlap_vp_copy(const Overlap *ov, const i32 *vp, i64 N, cudaStream_t s)
{
    if (!ov || !ov->vp_done)
        return PANDORA_OK;
    PANDORA_CUDA(cudaEventRecord(ov->vp_done, s));
    if (ov->vp_stream && ov->vp_host) {
        PANDORA_CUDA(cudaStreamWaitEvent(ov->vp_stream, ov->vp_done, 0));
        PANDORA_CUDA(cudaMemcpyAsync(ov->vp_host, vp, (size_t)N * 4, cudaMemcpyDeviceToHost,
                                     ov->vp_stream));
    }
    return PANDORA_OK;
}

int run_core(const i32 *u, const i32 *v, const float *w, i64 M, i64 T, const i64 *d_off,
             i32 *ep, i32 *vp, void *ws, size_t ws_bytes, pandora_stats *stats, cudaStream_t s,
             bool blocking, const Overlap *ov = nullptr)
{
    const i64 N = M + T;
    if (stats)
        std::memset(stats, 0, sizeof(*stats));
    const Layout L = make_layout(M, T);
    if (!ws || ws_bytes < L.total)
        return PANDORA_ERR_WORKSPACE_TOO_SMALL;
    char *base = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    Ctrl *ctrl = (Ctrl *)(base + L.ctrl);
    u32 *keysA = (u32 *)(base + L.keysA), *keysB = (u32 *)(base + L.keysB);
    u32 *valsA = (u32 *)(base + L.valsA), *valsB = (u32 *)(base + L.valsB);
    u32 *perm = (u32 *)(base + L.perm);
    int2 *ab0 = (int2 *)(base + L.ab0);
    u64 *lb = (u64 *)(base + L.lb);
    u64 *min_word = (u64 *)(base + L.min_word);
    i32 *ptr = (i32 *)(base + L.ptr);
    i32 *deep = (i32 *)(base + L.deep), *uf = (i32 *)(base + L.uf);
    i32 *root_of = (i32 *)(base + L.root_of);
    int2 *kept_rec = (int2 *)(base + L.kept_rec);
    int2 *abX = (int2 *)(base + L.abX), *abY = (int2 *)(base + L.abY);
    u32 *erX = (u32 *)(base + L.erX), *erY = (u32 *)(base + L.erY);
    unsigned char *lev = (unsigned char *)(base + L.lev);
    i32 *start = (i32 *)(base + L.start);
    int *status = &ctrl->status;

    CallTimer timer(s, blocking);
    const u32 report = wait_report_limit();
    HostCounters h{};
    h.lvl_m[0] = (u64)M;
    h.lvl_n[0] = (u64)N;
    // control block: zero, then level 0's sizes
    PANDORA_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
    // set by a kernel, not copied from host memory, so that a captured graph
    // does not depend on host memory that is gone at replay
    timer.launch(K_FILL, 1, [&] { launch_set_u64_pair(&ctrl->lvl_m[0], (u64)M, &ctrl->lvl_n[0], (u64)N, s); });
    if (d_off)
        timer.launch(K_CHECK_OFFSETS, T + 1, [&] { launch_check_offsets(d_off, T, M, status, s); });
    if (M == 0) {
        timer.launch(K_FILL, N, [&] { launch_fill(vp, N, -1, s); });
        if (int e = overlap_vp_copy(ov, vp, N, s))
            return e;
        PANDORA_CUDA(cudaGetLastError());
        if (!blocking)
            return PANDORA_OK;
        if (int e = read_counters(ctrl, &h, s))
            return e;
        return h.status;
    }

    // ---- 1. sort by (weight, index) -------------------------------------------
    timer.launch(K_HIST_WEIGHTS, M, 2, [&] {
        launch_hist_weights(w, M, &ctrl->hist1[0][0], status, s);
        launch_hist_scan(&ctrl->hist1[0][0], &ctrl->base1[0][0], 4, s);
    });
    std::vector<int> passes = {0, 1, 2, 3};
    if (blocking) {
        static thread_local u32 hhist[4][RADIX];
        PANDORA_CUDA(cudaMemcpyAsync(hhist, ctrl->hist1, sizeof(hhist), cudaMemcpyDeviceToHost, s));
        if (int e = read_counters(ctrl, &h, s))
            return e;
        if (h.status)
            return h.status;
        passes = useful_passes(hhist, 4, M);
        if (passes.empty())
            passes.push_back(3);   // still one pass: it writes the permutation and endpoints
    }
    // the endpoint stream (an int2 per edge) ping-pongs through arrays that
    // are idle until the level loop: kept_rec (>= M int2) and min_word (N
    // words of 8 bytes), both 256-byte aligned as the sort's bulk copies need
    // the histogram pass read only the weights; the endpoints must be here now
    // (or, arriving in chunks, before each chunk of the first pass)
    const bool chunked = ov && ov->n_uv_chunks > 0;
    if (ov && ov->uv_ready && !chunked)
        PANDORA_CUDA(cudaStreamWaitEvent(s, ov->uv_ready, 0));
    int2 *uvA = (int2 *)kept_rec, *uvB = (int2 *)min_word;
    const u32 *cur_k = nullptr, *cur_v = nullptr;
    const int2 *cur_uv = nullptr;
    bool toA = false;
    for (size_t k = 0; k < passes.size(); ++k) {
        const bool first = k == 0, last = k + 1 == passes.size();
        OnesweepParams P{};
        P.report_limit = report;
        P.n = M;
        P.shift = 8 * passes[k];
        P.hist = ctrl->hist1[passes[k]];
        P.bin_base = ctrl->base1[passes[k]];
        P.lb = lb;
        P.tile_counter = &ctrl->tile_counter[0];
        P.status = status;
        P.u = u;
        P.v = v;
        P.n_vertices = N;
        P.edge_off = d_off;
        P.n_trees = T;
        int flags = OS_PAYLOAD_UV;
        if (first) {
            flags |= OS_KEY_FROM_W | OS_GEN_VALS | (d_off ? OS_FOREST : 0);
            P.w_in = w;
        } else {
            P.keys_in = cur_k;
            P.vals_in = cur_v;
            P.uv_in = cur_uv;
        }
        if (last) {
            flags |= OS_LAST_AB;
            P.vals_out = perm;
            P.uv_out = ab0;
        } else {
            flags |= OS_WRITE_KEYS;
            P.keys_out = toA ? keysA : keysB;
            P.vals_out = toA ? valsA : valsB;
            P.uv_out = toA ? uvA : uvB;
        }
        PANDORA_CUDA(cudaMemsetAsync(lb, 0, (size_t)onesweep_tiles(M) * RADIX * 8, s));
        PANDORA_CUDA(cudaMemsetAsync(&ctrl->tile_counter[0], 0, 4, s));
        if (first && chunked) {
            // consecutive tile ranges, each launched once its endpoints landed
            const i64 tiles = onesweep_tiles(M);
            cudaError_t ce = cudaSuccess;
            timer.launch(K_SORT_WEIGHTS, M, ov->n_uv_chunks, [&] {
                for (int c = 0; c < ov->n_uv_chunks; ++c) {
                    const i64 t0 = (i64)c * ov->uv_chunk_tiles;
                    const i64 t1 = std::min(tiles, t0 + ov->uv_chunk_tiles);
                    if (t1 <= t0)
                        continue;
                    if (ce == cudaSuccess)
                        ce = cudaStreamWaitEvent(s, ov->uv_chunk[c], 0);
                    OnesweepParams Pc = P;
                    Pc.grid_tiles = t1 - t0;
                    launch_onesweep(flags, Pc, s);
                }
            });
            PANDORA_CUDA(ce);
        } else {
            timer.launch(K_SORT_WEIGHTS, M, [&] { launch_onesweep(flags, P, s); });
        }
        cur_k = P.keys_out;
        cur_v = P.vals_out;
        cur_uv = P.uv_out;
        toA = !toA;
    }
    PANDORA_CUDA(cudaGetLastError());

    // ---- 2. contraction levels ------------------------------------------------
    const int L_bound = level_bound(M);
    const int2 *ab = ab0;
    const u32 *er = nullptr;
    i64 m_grid = M, n_grid = N, m_cap = M, n_cap = N, kept_used = 0;
    LevelTable table{};
    int n_levels = 0;
    bool useX = true;
    // the last levels of a single tree run in one block once a level has at
    // most TAIL_CAP edges (exactly known when blocking, a bound otherwise)
    const bool tail_ok = T == 1 && !stats && tuning_snapshot().small_max_edges > 0;
    bool tail_done = false;
    for (int l = 0; l < L_bound; ++l) {
        if (tail_ok && l >= 1 && m_cap <= TAIL_CAP) {
            TailParams Q{};
            Q.level = l;
            Q.d_m = ctrl->lvl_m;
            Q.lvl_m = ctrl->lvl_m;
            Q.lvl_n = ctrl->lvl_n;
            Q.d_n_levels = &ctrl->n_levels;
            Q.ab = ab;
            Q.er = er;
            Q.ab_cap = L.half_cap;
            Q.lev = lev;
            Q.start = start;
            Q.max_levels = L_bound;
            Q.status = status;
            int k = 0;
            for (; k < TAIL_MAX_LEVELS && l + k < L_bound; ++k) {
                const i64 cap = (m_cap >> k) + T;
                if (kept_used + cap > L.kept_cap)
                    break;
                Q.rec[k] = kept_rec + kept_used;
                Q.rec_cap[k] = cap;
                table.rec[l + k] = Q.rec[k];
                table.n_cap[l + k] = cap;
                kept_used += cap;
            }
            timer.launch(K_TAIL, m_cap, [&] { launch_tail(Q, s); });
            PANDORA_CUDA(cudaGetLastError());
            n_levels = l + k;
            tail_done = true;
            if (blocking) {
                if (int e = read_counters(ctrl, &h, s))
                    return e;
                if (h.status)
                    return h.status;
            }
            break;
        }
        LevelParams P{};
        P.report_limit = report;
        P.level = l;
        P.d_m = &ctrl->lvl_m[l];
        P.d_n = &ctrl->lvl_n[l];
        P.d_m_next = &ctrl->lvl_m[l + 1];
        P.d_n_next = &ctrl->lvl_n[l + 1];
        P.m_cap = m_cap;
        P.n_cap = n_cap;
        P.m_grid = m_grid;
        P.n_grid = n_grid;
        P.d_n_levels = &ctrl->n_levels;
        P.ab = ab;
        P.er = er;
        P.min_word = min_word;
        P.ptr = ptr;
        P.deep = deep;
        P.uf = uf;
        P.root_of = root_of;
        P.d_n_deep = &ctrl->n_deep;
        if (l == 0) {
            P.perm = perm;
            P.vertex_parent = vp;
            if (T > 1) {
                P.tree_roots = (u32 *)(base + L.troots);
                P.tree_root_id = (i32 *)(base + L.troots) + T;
                PANDORA_CUDA(cudaMemsetAsync(P.tree_roots, 0, (size_t)T * 4, s));
            }
        } else {
            if (kept_used + n_cap > L.kept_cap)
                return PANDORA_ERR_NOT_A_TREE;   // only reachable in blocking mode
            P.rec = kept_rec + kept_used;
            kept_used += n_cap;
            table.rec[l] = P.rec;
            table.n_cap[l] = n_cap;
        }
        P.edge_off = d_off;
        P.n_trees = T;
        P.ab_next = useX ? abX : abY;
        P.er_next = useX ? erX : erY;
        P.cap_next = L.half_cap;
        P.lev = lev;
        P.start = start;
        P.lb = lb;
        P.tile_counter = ctrl->tile_counter;
        P.status = status;
        // bucketed marking when the level's words (8 B per vertex) are well
        // above L2; its records live in arrays idle during the level loop:
        // the sort buffers (keysA .. valsB, 16 M bytes) and, on level 0, the
        // kept records (filled from level 1 on)
        if (n_grid > (l == 0 ? MARK_DIRECT_MAX0_VERTICES : MARK_DIRECT_MAX_VERTICES)) {
            // buckets of 2^MARK_BUCKET_SHIFT vertices, wider when the level
            // would need more than MARK_MAX_BUCKETS of them
            int shift = MARK_BUCKET_SHIFT;
            while (((n_grid - 1) >> shift) >= MARK_MAX_BUCKETS)
                ++shift;
            P.mark_shift = shift;
            P.mark_buckets = (int)((n_grid + (i64(1) << shift) - 1) >> shift);
            char *sort_region = base + L.keysA;   // keysA, keysB, valsA, valsB in a row
            const size_t sort_bytes = L.perm - L.keysA;
            P.rec_w = (u64 *)sort_region;
            if (l == 0) {
                P.rec_x = (u32 *)kept_rec;
                if ((size_t)(2 * m_cap) * 8 > sort_bytes ||
                    (size_t)(2 * m_cap) * 4 > (size_t)L.kept_cap * 8)
                    P.mark_buckets = 0;
            } else {
                P.rec_x = (u32 *)(sort_region + align_up((size_t)(2 * m_cap) * 8));
                if (align_up((size_t)(2 * m_cap) * 8) + (size_t)(2 * m_cap) * 4 > sort_bytes)
                    P.mark_buckets = 0;
            }
            P.mark_count = ctrl->mark_count;
            P.mark_cursor = ctrl->mark_cursor;
            P.mark_base = ctrl->mark_base;
            if (P.mark_buckets > 0)
                PANDORA_CUDA(cudaMemsetAsync(ctrl->mark_count, 0,
                                             sizeof(ctrl->mark_count) + sizeof(ctrl->mark_cursor),
                                             s));
            // level 0: the records also carry caller ids (in the next-level
            // edge arrays abX .. erY, written only by compact) and a flag pass
            // classifies every edge for Eq. 2 and writes vertex_parent
            const size_t next_region = L.erY + (size_t)L.half_cap * 4 - L.abX;
            if (l == 0 && P.mark_buckets > 0 && (size_t)(2 * m_cap) * 4 <= next_region) {
                P.rec_c = (u32 *)(base + L.abX);
                P.eflag = (u32 *)(base + L.eflag);
                PANDORA_CUDA(cudaMemsetAsync(P.eflag, 0, (size_t)eflag_words(M) * 4, s));
            }
        }
        PANDORA_CUDA(cudaMemsetAsync(
            lb, 0, (size_t)(level_tiles(n_grid) + 1 + level_tiles(m_grid) + 1) * 8, s));
        PANDORA_CUDA(cudaMemsetAsync(ctrl->tile_counter, 0, 16, s));
        timer.launch(K_INIT_LEVEL, n_grid, [&] { launch_init_level(P, s); });
        timer.launch(K_MARK, m_grid, P.mark_buckets > 0 ? (P.eflag ? 5 : 4) : 1,
                     [&] { launch_mark(P, s); });
        timer.launch(K_PTR_INIT, n_grid, [&] { launch_ptr_init(P, s); });
        if (l == 0)   // vertex_parent is final after level 0's ptr_init
            if (int e = overlap_vp_copy(ov, vp, N, s))
                return e;
        timer.launch(K_COMPRESS, n_grid, 4, [&] { launch_compress(P, s); });
        timer.launch(K_COMPACT, m_grid, [&] { launch_compact(P, s); });
        PANDORA_CUDA(cudaGetLastError());
        n_levels = l + 1;
        ab = P.ab_next;
        er = P.er_next;
        useX = !useX;
        if (blocking) {
            if (int e = read_counters(ctrl, &h, s))
                return e;
            if (stats) {
                stats->level_edges[l] = (i64)h.lvl_m[l];
                stats->level_vertices[l] = (i64)h.lvl_n[l];
                stats->n_levels = l + 1;
            }
            if (h.status)
                return h.status;
            if (h.n_levels)
                break;
            if ((i64)h.lvl_m[l + 1] > L.half_cap)
                return PANDORA_ERR_NOT_A_TREE;
            m_grid = m_cap = (i64)h.lvl_m[l + 1];
            n_grid = n_cap = (i64)h.lvl_n[l + 1];
        } else {
            // worst case for the next level (a forest loses at least half its edges)
            m_cap = m_grid = std::min<i64>(m_cap / 2, L.half_cap);
            n_cap = n_grid = m_cap + T;
        }
    }
    if (blocking && h.n_levels == 0)
        return PANDORA_ERR_NOT_A_TREE;   // the level bound of Section 4.2 was exceeded
    (void)tail_done;

    // ---- 3. expansion: chain key of every edge -----------------------------
    const u32 root_base = (u32)(2 * M);
    ExpandParams E{};
    E.m = M;
    E.max_levels = n_levels;
    E.d_n_levels = &ctrl->n_levels;
    E.lvl_n = ctrl->lvl_n;
    E.lev = lev;
    E.start = start;
    E.perm = perm;
    E.keys_out = keysA;
    E.root_base = root_base;
    E.edge_off = d_off;
    E.n_trees = T;
    E.hist = ctrl->hist2;
    E.plan = chain_digit_plan(M, T);
    E.status = status;
    const DigitPlan &plan = E.plan;
    timer.launch(K_EXPAND, M, 2, [&] {
        launch_expand(E, table, s);
        launch_hist_scan_plan(ctrl->hist2, ctrl->base2, plan, s);
    });
    PANDORA_CUDA(cudaGetLastError());
    std::vector<int> passes2;
    for (int q = 0; q < plan.n; ++q)
        passes2.push_back(q);
    if (blocking) {
        static thread_local u32 hhist2[DIGIT_PLAN_HIST];
        PANDORA_CUDA(cudaMemcpyAsync(hhist2, ctrl->hist2, sizeof(hhist2), cudaMemcpyDeviceToHost, s));
        if (int e = read_counters(ctrl, &h, s))
            return e;
        if (h.status)
            return h.status;
        // a pass whose digit is the same for every key is the identity
        passes2.clear();
        for (int q = 0; q < plan.n; ++q) {
            bool trivial = false;
            for (int d = 0; d < (1 << plan.width[q]); ++d)
                if ((i64)hhist2[plan.off[q] + d] == M)
                    trivial = true;
            if (!trivial)
                passes2.push_back(q);
        }
    }

    // ---- 4. stable sort by chain key, then link -------------------------------
    const u32 *sk = keysA, *sv = perm;
    for (size_t k = 0; k < passes2.size(); ++k) {
        OnesweepParams P{};
        P.report_limit = report;
        P.n = M;
        const int q = passes2[k];
        P.shift = plan.shift[q];
        P.dbits = plan.width[q];
        P.hist = ctrl->hist2 + plan.off[q];
        P.bin_base = ctrl->base2 + plan.off[q];
        P.lb = lb;
        P.tile_counter = &ctrl->tile_counter[0];
        P.status = status;
        P.keys_in = sk;
        P.vals_in = sv;
        const bool outB = (sk == keysA);
        P.keys_out = outB ? keysB : keysA;
        P.vals_out = outB ? valsB : valsA;
        PANDORA_CUDA(cudaMemsetAsync(lb, 0, (size_t)onesweep_tiles(M) * (1 << P.dbits) * 8, s));
        PANDORA_CUDA(cudaMemsetAsync(&ctrl->tile_counter[0], 0, 4, s));
        timer.launch(K_SORT_CHAINS, M, [&] { launch_onesweep(OS_WRITE_KEYS, P, s); });
        sk = P.keys_out;
        sv = P.vals_out;
    }
    LinkParams K{};
    K.m = M;
    K.skeys = sk;
    K.svals = sv;
    K.perm = perm;
    K.root_base = root_base;
    K.edge_parent = ep;
    K.edge_off = d_off;
    K.n_trees = T;
    // bucketed link when edge_parent is well above L2; the pairs go to the
    // level-0 endpoint array (8 bytes per edge), idle after the level loop
    if (M > LINK_BUCKET_MIN_EDGES) {
        K.bucket_shift = LINK_BUCKET_SHIFT;
        K.n_buckets = (int)((M + (i64(1) << LINK_BUCKET_SHIFT) - 1) >> LINK_BUCKET_SHIFT);
        K.rec = ab0;
        K.cursor = ctrl->link_cursor;
        if (K.n_buckets > MARK_MAX_BUCKETS)
            K.n_buckets = 0;
        else
            PANDORA_CUDA(cudaMemsetAsync(ctrl->link_cursor, 0, sizeof(ctrl->link_cursor), s));
    }
    const bool ep_parts = ov && ov->ep_host && ov->ep_done && ov->vp_stream && K.n_buckets > 0;
    if (ep_parts) {
        K.apply_parts = EP_PARTS;
        K.apply_done = ov->ep_done;
    }
    timer.launch(K_LINK, M, K.n_buckets > 0 ? 1 + (ep_parts ? EP_PARTS : 1) : 1,
                 [&] { launch_link(K, s); });
    PANDORA_CUDA(cudaGetLastError());
    if (ep_parts) {
        // the same bucket ranges as the apply launches
        const i64 per = (((i64)K.n_buckets + EP_PARTS - 1) / EP_PARTS) << K.bucket_shift;
        for (int k = 0; k < EP_PARTS; ++k) {
            const i64 b = std::min(M, (i64)k * per), e = std::min(M, (i64)(k + 1) * per);
            PANDORA_CUDA(cudaStreamWaitEvent(ov->vp_stream, ov->ep_done[k], 0));
            if (e > b)
                PANDORA_CUDA(cudaMemcpyAsync(ov->ep_host + b, ep + b, (size_t)(e - b) * 4,
                                             cudaMemcpyDeviceToHost, ov->vp_stream));
        }
        if (ov->ep_copied)
            *ov->ep_copied = true;
    }
    if (!blocking)
        return PANDORA_OK;
    if (int e = read_counters(ctrl, &h, s))
        return e;
    return h.status;
}

// ---- small trees: the single-CTA solver and the batched dispatch ------------
struct Tuning {
    std::mutex mu;
    pandora_tuning t{};
    Tuning()
    {
        t.small_max_edges = PANDORA_SMALL_CAP;
        for (int k = 0; k < 13; ++k)
            t.small_threads[k] = 512;
        t.split_min_permille = 50;
    }
};
Tuning &tuning()
{
    static Tuning t;
    return t;
}
std::atomic<u32> g_report_limit{SPIN_LIMIT};

pandora_tuning tuning_snapshot()
{
    Tuning &t = tuning();
    std::lock_guard<std::mutex> lock(t.mu);
    return t.t;
}
// Extra workspace of a split batched call.  The plan part (tree lists,
// packed offsets, the plan's status word) is needed by every split; the
// packed forest (inputs and outputs of the large trees) only when the batch
// has large trees, which takes two or more trees.
struct DispatchLayout {
    size_t lists, coff, dstat, plan_total;
    size_t cu, cv, cw, cep, cvp, total;
};
DispatchLayout dispatch_layout(i64 M, i64 T)
{
    DispatchLayout D{};
    size_t off = 0;
    auto take = [&](i64 bytes) {
        const size_t o = off;
        off = align_up(off + (size_t)std::max<i64>(bytes, 0));
        return o;
    };
    D.lists = take(T * 4);
    D.coff = take((T + 1) * 8);
    D.dstat = take(4);
    D.plan_total = off;
    D.cu = take(M * 4);
    D.cv = take(M * 4);
    D.cw = take(M * 4);
    D.cep = take(M * 4);
    D.cvp = take((M + T) * 4);
    D.total = off;
    return D;
}
// Workspace of a call with M edges in T trees (what pandora_workspace_size
// reports): the pipeline's layout, then the dispatch part a batched call may
// need (a single-tree batch can only split into the single-block solver).
size_t total_workspace(i64 M, i64 T)
{
    const DispatchLayout D = dispatch_layout(M, T);
    return make_layout(M, T).total + (T > 1 ? D.total : D.plan_total) + 256;
}

bool offsets_partition(const i64 *h_off, i64 T, i64 M)
{
    if (h_off[0] != 0 || h_off[T] != M)
        return false;
    for (i64 t = 0; t < T; ++t)
        if (h_off[t + 1] < h_off[t])
            return false;
    return true;
}

// A batched call whose offsets the host also holds (h_off, a partition of
// [0, M)).  Every tree at or under the cutoff goes to the single-block
// solver, one block per tree and one launch per size bucket; the others are
// packed into one forest for the pipeline and copied back.  The packing costs
// about 40 sequential bytes per large-tree edge, so a batch is only split when
// its small trees hold at least split_min_permille of the edges (or there are
// no large trees).  Every launch has a host-known grid: with blocking == false
// nothing waits on the device and the call can be captured in a graph.
int run_planned(const i32 *u, const i32 *v, const float *w, i64 M, i64 T, const i64 *d_off,
                const i64 *h_off, i32 *ep, i32 *vp, void *ws, size_t ws_bytes, cudaStream_t s,
                bool blocking, const pandora_tuning &tn)
{
    const i64 cutoff = std::min<i64>(tn.small_max_edges, small_tree_capacity());
    if (!ws || ws_bytes < make_layout(M, T).total)
        return PANDORA_ERR_WORKSPACE_TOO_SMALL;
    PlanParams plan{};
    i64 m_small = 0;
    for (i64 t = 0; t < T; ++t) {
        const i64 m = h_off[t + 1] - h_off[t];
        const int c = size_class(m, cutoff);
        ++plan.count[c];
        if (c == CLASS_LARGE)
            plan.m_large += m;
        else
            m_small += m;
    }
    const i64 T_L = plan.count[CLASS_LARGE], M_L = plan.m_large;
    const Layout L = make_layout(M, T);
    const DispatchLayout D = dispatch_layout(M, T);
    const size_t need = L.total + (T_L > 0 ? D.total : D.plan_total) + 256;
    const bool split = cutoff > 0 && T_L < T && ws_bytes >= need &&
                       (T_L == 0 || m_small * 1000 >= (i64)tn.split_min_permille * M);
    if (!split)
        return run_core(u, v, w, M, T, d_off, ep, vp, ws, ws_bytes, nullptr, s, blocking);

    char *base = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    Ctrl *ctrl = (Ctrl *)base;   // the control block heads every layout
    char *dbase = base + L.total;
    i32 *cu = (i32 *)(dbase + D.cu), *cv = (i32 *)(dbase + D.cv);
    float *cw = (float *)(dbase + D.cw);
    i32 *cep = (i32 *)(dbase + D.cep), *cvp = (i32 *)(dbase + D.cvp);
    i64 *coff = (i64 *)(dbase + D.coff);
    i32 *lists = (i32 *)(dbase + D.lists);
    int *dstat = (int *)(dbase + D.dstat);
    // lists: large trees first, then bucket 0, 1, ...
    plan.base[CLASS_LARGE] = 0;
    i64 acc = T_L;
    for (int k = 0; k < CLASS_LARGE; ++k) {
        plan.base[k] = acc;
        acc += plan.count[k];
    }
    plan.off = d_off;
    plan.n_trees = T;
    plan.total_edges = M;
    plan.cutoff = cutoff;
    plan.lists = lists;
    plan.coff = coff;
    plan.status = dstat;
    int st_core = PANDORA_OK;
    {
        CallTimer timer(s, blocking);
        PANDORA_CUDA(cudaMemsetAsync(lists, 0xFF, (size_t)T * 4, s));
        PANDORA_CUDA(cudaMemsetAsync(coff, 0, (size_t)(T + 1) * 8, s));
        PANDORA_CUDA(cudaMemsetAsync(dstat, 0, 4, s));
        timer.launch(K_GATHER, T, [&] { launch_plan(plan, s); });
        if (T_L > 0) {
            timer.launch(K_GATHER, M_L, [&] {
                launch_gather_trees(u, v, w, d_off, T, M, lists, coff, T_L, M_L, cu, cv, cw, s);
            });
            PANDORA_CUDA(cudaGetLastError());
        }
    }
    if (T_L > 0) {
        // the pipeline resets the control block, so it runs before the small trees
        st_core = run_core(cu, cv, cw, M_L, T_L, coff, cep, cvp, ws, L.total, nullptr, s, blocking);
        if (st_core == PANDORA_ERR_CUDA)
            return st_core;
    } else {
        PANDORA_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
    }
    {
        CallTimer timer(s, blocking);
        if (T_L > 0)
            timer.launch(K_GATHER, M_L, [&] {
                launch_scatter_trees(cep, cvp, d_off, T, M, lists, coff, T_L, M_L, ep, vp, s);
            });
        for (int k = 0; k < CLASS_LARGE; ++k) {
            if (plan.count[k] == 0)
                continue;
            SmallParams P{};
            P.u = u;
            P.v = v;
            P.w = w;
            P.edge_off = d_off;
            P.n_trees = T;
            P.tree_list = lists + plan.base[k];
            P.cutoff = cutoff;
            P.total_edges = M;
            P.edge_parent = ep;
            P.vertex_parent = vp;
            P.status = &ctrl->status;
            timer.launch(K_SMALL, plan.count[k], [&] {
                launch_small(P, tn.small_threads[k], std::min<i64>(cutoff, (i64(2) << k) - 1),
                             (unsigned)plan.count[k], s);
            });
        }
        timer.launch(K_GATHER, 1, [&] { launch_merge_status(dstat, &ctrl->status, s); });
    }
    PANDORA_CUDA(cudaGetLastError());
    if (!blocking)
        return PANDORA_OK;
    int st = 0;
    PANDORA_CUDA(cudaMemcpyAsync(&st, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PANDORA_CUDA(cudaStreamSynchronize(s));
    return st_core ? st_core : st;
}

int run(const i32 *u, const i32 *v, const float *w, i64 M, i64 T, const i64 *d_off, i32 *ep,
        i32 *vp, void *ws, size_t ws_bytes, pandora_stats *stats, cudaStream_t s,
        bool blocking = true)
{
    const pandora_tuning tn = tuning_snapshot();
    const i64 cutoff = std::min<i64>(tn.small_max_edges, small_tree_capacity());
    if (!ws || ws_bytes < total_workspace(M, T))
        return PANDORA_ERR_WORKSPACE_TOO_SMALL;
    char *base = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    Ctrl *ctrl = (Ctrl *)base;   // the control block heads every layout
    if (!d_off && !stats && M >= 1 && M <= cutoff) {
        // one small tree: one block, whole method in shared memory
        SmallParams P{};
        P.u = u;
        P.v = v;
        P.w = w;
        P.m = M;
        P.cutoff = cutoff;
        P.total_edges = M;
        P.edge_parent = ep;
        P.vertex_parent = vp;
        P.status = &ctrl->status;
        CallTimer timer(s, blocking);
        PANDORA_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
        timer.launch(K_SMALL, M, [&] {
            launch_small(P, tn.small_threads[size_class(M, cutoff)], M, 1, s);
        });
        PANDORA_CUDA(cudaGetLastError());
        if (!blocking)
            return PANDORA_OK;
        int st = 0;
        PANDORA_CUDA(cudaMemcpyAsync(&st, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        PANDORA_CUDA(cudaStreamSynchronize(s));
        return st;
    }
    if (!d_off || !blocking || stats || cutoff <= 0 || M == 0)
        return run_core(u, v, w, M, T, d_off, ep, vp, ws, ws_bytes, stats, s, blocking);
    // batched and blocking: read the offsets, then split the batch like a
    // caller that holds them on the host
    std::vector<i64> h_off(T + 1);
    PANDORA_CUDA(cudaMemcpyAsync(h_off.data(), d_off, (T + 1) * sizeof(i64), cudaMemcpyDeviceToHost, s));
    PANDORA_CUDA(cudaStreamSynchronize(s));
    if (!offsets_partition(h_off.data(), T, M))   // the pipeline's own check reports it
        return run_core(u, v, w, M, T, d_off, ep, vp, ws, ws_bytes, stats, s, blocking);
    return run_planned(u, v, w, M, T, d_off, h_off.data(), ep, vp, ws, ws_bytes, s, true, tn);
}

int check_common(const i32 *u, const i32 *v, const float *w, i64 M, i64 T, i32 *ep, i32 *vp)
{
    if (M < 0 || T < 0)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (M + T > (i64)INT32_MAX)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (M > 0 && (!u || !v || !w || !ep))
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (M + T > 0 && !vp)
        return PANDORA_ERR_INVALID_ARGUMENT;
    return PANDORA_OK;
}

cudaMemPool_t library_pool(int dev)
{
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(dev);
    if (it != pools.end())
        return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess)
        return nullptr;
    u64 threshold = ~0ull;   // keep freed blocks for the next call
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    pools[dev] = pool;
    return pool;
}

int run_pooled(const i32 *u, const i32 *v, const float *w, i64 M, i64 T, const i64 *d_off,
               i32 *ep, i32 *vp, cudaStream_t s)
{
    int dev = 0;
    PANDORA_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = library_pool(dev);
    if (!pool)
        return PANDORA_ERR_CUDA;
    const size_t bytes = total_workspace(M, T);
    void *ws = nullptr;
    if (cudaMallocFromPoolAsync(&ws, bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return PANDORA_ERR_OUT_OF_MEMORY;
    }
    const int st = run(u, v, w, M, T, d_off, ep, vp, ws, bytes, nullptr, s);
    cudaFreeAsync(ws, s);
    if (st != PANDORA_OK)
        cudaStreamSynchronize(s);
    return st;
}

// Streams and events of the host-buffer entry point, one set per device and
// host thread (created once, kept for the process).
struct HostIoRes {
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_alloc = nullptr, ev_uv = nullptr, ev_vp = nullptr, ev_out = nullptr;
    cudaEvent_t ev_w = nullptr;
    cudaEvent_t ev_chunk[UV_CHUNKS] = {};
    cudaEvent_t ev_ep[EP_PARTS] = {};
};
HostIoRes *host_io_res(int dev)
{
    static thread_local std::map<int, HostIoRes> res;
    auto it = res.find(dev);
    if (it != res.end())
        return &it->second;
    HostIoRes r;
    if (cudaStreamCreateWithFlags(&r.s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&r.s_out, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&r.ev_alloc, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r.ev_uv, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r.ev_vp, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r.ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r.ev_w, cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    for (int c = 0; c < UV_CHUNKS; ++c)
        if (cudaEventCreateWithFlags(&r.ev_chunk[c], cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
    for (int c = 0; c < EP_PARTS; ++c)
        if (cudaEventCreateWithFlags(&r.ev_ep[c], cudaEventDisableTiming) != cudaSuccess)
            return nullptr;
    return &(res[dev] = r);
}

// One tree from host buffers to host buffers.  Device memory (inputs,
// outputs, workspace) comes from the library pool on `s`.  The weights go
// first on `s` (the histogram pass needs only them), then the endpoints on a
// second stream in eight chunks of whole sort tiles, the first sort pass
// running over each chunk once it has landed;
// vertex_parent goes back on a third stream as soon as level 0 has written
// it, overlapping the other levels, the expansion and the linking;
// edge_parent follows on that stream range by range as the bucketed link
// finishes each range of caller ids (after the last kernel when the link is
// not bucketed).  Blocking.
int run_host(const i32 *hu, const i32 *hv, const float *hw, i64 M, i32 *hep, i32 *hvp,
             cudaStream_t s)
{
    int dev = 0;
    PANDORA_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool = library_pool(dev);
    HostIoRes *r = host_io_res(dev);
    if (!pool || !r)
        return PANDORA_ERR_CUDA;
    const i64 N = M + 1;
    const size_t io_bytes = align_up((size_t)M * 4) * 4 + align_up((size_t)N * 4);
    const size_t ws_bytes = total_workspace(M, 1);
    char *io = nullptr;
    void *ws = nullptr;
    if (cudaMallocFromPoolAsync((void **)&io, io_bytes, pool, s) != cudaSuccess ||
        cudaMallocFromPoolAsync(&ws, ws_bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        if (io)
            cudaFreeAsync(io, s);
        return PANDORA_ERR_OUT_OF_MEMORY;
    }
    const size_t a = align_up((size_t)M * 4);
    i32 *du = (i32 *)io, *dv = (i32 *)(io + a);
    float *dw = (float *)(io + 2 * a);
    i32 *dep = (i32 *)(io + 3 * a), *dvp = (i32 *)(io + 4 * a);
    int st = PANDORA_OK;
    do {
        if (cudaEventRecord(r->ev_alloc, s) != cudaSuccess ||
            cudaStreamWaitEvent(r->s_in, r->ev_alloc, 0) != cudaSuccess ||
            cudaStreamWaitEvent(r->s_out, r->ev_alloc, 0) != cudaSuccess) {
            st = PANDORA_ERR_CUDA;
            break;
        }
        // the weights first (the histogram pass needs only them), then the
        // endpoints in chunks of whole sort tiles, each chunk's event letting
        // the first sort pass run over it while the next ones arrive
        const i64 ct = (onesweep_tiles(M) + UV_CHUNKS - 1) / UV_CHUNKS;
        if (M > 0) {
            bool ok = cudaMemcpyAsync(dw, hw, (size_t)M * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
                      cudaEventRecord(r->ev_w, s) == cudaSuccess &&
                      cudaStreamWaitEvent(r->s_in, r->ev_w, 0) == cudaSuccess;
            for (int c = 0; ok && c < UV_CHUNKS; ++c) {
                const i64 e0 = std::min<i64>(M, (i64)c * ct * OS_TILE);
                const i64 e1 = std::min<i64>(M, (i64)(c + 1) * ct * OS_TILE);
                if (e1 > e0)
                    ok = cudaMemcpyAsync(du + e0, hu + e0, (size_t)(e1 - e0) * 4, cudaMemcpyHostToDevice,
                                         r->s_in) == cudaSuccess &&
                         cudaMemcpyAsync(dv + e0, hv + e0, (size_t)(e1 - e0) * 4, cudaMemcpyHostToDevice,
                                         r->s_in) == cudaSuccess;
                ok = ok && cudaEventRecord(r->ev_chunk[c], r->s_in) == cudaSuccess;
            }
            if (!ok) {
                st = PANDORA_ERR_CUDA;
                break;
            }
        }
        if (cudaEventRecord(r->ev_uv, r->s_in) != cudaSuccess) {
            st = PANDORA_ERR_CUDA;
            break;
        }
        const pandora_tuning tn = tuning_snapshot();
        const i64 cutoff = std::min<i64>(tn.small_max_edges, small_tree_capacity());
        if (M >= 1 && M <= cutoff) {
            // one small tree: the single-block solver, nothing to overlap
            if (cudaStreamWaitEvent(s, r->ev_uv, 0) != cudaSuccess) {
                st = PANDORA_ERR_CUDA;
                break;
            }
            st = run(du, dv, dw, M, 1, nullptr, dep, dvp, ws, ws_bytes, nullptr, s, true);
            if (st == PANDORA_OK &&
                (cudaMemcpyAsync(hvp, dvp, (size_t)N * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(hep, dep, (size_t)M * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess))
                st = PANDORA_ERR_CUDA;
            break;
        }
        Overlap ov;
        ov.uv_ready = r->ev_uv;
        ov.n_uv_chunks = UV_CHUNKS;
        ov.uv_chunk_tiles = ct;
        ov.uv_chunk = r->ev_chunk;
        bool ep_copied = false;
        ov.ep_host = hep;
        ov.ep_done = r->ev_ep;
        ov.ep_copied = &ep_copied;
        ov.vp_done = r->ev_vp;
        ov.vp_stream = r->s_out;
        ov.vp_host = hvp;
        st = run_core(du, dv, dw, M, 1, nullptr, dep, dvp, ws, ws_bytes, nullptr, s, true, &ov);
        if (st != PANDORA_OK)
            break;
        if (M > 0 && !ep_copied &&
            cudaMemcpyAsync(hep, dep, (size_t)M * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            st = PANDORA_ERR_CUDA;
            break;
        }
    } while (false);
    // s waits for the other streams' last work before the memory goes back
    cudaEventRecord(r->ev_out, r->s_out);
    cudaStreamWaitEvent(s, r->ev_out, 0);
    cudaEventRecord(r->ev_uv, r->s_in);
    cudaStreamWaitEvent(s, r->ev_uv, 0);
    cudaFreeAsync(ws, s);
    cudaFreeAsync(io, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == PANDORA_OK)
        st = PANDORA_ERR_CUDA;
    return st;
}

}  // namespace

// Entry for other translation units of the library (the allocation-free
// entry point): the same pipeline on a workspace the caller of this function
// provides.
int run_on_workspace(const i32 *u, const i32 *v, const float *w, i64 M, i32 *ep, i32 *vp,
                     void *ws, size_t ws_bytes, cudaStream_t s)
{
    return run(u, v, w, M, 1, nullptr, ep, vp, ws, ws_bytes, nullptr, s);
}

size_t workspace_bytes(i64 M, i64 T) { return total_workspace(M, T); }

// The library's stream-ordered pool of `dev`, for the flat-cluster entry point.
cudaMemPool_t flat_pool(int dev) { return library_pool(dev); }

}  // namespace pandora

using namespace pandora;

namespace pandora {
u32 wait_report_limit() { return g_report_limit.load(); }
}  // namespace pandora

extern "C" {

int pandora_workspace_size(int64_t total_edges, int64_t n_trees, size_t *bytes)
{
    if (!bytes || total_edges < 0 || n_trees < 1 || total_edges + n_trees > (i64)INT32_MAX)
        return PANDORA_ERR_INVALID_ARGUMENT;
    *bytes = total_workspace(total_edges, n_trees);
    return PANDORA_OK;
}

int pandora_dendrogram(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                       int32_t *edge_parent, int32_t *vertex_parent, void *stream)
{
    if (int e = check_common(u, v, w, n_edges, 1, edge_parent, vertex_parent))
        return e;
    return run_pooled(u, v, w, n_edges, 1, nullptr, edge_parent, vertex_parent,
                      (cudaStream_t)stream);
}

int pandora_dendrogram_host(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                            int32_t *edge_parent, int32_t *vertex_parent, void *stream)
{
    if (int e = check_common(u, v, w, n_edges, 1, edge_parent, vertex_parent))
        return e;
    return run_host(u, v, w, n_edges, edge_parent, vertex_parent, (cudaStream_t)stream);
}

int pandora_dendrogram_ws(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                          int32_t *edge_parent, int32_t *vertex_parent, void *workspace,
                          size_t workspace_bytes, pandora_stats *stats, void *stream)
{
    if (int e = check_common(u, v, w, n_edges, 1, edge_parent, vertex_parent))
        return e;
    return run(u, v, w, n_edges, 1, nullptr, edge_parent, vertex_parent, workspace,
               workspace_bytes, stats, (cudaStream_t)stream);
}

int pandora_dendrogram_batched(const int32_t *u, const int32_t *v, const float *w,
                               const int64_t *edge_offsets, int64_t n_trees, int64_t total_edges,
                               int32_t *edge_parent, int32_t *vertex_parent, void *stream)
{
    if (int e = check_common(u, v, w, total_edges, n_trees, edge_parent, vertex_parent))
        return e;
    if (n_trees == 0)
        return total_edges == 0 ? PANDORA_OK : PANDORA_ERR_INVALID_ARGUMENT;
    if (!edge_offsets)
        return PANDORA_ERR_INVALID_ARGUMENT;
    return run_pooled(u, v, w, total_edges, n_trees, edge_offsets, edge_parent, vertex_parent,
                      (cudaStream_t)stream);
}

int pandora_dendrogram_batched_ws(const int32_t *u, const int32_t *v, const float *w,
                                  const int64_t *edge_offsets, int64_t n_trees,
                                  int64_t total_edges, int32_t *edge_parent,
                                  int32_t *vertex_parent, void *workspace,
                                  size_t workspace_bytes, pandora_stats *stats, void *stream)
{
    if (int e = check_common(u, v, w, total_edges, n_trees, edge_parent, vertex_parent))
        return e;
    if (n_trees == 0)
        return total_edges == 0 ? PANDORA_OK : PANDORA_ERR_INVALID_ARGUMENT;
    if (!edge_offsets)
        return PANDORA_ERR_INVALID_ARGUMENT;
    return run(u, v, w, total_edges, n_trees, edge_offsets, edge_parent, vertex_parent,
               workspace, workspace_bytes, stats, (cudaStream_t)stream);
}

int pandora_profile_start(int with_timing)
{
    Profiler &p = profiler();
    std::lock_guard<std::mutex> lock(p.mu);
    p.timing = with_timing != 0;
    for (int k = 0; k < K_SLOTS; ++k) {
        p.launches[k] = 0;
        p.kernels[k] = 0;
        p.elements[k] = 0;
        p.ms[k] = 0.0;
    }
    return PANDORA_OK;
}

int pandora_profile_read(pandora_profile *out)
{
    if (!out)
        return PANDORA_ERR_INVALID_ARGUMENT;
    std::memset(out, 0, sizeof(*out));
    Profiler &p = profiler();
    std::lock_guard<std::mutex> lock(p.mu);
    out->n_kernels = K_SLOTS;
    out->timing = p.timing ? 1 : 0;
    for (int k = 0; k < K_SLOTS; ++k) {
        std::strncpy(out->name[k], kSlotNames[k], sizeof(out->name[k]) - 1);
        out->launches[k] = p.launches[k];
        out->kernels[k] = p.kernels[k];
        out->elements[k] = p.elements[k];
        out->total_ms[k] = p.timing ? p.ms[k] : -1.0;
    }
    return PANDORA_OK;
}

int pandora_dendrogram_async(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                             int32_t *edge_parent, int32_t *vertex_parent, void *workspace,
                             size_t workspace_bytes, void *stream)
{
    if (int e = check_common(u, v, w, n_edges, 1, edge_parent, vertex_parent))
        return e;
    return run(u, v, w, n_edges, 1, nullptr, edge_parent, vertex_parent, workspace,
               workspace_bytes, nullptr, (cudaStream_t)stream, false);
}

int pandora_dendrogram_batched_async(const int32_t *u, const int32_t *v, const float *w,
                                     const int64_t *edge_offsets, int64_t n_trees,
                                     int64_t total_edges, int32_t *edge_parent,
                                     int32_t *vertex_parent, void *workspace,
                                     size_t workspace_bytes, void *stream)
{
    if (int e = check_common(u, v, w, total_edges, n_trees, edge_parent, vertex_parent))
        return e;
    if (n_trees == 0)
        return total_edges == 0 ? PANDORA_OK : PANDORA_ERR_INVALID_ARGUMENT;
    if (!edge_offsets)
        return PANDORA_ERR_INVALID_ARGUMENT;
    return run(u, v, w, total_edges, n_trees, edge_offsets, edge_parent, vertex_parent, workspace,
               workspace_bytes, nullptr, (cudaStream_t)stream, false);
}

int pandora_dendrogram_batched_planned(const int32_t *u, const int32_t *v, const float *w,
                                       const int64_t *edge_offsets,
                                       const int64_t *host_edge_offsets, int64_t n_trees,
                                       int64_t total_edges, int32_t *edge_parent,
                                       int32_t *vertex_parent, void *workspace,
                                       size_t workspace_bytes, void *stream)
{
    if (int e = check_common(u, v, w, total_edges, n_trees, edge_parent, vertex_parent))
        return e;
    if (n_trees == 0)
        return total_edges == 0 ? PANDORA_OK : PANDORA_ERR_INVALID_ARGUMENT;
    if (!edge_offsets || !host_edge_offsets ||
        !offsets_partition(host_edge_offsets, n_trees, total_edges))
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (!workspace || workspace_bytes < total_workspace(total_edges, n_trees))
        return PANDORA_ERR_WORKSPACE_TOO_SMALL;
    if (total_edges == 0)
        return run_core(u, v, w, 0, n_trees, edge_offsets, edge_parent, vertex_parent, workspace,
                        workspace_bytes, nullptr, (cudaStream_t)stream, false);
    return run_planned(u, v, w, total_edges, n_trees, edge_offsets, host_edge_offsets,
                       edge_parent, vertex_parent, workspace, workspace_bytes,
                       (cudaStream_t)stream, false, tuning_snapshot());
}

int pandora_workspace_status(const void *workspace, void *stream)
{
    if (!workspace)
        return PANDORA_ERR_INVALID_ARGUMENT;
    const char *base = (const char *)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    int status = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&status, base, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    return status;
}

int pandora_set_tuning(const pandora_tuning *t)
{
    if (!t || t->small_max_edges < 0 || t->split_min_permille < 0 || t->split_min_permille > 1000)
        return PANDORA_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < 13; ++k)
        if (t->small_threads[k] != 256 && t->small_threads[k] != 512 && t->small_threads[k] != 1024)
            return PANDORA_ERR_INVALID_ARGUMENT;
    Tuning &g = tuning();
    std::lock_guard<std::mutex> lock(g.mu);
    g.t = *t;
    g.t.small_max_edges = std::min<int32_t>(t->small_max_edges, PANDORA_SMALL_CAP);
    return PANDORA_OK;
}

int pandora_get_tuning(pandora_tuning *t)
{
    if (!t)
        return PANDORA_ERR_INVALID_ARGUMENT;
    *t = tuning_snapshot();
    return PANDORA_OK;
}

const char *pandora_status_string(int status)
{
    switch (status) {
    case PANDORA_OK: return "ok";
    case PANDORA_ERR_INVALID_ARGUMENT: return "invalid argument";
    case PANDORA_ERR_NAN_WEIGHT: return "NaN weight";
    case PANDORA_ERR_VERTEX_OUT_OF_RANGE: return "vertex id out of range";
    case PANDORA_ERR_SELF_LOOP: return "self-loop edge";
    case PANDORA_ERR_NOT_A_TREE: return "input is not a tree (cycle / disconnected)";
    case PANDORA_ERR_ITERATION_LIMIT: return "device iteration limit reached";
    case PANDORA_ERR_OUT_OF_MEMORY: return "out of device memory";
    case PANDORA_ERR_CUDA: return "CUDA runtime error";
    case PANDORA_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case PANDORA_ERR_SIZE_LIMIT: return "input above the entry point's size limit";
    case PANDORA_ERR_BAD_WEIGHT: return "weight not positive and finite";
    case PANDORA_ERR_NOT_A_DENDROGRAM: return "parent arrays are not a weight-ordered binary dendrogram";
    case PANDORA_ERR_BAD_POINT: return "point coordinate not finite";
    default: return "unknown status";
    }
}

int pandora_set_wait_report_limit(int64_t spins)
{
    pandora::g_report_limit.store(spins < 0 || spins >= (int64_t)pandora::SPIN_LIMIT
                                      ? pandora::SPIN_LIMIT
                                      : (pandora::u32)spins);
    return PANDORA_OK;
}

int pandora_version(void) { return 100; }

}  // extern "C"

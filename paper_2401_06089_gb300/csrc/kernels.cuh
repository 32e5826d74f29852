// Launch interfaces of the kernels of the dendrogram path (internal to the
// library; the public C ABI is include/pandora.h).
#pragma once

#include "common.cuh"

namespace pandora {

// ---------------------------------------------------------------------------
// sort.cu - onesweep LSD radix sort (8-bit digits, decoupled look-back)
// ---------------------------------------------------------------------------
#ifndef PANDORA_OS_THREADS
#define PANDORA_OS_THREADS 512
#endif
#ifndef PANDORA_OS_ITEMS
#define PANDORA_OS_ITEMS 8
#endif
#ifndef PANDORA_OS_MIN_BLOCKS
#define PANDORA_OS_MIN_BLOCKS 2
#endif
constexpr int OS_THREADS = PANDORA_OS_THREADS;
constexpr int OS_ITEMS = PANDORA_OS_ITEMS;
constexpr int OS_MIN_BLOCKS = PANDORA_OS_MIN_BLOCKS;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;
constexpr int RADIX = 256;

enum OnesweepFlags : int {
    OS_KEY_FROM_W = 1,    // keys are weight_key(w[i]) computed on the fly
    OS_GEN_VALS = 2,      // value stream 0 is the input position (caller edge index);
                          // with OS_PAYLOAD_UV the endpoints come from the caller's u, v
    OS_WRITE_KEYS = 4,    // write the sorted keys
    OS_PAYLOAD_UV = 8,    // carry the endpoints (u, v) as value streams 1 and 2
    OS_LAST_AB = 16,      // write (u, v) as one int2 per edge (last weight pass)
    OS_FOREST = 32,       // endpoints are tree-local (batched mode, first pass)
};

struct OnesweepParams {
    const float *w_in;
    const u32 *keys_in;
    const u32 *vals_in;
    u32 *keys_out;
    u32 *vals_out;
    const int2 *uv_in;     // carried endpoints (OS_PAYLOAD_UV, later passes)
    int2 *uv_out;          // carried endpoints out; on the last pass the level-0 edges
    i64 n;
    int shift;
    const u32 *hist;       // [256] digit counts of this pass
    const u32 *bin_base;   // [256] their exclusive scan, or nullptr (scanned per tile)
    u64 *lb;               // [tiles * 256] look-back words, zeroed
    u32 *tile_counter;     // zeroed
    int *status;
    // caller endpoints (first pass) and level-0 output (last pass)
    const i32 *u;
    const i32 *v;
    i64 n_vertices;
    const i64 *edge_off;   // OS_FOREST
    i64 n_trees;
    u32 report_limit = SPIN_LIMIT;   // look-back waits longer than this record ITERATION_LIMIT
    int dbits = 8;         // digit width (9 only for the key-value sort, OS_WRITE_KEYS)
    // tiles this launch runs (0: all); a pass may be split into launches of
    // consecutive tile ranges on one stream, the tile counter carried over
    i64 grid_tiles = 0;
};

// Digit plan of an LSD sort: pass q sorts by the `width[q]` bits above
// `shift[q]`; its histogram row (2^width[q] counts) starts at off[q].
struct DigitPlan {
    int n;
    int shift[4];
    int width[4];
    int off[4];
};
// Plan for keys of `bits` significant bits: three passes of 8 or 9 bits for
// 25 to 27 bits, else 8-bit digits.  (Three passes over 28 to 30 bits need a
// 10-bit digit, whose 4096-key tiles write runs of four keys per digit: at
// 10^8 chain keys 10 + 9 + 9 bits took 3.54 ms against 2.94 ms for four
// 8-bit passes, while 9 + 9 + 8 bits at 2 * 10^7 took 0.60 against 0.64.)
DigitPlan digit_plan(int bits);
constexpr int DIGIT_PLAN_HIST = 4096;   // histogram entries of the widest plan
static_assert(sizeof(((Ctrl *)nullptr)->hist2) == DIGIT_PLAN_HIST * 4, "chain histogram size");

__host__ __device__ inline i64 onesweep_tiles(i64 n) { return (n + OS_TILE - 1) / OS_TILE; }

void launch_hist_weights(const float *w, i64 n, u32 *hist /*[4][256]*/, int *status,
                         cudaStream_t s);
void launch_onesweep(int flags, const OnesweepParams &p, cudaStream_t s);
// digit histograms of 32-bit keys for the four 8-bit passes ([4][256], added to)
void launch_hist_keys(const u32 *keys, i64 n, u32 *hist, cudaStream_t s);
// base[r][d] = sum of hist[r][d'] over d' < d, for `rows` rows of 256
void launch_hist_scan(const u32 *hist, u32 *base, int rows, cudaStream_t s);
// base = exclusive scan of every row of a digit plan's histogram
void launch_hist_scan_plan(const u32 *hist, u32 *base, const DigitPlan &plan, cudaStream_t s);

// ---------------------------------------------------------------------------
// levels.cu, mark.cu - one contraction level (Eq. 1, Eq. 2, Section 3.2)
// ---------------------------------------------------------------------------
constexpr int LV_THREADS = 256;
constexpr int LV_ITEMS = 8;
constexpr int LV_TILE = LV_THREADS * LV_ITEMS;

__host__ __device__ inline i64 level_tiles(i64 n) { return (n + LV_TILE - 1) / LV_TILE; }

// Lightest-incident-edge word of a vertex x on one level (Eq. 1):
//   bits 63..32  global rank r of the edge (ascending order of Section 3.1)
//   bits 31..1   the edge's other endpoint y
//   bit  0       side: 1 when x is the edge's second endpoint
// The minimum over x's edges is the lightest edge, and the word carries what
// the pointer forest and the chain key need without another gather.
constexpr u64 NO_EDGE = ~0ull;

struct LevelParams {
    int level;
    // sizes: the device counts are the truth; *_cap bound them (buffer
    // capacity) and *_grid is what the host sized the launch for
    const u64 *d_m;        // edges of this level
    const u64 *d_n;        // vertices of this level
    u64 *d_m_next;         // alpha-edges = edges of the next level
    u64 *d_n_next;         // roots = vertices of the next level
    i64 m_cap, n_cap;
    i64 m_grid, n_grid;
    int *d_n_levels;       // Ctrl::n_levels
    const int2 *ab;        // endpoints (level vertex ids), ascending rank
    const u32 *er;         // global rank of each edge (nullptr on level 0: rank = index)
    u64 *min_word;         // [n] lightest-incident-edge word (see above); on level 0
                           // compress swaps its low half for the supervertex
    i32 *ptr;              // [n] pointer forest scratch
    i32 *deep;             // [n] vertices the bounded walk left unresolved (list)
    i32 *uf;               // [n] union-find parents of those vertices
    i32 *root_of;          // [n] dense root id, stored at union-find representatives
    u64 *d_n_deep;         // length of the deep list
    int2 *rec;             // [n] {chain key, supervertex} kept for the expansion (levels >= 1)
    // level 0 only: vertex_parent output
    const u32 *perm;
    i32 *vertex_parent;
    const i64 *edge_off;   // forest mode (nullptr for one tree)
    i64 n_trees;
    // next level
    int2 *ab_next;
    u32 *er_next;
    i64 cap_next;          // capacity of ab_next / er_next
    unsigned char *lev;    // [M] contraction level of each edge (by rank)
    i32 *start;            // [M] supervertex holding the edge on the next level
    u64 *lb;               // look-back words (zeroed per level)
    u32 *tile_counter;     // three counters (zeroed per level)
    int *status;
    // bucketed marking: the level's incidences are first grouped by vertex
    // bucket (2^mark_shift vertices each) so that each bucket's atomics hit
    // a word range that stays in L2; mark_buckets == 0 marks directly
    int mark_shift;
    int mark_buckets;
    u32 *rec_x;            // [2 m] incidence records: vertex
    u64 *rec_w;            // [2 m] incidence records: candidate word
    u32 *mark_count;       // Ctrl::mark_count (zeroed per level)
    u32 *mark_cursor;      // Ctrl::mark_cursor (zeroed per level)
    u64 *mark_base;        // Ctrl::mark_base
    // level 0 with bucketed marking: the records also carry the caller id of
    // their edge, and after the minima are applied a pass over the records in
    // bucket order finds the record that won at each vertex and
    //   - sets the edge's bit for that endpoint in eflag (2 bits per edge by
    //     rank: bit 0 lightest at the first endpoint, bit 1 at the second;
    //     Eq. 2 reads them: alpha = no bit, leaf edge = both bits),
    //   - writes vertex_parent (Eq. 1) from the record's caller id,
    // so that ptr_init and compact need no random read to classify an edge.
    // eflag == nullptr: classify by reading the endpoints' words.
    u32 *rec_c;            // [2 m] incidence records: caller edge id
    u32 *eflag;            // [ceil(m / 16)] zeroed
    // forests, level 0: roots found per tree and the dense id of one of them
    // (zeroed counts).  A tree with a single root is one supervertex, so a
    // vertex whose bounded walk does not reach a root takes that id instead
    // of going to union-find (the whole level of such a tree is one chain,
    // Section 3.2).  A single tree uses the level's root count instead.
    u32 *tree_roots;       // [n_trees]
    i32 *tree_root_id;     // [n_trees]
    // look-back waits and union-find loops running longer than this record
    // PANDORA_ERR_ITERATION_LIMIT (and go on to their hard bounds)
    u32 report_limit = SPIN_LIMIT;
};

// Process-wide report limit of the bounded device loops (host side).
u32 wait_report_limit();

__host__ __device__ inline i64 eflag_words(i64 m) { return (m + 15) / 16; }

// Level kernels run only while the loop is open: once a level without
// alpha-edges has set n_levels, kernels launched for later (bound) levels
// exit at once.
__device__ __forceinline__ bool loop_closed(const LevelParams &p)
{
    return *(const volatile int *)p.d_n_levels != 0;
}

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
inline unsigned grid_for(i64 n, int per_block, int bps = PANDORA_LV_BPS)
{
    i64 b = (n + per_block - 1) / per_block;
    const i64 cap = 152 * bps;
    if (b > cap)
        b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

void launch_init_level(const LevelParams &p, cudaStream_t s);   // min_word = NO_EDGE
void launch_mark(const LevelParams &p, cudaStream_t s);   // with eflag: also the flag pass
void launch_ptr_init(const LevelParams &p, cudaStream_t s);
void launch_compress(const LevelParams &p, cudaStream_t s);   // walk + union-find fallback
void launch_compact(const LevelParams &p, cudaStream_t s);

// ---------------------------------------------------------------------------
// expand.cu, link.cu - multilevel expansion (Section 3.3.2) and chain linking (3.3.3)
// ---------------------------------------------------------------------------
struct LevelTable {
    const int2 *rec[MAX_LEVELS];   // {chain key, supervertex} of every vertex of level l >= 1
    i64 n_cap[MAX_LEVELS];         // capacity of rec[l]
};

struct ExpandParams {
    i64 m;
    int max_levels;        // levels launched (bound); the device count is in *d_n_levels
    const int *d_n_levels;
    const u64 *lvl_n;      // Ctrl::lvl_n (vertices of every level)
    const unsigned char *lev;
    const i32 *start;
    const u32 *perm;
    u32 *keys_out;
    u32 root_base;
    const i64 *edge_off;   // forest mode
    i64 n_trees;
    u32 *hist;             // digit histograms of the chain keys, rows of `plan`
    DigitPlan plan;
    int *status;
};

void launch_expand(const ExpandParams &p, const LevelTable &t, cudaStream_t s);

struct LinkParams {
    i64 m;
    const u32 *skeys;      // chain keys sorted
    const u32 *svals;      // caller edge ids in the same order
    const u32 *perm;
    u32 root_base;
    i32 *edge_parent;
    const i64 *edge_off;
    i64 n_trees;
    // bucketed link (n_buckets > 0): the (edge, parent) pairs are first
    // written grouped by caller-id bucket (2^bucket_shift ids, whose
    // edge_parent range stays in L2), then applied bucket after bucket.
    // The caller ids are a permutation of [0, m), so bucket b holds exactly
    // the ids [b << shift, (b + 1) << shift) and starts at rec + (b << shift).
    int bucket_shift;
    int n_buckets;
    int2 *rec;             // [m] (edge, parent) pairs by bucket
    u32 *cursor;           // [n_buckets] write cursors, zeroed
    // the apply pass in apply_parts launches over consecutive bucket ranges
    // (ids [k * per, (k + 1) * per), per a whole number of buckets), the
    // event apply_done[k] recorded after launch k; 0 or 1: one launch
    int apply_parts = 0;
    cudaEvent_t *apply_done = nullptr;
    i64 apply_begin = 0;   // record range of one launch (apply_end 0: all)
    i64 apply_end = 0;
};

void launch_link(const LinkParams &p, cudaStream_t s);

// ---------------------------------------------------------------------------
// small.cu - single-CTA solver (whole method in shared memory, m <= 4096)
// ---------------------------------------------------------------------------
struct SmallParams {
    const i32 *u;
    const i32 *v;
    const float *w;
    i64 m;                 // one tree: its edge count (edge_off == nullptr)
    const i64 *edge_off;   // batched: per-tree offsets
    i64 n_trees;
    const i32 *tree_list;  // batched: the trees this launch takes (block b -> tree_list[b]),
                           // or nullptr for block b -> tree b
    i64 cutoff;            // trees with more edges are skipped (forest pipeline)
    i64 total_edges;       // batched: edges of the whole batch (bounds every tree)
    i32 *edge_parent;
    i32 *vertex_parent;
    int *status;
};

int small_tree_capacity();
// Layout capacity (256, 1024 or 4096 edges) that holds trees of max_edges.
int small_layout_capacity(i64 max_edges);
// One block per tree; every tree the launch covers has at most max_edges edges.
void launch_small(const SmallParams &p, int threads, i64 max_edges, unsigned blocks,
                  cudaStream_t s);
// The last levels of a single tree in one block: once a level has at most
// TAIL_CAP edges, one block runs that level and every later one in shared
// memory (Eq. 1, Eq. 2, Section 3.2) and writes what the expansion reads:
// the contraction level and supervertex of every edge it contracts, the
// {chain key, supervertex} record of every vertex of each level, and the
// level sizes and level count in the control block.
constexpr int TAIL_CAP = 4096;
constexpr int TAIL_MAX_LEVELS = 16;
struct TailParams {
    int level;              // first level the block runs
    const u64 *d_m;         // Ctrl::lvl_m (indexed by level)
    u64 *lvl_m;
    u64 *lvl_n;
    int *d_n_levels;        // Ctrl::n_levels; nonzero: an earlier level ended the loop
    const int2 *ab;         // the level's edges (level vertex ids), ascending rank
    const u32 *er;          // their global ranks
    i64 ab_cap;             // capacity of ab / er
    unsigned char *lev;     // [M] contraction level of every edge
    i32 *start;             // [M] supervertex on the next level
    int2 *rec[TAIL_MAX_LEVELS];   // records of levels level .. level + TAIL_MAX_LEVELS - 1
    i64 rec_cap[TAIL_MAX_LEVELS];
    int max_levels;         // bound on the levels of the whole loop
    int *status;
};
void launch_tail(const TailParams &p, cudaStream_t s);

// Size classes of a batched call: 0..12 = single-block buckets (2^k <= m <
// 2^(k+1); bucket 0 also takes m = 0), 13 = trees for the forest pipeline.
constexpr int N_CLASSES = 14;
constexpr int CLASS_LARGE = 13;
__host__ __device__ inline int size_class(i64 m, i64 cutoff)
{
    if (m > cutoff)
        return CLASS_LARGE;
    int k = 0;
    while (k < 12 && (i64(2) << k) <= m)
        ++k;
    return k;
}

// The device half of a plan the host made from its copy of the offsets:
// tree lists per class (large trees first, then bucket 0, 1, ...) and the
// packed offsets of the large trees.  The host's counts are checked against
// the device offsets; a mismatch is PANDORA_ERR_INVALID_ARGUMENT and leaves
// lists and offsets that stay inside their buffers.
struct PlanParams {
    const i64 *off;
    i64 n_trees;
    i64 total_edges;
    i64 cutoff;
    i32 *lists;                // [n_trees]
    i64 *coff;                 // [count[CLASS_LARGE] + 1]
    int *status;
    i64 base[N_CLASSES];       // first list slot of each class
    i64 count[N_CLASSES];      // trees of each class (host plan)
    i64 m_large;               // edges of the large trees (host plan)
};
void launch_plan(const PlanParams &p, cudaStream_t s);
// *to gets *from when *from holds an error (a plan error is the cause of
// whatever the kernels that followed it found).
void launch_merge_status(const int *from, int *to, cudaStream_t s);

// Packs the large trees (lists[0, n_list)) into one forest with offsets coff,
// and copies that forest's outputs back.  Trees whose sizes disagree with
// the packed offsets are skipped.
void launch_gather_trees(const i32 *u, const i32 *v, const float *w, const i64 *off, i64 n_trees,
                         i64 total, const i32 *list, const i64 *coff, i64 n_list, i64 packed_total,
                         i32 *cu, i32 *cv, float *cw, cudaStream_t s);
void launch_scatter_trees(const i32 *cep, const i32 *cvp, const i64 *off, i64 n_trees, i64 total,
                          const i32 *list, const i64 *coff, i64 n_list, i64 packed_total, i32 *ep,
                          i32 *vp, cudaStream_t s);

// forest mode: check the offsets (off[0] == 0, non-decreasing, off[T] == M)
void launch_check_offsets(const i64 *off, i64 n_trees, i64 total, int *status, cudaStream_t s);
// two 64-bit device words set from kernel parameters (graph-capture safe)
void launch_set_u64_pair(u64 *a, u64 va, u64 *b, u64 vb, cudaStream_t s);
// vertex_parent = -1 for every vertex of an edgeless input
void launch_fill(i32 *p, i64 n, i32 value, cudaStream_t s);

}  // namespace pandora

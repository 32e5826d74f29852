/*
 * pandora.h - C ABI of the GB300 (sm_103a) single-linkage dendrogram library.
 *
 * Given a tree of n vertices and m = n - 1 weighted edges (for instance the
 * minimum spanning tree of a point set), the library computes its
 * single-linkage dendrogram with the recursive tree-contraction method of
 * PANDORA (Sao, Prokopenko, Lebrun-Grandie, arXiv 2401.06089):
 *
 *   - the edges are sorted by (weight, edge index)          (Section 3.1)
 *   - every vertex marks its lightest incident edge         (Eq. 1)
 *   - edges marked by neither endpoint are alpha-edges      (Eq. 2)
 *   - all other edges are contracted, the tree of alpha-edges is solved
 *     recursively                                           (Section 3.2)
 *   - every contracted edge is assigned to a dendrogram chain, the chains
 *     are sorted and stitched                               (Section 3.3,
 *                                                            Algorithm 1)
 *
 * Output (the parent function P of Section 3.1): for every edge e,
 * edge_parent[e] is the index of its parent edge, or -1 for the root (the
 * heaviest edge); for every vertex x, vertex_parent[x] is the index of its
 * parent edge, which is its lightest incident edge (Eq. 1), or -1 when the
 * tree has a single vertex.  Results are exact integers: the weights are only
 * compared, never combined.
 *
 * Edge order (Section 3.1 asks for a consistent tie rule; this library reads
 * it as): edge e is lighter than edge f iff w_e < w_f, or the weights are
 * equal and e is -0.0 while f is +0.0, or they are equal with the same sign
 * and e < f (caller index).  -inf, +inf, subnormal and negative weights are
 * allowed; NaN is an error.
 *
 * Memory: every pointer argument is DEVICE memory of the current CUDA device
 * unless stated otherwise, owned by the caller, and must stay valid until the
 * work enqueued on `stream` has finished.  The library never frees caller
 * memory.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).
 *
 * Errors: every entry point returns a pandora_status.  Argument errors are
 * found on the host before any work is enqueued.  Errors found by the kernels
 * (NaN weight, vertex id out of range, self-loop, input that is not a tree,
 * an internal iteration limit) are collected in a device status word; the
 * blocking entry points below read it before returning.  On any error the
 * contents of the output arrays are unspecified.
 */
#ifndef PANDORA_H
#define PANDORA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pandora_status {
    PANDORA_OK = 0,
    PANDORA_ERR_INVALID_ARGUMENT = 1,   /* null pointer, negative size, bad offsets ... */
    PANDORA_ERR_NAN_WEIGHT = 2,         /* a weight is NaN */
    PANDORA_ERR_VERTEX_OUT_OF_RANGE = 3,/* an endpoint id is outside [0, n) */
    PANDORA_ERR_SELF_LOOP = 4,          /* an edge has u == v */
    PANDORA_ERR_NOT_A_TREE = 5,         /* the edges contain a cycle (so the graph is
                                           disconnected, since m = n - 1) */
    PANDORA_ERR_ITERATION_LIMIT = 6,    /* a bounded device loop gave up (never expected
                                           on valid input) */
    PANDORA_ERR_OUT_OF_MEMORY = 7,      /* scratch allocation failed */
    PANDORA_ERR_CUDA = 8,               /* a CUDA runtime call failed */
    PANDORA_ERR_WORKSPACE_TOO_SMALL = 9,/* caller workspace below pandora_workspace_size() */
    PANDORA_ERR_SIZE_LIMIT = 10,        /* n_edges above PANDORA_NOALLOC_MAX_EDGES, or
                                           n_vertices above PANDORA_FLAT_MAX_VERTICES */
    PANDORA_ERR_BAD_WEIGHT = 11,        /* flat clusters: a weight is not positive and
                                           finite (lambda = 1 / w is needed) */
    PANDORA_ERR_NOT_A_DENDROGRAM = 12,  /* flat clusters: the parent arrays are not a
                                           binary tree with one root in which every
                                           edge comes after its children in the
                                           (weight, index) order */
    PANDORA_ERR_BAD_POINT = 13          /* spanning tree of points: a coordinate is
                                           not finite */
} pandora_status;

/* Per-call statistics (optional output of the *_ws entry points). */
#define PANDORA_MAX_LEVELS 64
typedef struct pandora_stats {
    int32_t n_levels;                         /* contraction levels run (Section 3.2) */
    int32_t reserved;
    int64_t level_edges[PANDORA_MAX_LEVELS];  /* edges of level l (level 0 = all edges) */
    int64_t level_vertices[PANDORA_MAX_LEVELS];
} pandora_stats;

/*
 * Dendrogram of one tree (Algorithm 1).
 *   u, v          int32[n_edges]: endpoints, vertex ids in [0, n_edges].
 *   w             float[n_edges]: weights.
 *   n_edges       m >= 0; the tree has n = m + 1 vertices; m + 1 <= INT32_MAX.
 *   edge_parent   int32[n_edges] out (may be NULL when n_edges == 0).
 *   vertex_parent int32[n_edges + 1] out.
 * Scratch memory is taken stream-ordered from a library-owned CUDA memory
 * pool.  The call blocks the calling host thread until the result is complete
 * on `stream` (it reads the level sizes back between contraction levels) and
 * returns the device-detected status.
 */
int pandora_dendrogram(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                       int32_t *edge_parent, int32_t *vertex_parent, void *stream);

/*
 * As pandora_dendrogram, but u, v, w, edge_parent and vertex_parent are HOST
 * memory (pinned memory copies fastest; pageable memory works).  The paper has
 * no counterpart: this is the transfer schedule around its method for data
 * that lives on the host.  Device memory for the inputs, the outputs and the
 * workspace comes from the library's pool.  The copies overlap the path: the
 * weights go first (the histogram pass needs only them) while the endpoints
 * follow on a second stream, which the first sort pass waits for;
 * vertex_parent is copied back on a third stream as soon as level 0 has
 * written it (Eq. 1), while the other levels, the expansion and the linking
 * run; edge_parent follows the last kernel.  Blocking: returns when both
 * outputs are in host memory (the stream is synchronised).  Host buffers must
 * stay valid and unmodified until the call returns.  Errors as
 * pandora_dendrogram.
 */
int pandora_dendrogram_host(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                            int32_t *edge_parent, int32_t *vertex_parent, void *stream);

/*
 * Bytes of caller workspace that pandora_dendrogram_ws / _batched_ws need for
 * a total of `total_edges` edges in `n_trees` trees (n_trees = 1 for a single
 * tree).  Writes the size to *bytes.  Host only; enqueues nothing.
 */
int pandora_workspace_size(int64_t total_edges, int64_t n_trees, size_t *bytes);

/*
 * As pandora_dendrogram, with caller-provided device workspace (at least
 * pandora_workspace_size(n_edges, 1) bytes, 256-byte aligned) and optional
 * host-memory statistics (NULL to skip).  Allocates nothing.
 */
int pandora_dendrogram_ws(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                          int32_t *edge_parent, int32_t *vertex_parent, void *workspace,
                          size_t workspace_bytes, pandora_stats *stats, void *stream);

/*
 * Dendrograms of many independent trees in one pass (the whole batch is
 * processed as one forest: one sort, one contraction loop, one expansion).
 *   edge_offsets  int64[n_trees + 1], DEVICE memory: tree t owns the edges
 *                 [edge_offsets[t], edge_offsets[t+1]) and the vertices
 *                 [edge_offsets[t] + t, edge_offsets[t+1] + t + 1) of the
 *                 packed arrays.  edge_offsets[0] = 0, non-decreasing.
 *   total_edges   must equal edge_offsets[n_trees] (checked on the device).
 *   u, v          int32[total_edges]: TREE-LOCAL vertex ids (0 .. n_t - 1).
 *   w             float[total_edges].
 *   edge_parent   int32[total_edges] out: tree-local edge ids or -1.
 *   vertex_parent int32[total_edges + n_trees] out: tree-local edge ids, or -1
 *                 for a tree with a single vertex.
 * total_edges + n_trees <= INT32_MAX.  Blocking, like pandora_dendrogram.
 * Every tree's result equals the result of pandora_dendrogram on that tree.
 */
int pandora_dendrogram_batched(const int32_t *u, const int32_t *v, const float *w,
                               const int64_t *edge_offsets, int64_t n_trees, int64_t total_edges,
                               int32_t *edge_parent, int32_t *vertex_parent, void *stream);

/* As pandora_dendrogram_batched with caller workspace
 * (pandora_workspace_size(total_edges, n_trees) bytes) and optional stats. */
int pandora_dendrogram_batched_ws(const int32_t *u, const int32_t *v, const float *w,
                                  const int64_t *edge_offsets, int64_t n_trees,
                                  int64_t total_edges, int32_t *edge_parent,
                                  int32_t *vertex_parent, void *workspace,
                                  size_t workspace_bytes, pandora_stats *stats, void *stream);

/*
 * Asynchronous variants (same arguments as the *_ws entry points, minus the
 * statistics).  They enqueue the whole pipeline on `stream` and return at
 * once: no host synchronisation, no allocation, no host memory read by the
 * enqueued work, so a call can be captured into a CUDA graph and replayed.
 * The contraction loop is enqueued for its worst case, ceil(log2(m + 1))
 * levels (Section 4.2); kernels of levels past the last one exit at once.
 * The return value reports argument errors only; errors found by the kernels
 * stay in the workspace's status word until pandora_workspace_status() reads
 * it.  The workspace must not be shared by calls in flight at the same time.
 */
int pandora_dendrogram_async(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                             int32_t *edge_parent, int32_t *vertex_parent, void *workspace,
                             size_t workspace_bytes, void *stream);
int pandora_dendrogram_batched_async(const int32_t *u, const int32_t *v, const float *w,
                                     const int64_t *edge_offsets, int64_t n_trees,
                                     int64_t total_edges, int32_t *edge_parent,
                                     int32_t *vertex_parent, void *workspace,
                                     size_t workspace_bytes, void *stream);

/*
 * Asynchronous batched call for a caller that also holds the offsets in host
 * memory (host_edge_offsets: n_trees + 1 values equal to edge_offsets; read
 * during the call only).  With them the library splits the batch without a
 * host synchronisation: trees of at most small_max_edges edges (see
 * pandora_set_tuning) go to the single-block solver, one block per tree and
 * one launch per size bucket; the others are packed into one forest for the
 * pipeline and their results copied back.  A batch is split only when its
 * small trees hold at least split_min_permille of the edges or there are no
 * large trees (the packing costs about 40 bytes of copies per large-tree
 * edge); otherwise it runs as pandora_dendrogram_batched_async.  Every launch
 * has a grid fixed by the host offsets, so the call can be captured in a CUDA
 * graph and replayed for batches with the same tree sizes.  The device checks
 * the host plan against edge_offsets; a mismatch is
 * PANDORA_ERR_INVALID_ARGUMENT in the workspace's status word.
 * Returns PANDORA_ERR_INVALID_ARGUMENT at once when host_edge_offsets is
 * null or not a partition of [0, total_edges) (non-decreasing, first 0, last
 * total_edges); other errors as pandora_dendrogram_batched_async.  Workspace:
 * pandora_workspace_size(total_edges, n_trees) bytes.
 */
int pandora_dendrogram_batched_planned(const int32_t *u, const int32_t *v, const float *w,
                                       const int64_t *edge_offsets,
                                       const int64_t *host_edge_offsets, int64_t n_trees,
                                       int64_t total_edges, int32_t *edge_parent,
                                       int32_t *vertex_parent, void *workspace,
                                       size_t workspace_bytes, void *stream);

/* Waits for `stream` and returns the device status word of the last call
 * that used `workspace` (PANDORA_OK when it found no error). */
int pandora_workspace_status(const void *workspace, void *stream);

/*
 * Failure reporting of the bounded device loops (process-wide, host only;
 * the paper has no counterpart).  Every wait of a kernel on another block
 * (the single-pass scans' and sorts' look-back) and every union-find loop of
 * the contraction (Section 3.2) is bounded; a loop that runs into its bound
 * records PANDORA_ERR_ITERATION_LIMIT in the call's status word, which the
 * blocking entry points return and pandora_workspace_status reads.  This
 * setter makes those loops record that status as soon as they run longer
 * than `spins` iterations, WITHOUT cutting them short: the results stay
 * exact, only the status reports the long loop.  It exists so that a test
 * can drive the reporting path on a real GPU without faulting or hanging
 * it.  spins < 0 restores the default (report only at the hard bound).
 * Calls already enqueued keep the limit they were enqueued with.  Returns
 * PANDORA_OK.
 */
int pandora_set_wait_report_limit(int64_t spins);

/*
 * Allocation-free variant of pandora_dendrogram.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory at the time of the call -- for example code whose device
 * memory is entirely owned by another allocator (a framework that reserved
 * the GPU up front), or a latency-critical loop in which cudaMalloc/cudaFree
 * would synchronise the device.  It takes the same arguments and gives the
 * same result as pandora_dendrogram, but its scratch memory is a fixed
 * 32 MiB array in the library's device image (held by every GPU that loads
 * the library until the process exits), so it accepts at most
 * PANDORA_NOALLOC_MAX_EDGES edges and returns PANDORA_ERR_SIZE_LIMIT above
 * that.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * The first call on a device looks up the device address of the array on
 * that device (cudaGetSymbolAddress, with the device current); make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: it belongs to the device's primary context, so the entry
 * point must not be used after cudaDeviceReset or from a non-primary
 * context.  Every call reuses the same array
 * and leaves its contents behind; each call clears what it needs zeroed, but
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on the array and must be serialised by the caller.  Blocking, like
 * pandora_dendrogram.
 */
#define PANDORA_NOALLOC_MAX_EDGES 262143
int pandora_dendrogram_noalloc(const int32_t *u, const int32_t *v, const float *w,
                               int64_t n_edges, int32_t *edge_parent, int32_t *vertex_parent,
                               void *stream);

/*
 * Small trees (process-wide tuning, thread-safe; host only).  The paper has
 * no counterpart: its method is run unchanged, only the launch shape differs.
 *
 * A tree with at most small_max_edges edges is solved by one thread block
 * that runs every step of Algorithm 1 (sort, contraction levels of Eq. 1 and
 * Eq. 2, expansion and linking of Section 3.3) in shared memory: one launch
 * and no DRAM traffic beyond its input and output.  Results are identical to
 * the multi-kernel pipeline's.  It is used by
 *   - single-tree calls (blocking, asynchronous and allocation-free) that do
 *     not ask for statistics, when n_edges <= small_max_edges;
 *   - batched blocking calls (which read the offsets back) and
 *     pandora_dendrogram_batched_planned: trees at or under the cutoff go one
 *     block per tree, grouped by size bucket; the others are packed into one
 *     forest for the pipeline, when the small trees hold at least
 *     split_min_permille per mille of the batch's edges (or all of them).
 *     pandora_dendrogram_batched_async, which never sees the offsets on the
 *     host, always takes the forest pipeline.
 * small_threads[k] is the block size (256, 512 or 1024) for trees of
 * 2^k .. 2^(k+1)-1 edges (bucket 0 also takes empty trees).  small_max_edges
 * is clamped to PANDORA_SMALL_CAP; 0 disables the solver.  Defaults: 4096
 * edges, 512 threads in every bucket, 50 per mille; measured values come
 * from the autotuner (paper_2401_06089_gb300/autotune.py).
 *
 * set: PANDORA_ERR_INVALID_ARGUMENT for a null pointer, a negative cutoff, a
 * block size other than 256/512/1024 or split_min_permille outside
 * [0, 1000] (nothing changes then).  Calls already running keep the settings
 * they started with.
 * get: copies the settings in force; PANDORA_ERR_INVALID_ARGUMENT on null.
 */
#define PANDORA_SMALL_CAP 4096
typedef struct pandora_tuning {
    int32_t small_max_edges;
    int32_t small_threads[13];
    int32_t split_min_permille;
} pandora_tuning;

int pandora_set_tuning(const pandora_tuning *tuning);
int pandora_get_tuning(pandora_tuning *tuning);

/*
 * Optional instrumentation (process-wide, thread-safe, host memory).
 * pandora_profile_start resets the counters of every kernel of the path.  The
 * library always counts launches; with with_timing != 0 it also records a
 * CUDA event pair around every launch on the launching stream and adds the
 * elapsed time to the kernel's total when the call completes.
 * pandora_profile_read copies the counters into *out.  Enqueues nothing.
 */
#define PANDORA_PROFILE_SLOTS 16
typedef struct pandora_profile {
    int32_t n_kernels;
    int32_t timing;                               /* 1 when total_ms is valid */
    char name[PANDORA_PROFILE_SLOTS][32];
    int64_t launches[PANDORA_PROFILE_SLOTS];
    int64_t elements[PANDORA_PROFILE_SLOTS];      /* items processed (edges or vertices) */
    double total_ms[PANDORA_PROFILE_SLOTS];
    int64_t kernels[PANDORA_PROFILE_SLOTS];       /* CUDA kernels launched (a step of the
                                                     path can take several: the bucketed
                                                     marking 4, root finding 4) */
} pandora_profile;

int pandora_profile_start(int with_timing);
int pandora_profile_read(pandora_profile *out);

/*
 * HDBSCAN* flat clusters of a dendrogram (the optional last step of the
 * HDBSCAN* pipeline, Section 6.5, as defined by Campello et al.).
 *
 * Input: a dendrogram of n_vertices = m + 1 points as produced by
 * pandora_dendrogram (device arrays): edge_parent[m] (-1 at the root edge),
 * vertex_parent[n_vertices] and the weights w[m] (positive and finite;
 * lambda(e) = 1 / w(e) in float64).  As edges are removed from the heaviest
 * down, a cluster is a part of the tree that stays at least min_cluster_size
 * points large: it is born where its part splits off (the whole tree at
 * lambda 0), ends where it splits into two such parts, and loses the points
 * that fall off in smaller parts.  Its stability is the sum over its points
 * of (lambda at which the point leaves it - lambda at its birth), each term
 * in float64, summed exactly and rounded once (so the value does not depend
 * on any order).  Excess of mass: over all clusters but the whole tree, the
 * set of non-nested clusters of largest total stability, totals taken
 * exactly; a cluster is kept instead of the best set under it when its
 * stability is at least that set's total (a parent wins a tie).
 *
 * Output: labels[n_vertices] (device): the kept cluster that contains the
 * point, numbered 0, 1, ... in increasing order of each cluster's smallest
 * point id, or -1 for noise.  cluster_stability (device, optional, NULL to
 * skip): room for n_vertices / min_cluster_size doubles; entry k receives
 * the stability of cluster k.  n_clusters (host, optional): the number of
 * kept clusters.
 *
 * min_cluster_size >= 2 (else PANDORA_ERR_INVALID_ARGUMENT); at most
 * PANDORA_FLAT_MAX_VERTICES points (else PANDORA_ERR_SIZE_LIMIT).  The input
 * is validated on the device: PANDORA_ERR_BAD_WEIGHT,
 * PANDORA_ERR_NOT_A_DENDROGRAM.  Scratch (130 bytes per point plus 640 bytes
 * per possible cluster, 2 n_vertices / min_cluster_size + 1: 21 GB for 10^8
 * points at min_cluster_size 16, 77 GB at 2) comes from the library's
 * stream-ordered pool; PANDORA_ERR_OUT_OF_MEMORY when it does not fit.  Blocking: returns after the work on `stream` has finished.
 */
#define PANDORA_FLAT_MAX_VERTICES 536870912
int pandora_hdbscan_labels(const int32_t *edge_parent, const int32_t *vertex_parent,
                           const float *w, int64_t n_vertices, int32_t min_cluster_size,
                           int32_t *labels, double *cluster_stability, int64_t *n_clusters,
                           void *stream);

/* Static description of a status code (never NULL). */
const char *pandora_status_string(int status);

/* Library version as 10000 * major + 100 * minor + patch. */
int pandora_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PANDORA_H */

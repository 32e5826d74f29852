/*
 * CPU oracle for the single-linkage dendrogram of a weighted tree.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is compared against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * What it computes (paper, Section 2.2.2, bottom-up construction): visit the
 * edges from the lightest to the heaviest; for each edge find the clusters of
 * its two endpoints with a union-find structure and make the edge the parent
 * of both clusters' current top nodes.  The top node of a cluster is either a
 * vertex (a singleton cluster) or the edge that created the cluster.  The
 * paper proves (Theorems 1-3, Section 3.4) that its tree-contraction method
 * reaches exactly this dendrogram, so no part of that method is restated here.
 *
 * Order of edges (paper, Section 3.1: edges sorted by weight, ties ordered
 * consistently).  Reading used: edge e precedes edge f ("e is lighter") iff
 * w_e < w_f as IEEE numbers, or the weights are equal and e is -0.0 while f is
 * +0.0, or the weights are equal with the same sign and e < f as caller
 * indices.  NaN weights are rejected.
 *
 * Output encoding (paper, Section 3.1, parent function P): edge_parent[e] is
 * the caller index of the parent edge of edge e, or -1 for the root (the
 * heaviest edge); vertex_parent[x] is the caller index of the parent edge of
 * vertex x (Eq. 1: its lightest incident edge), or -1 when the tree has a
 * single vertex and no edges.
 *
 * Parity is pinned by the tests against brute-force rules, the top-down
 * construction, closed forms (star, path) and Theorem 1; nothing here is
 * "parity unpinned".
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID_ARGUMENT 1
#define ORACLE_ERR_NAN_WEIGHT 2
#define ORACLE_ERR_VERTEX_OUT_OF_RANGE 3
#define ORACLE_ERR_SELF_LOOP 4
#define ORACLE_ERR_NOT_A_TREE 5
#define ORACLE_ERR_OUT_OF_MEMORY 7

/* 1 when edge a is lighter than edge b under the order described above. */
static int lighter(const float *w, int32_t a, int32_t b)
{
    float wa = w[a];
    float wb = w[b];
    if (wa < wb)
        return 1;
    if (wa > wb)
        return 0;
    /* equal as numbers: only -0.0 and +0.0 can still differ */
    int sa = signbit(wa) ? 1 : 0;
    int sb = signbit(wb) ? 1 : 0;
    if (sa != sb)
        return sa; /* the negative zero is the lighter one */
    return a < b;
}

/* Stable merge of the sorted runs idx[lo, mid) and idx[mid, hi) by the order
 * above (on equal keys the left run goes first). */
static void merge_runs(int32_t *idx, int32_t *tmp, int64_t lo, int64_t mid, int64_t hi,
                       const float *w)
{
    int64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi) {
        if (lighter(w, idx[j], idx[i]))
            tmp[k++] = idx[j++];
        else
            tmp[k++] = idx[i++];
    }
    while (i < mid)
        tmp[k++] = idx[i++];
    while (j < hi)
        tmp[k++] = idx[j++];
    memcpy(idx + lo, tmp + lo, (size_t)(hi - lo) * sizeof(int32_t));
}

/* Top-down merge sort of edge indices by the order above. */
static void merge_sort(int32_t *idx, int32_t *tmp, int64_t lo, int64_t hi, const float *w)
{
    if (hi - lo < 2)
        return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_sort(idx, tmp, lo, mid, w);
    merge_sort(idx, tmp, mid, hi, w);
    merge_runs(idx, tmp, lo, mid, hi, w);
}

/* Union-find root with path halving. */
static int32_t find_root(int32_t *uf, int32_t x)
{
    while (uf[x] != x) {
        uf[x] = uf[uf[x]];
        x = uf[x];
    }
    return x;
}

/*
 * Sorted order of the edges (ascending: lightest first).  order[k] is the
 * caller index of the k-th lightest edge.  Returns 0 or an error code.
 */
int oracle_edge_order(const float *w, int64_t n_edges, int32_t *order)
{
    if (n_edges < 0 || (n_edges > 0 && (!w || !order)))
        return ORACLE_ERR_INVALID_ARGUMENT;
    for (int64_t e = 0; e < n_edges; ++e)
        if (isnan(w[e]))
            return ORACLE_ERR_NAN_WEIGHT;
    int32_t *tmp = (int32_t *)malloc((size_t)(n_edges > 0 ? n_edges : 1) * sizeof(int32_t));
    if (!tmp)
        return ORACLE_ERR_OUT_OF_MEMORY;
    for (int64_t e = 0; e < n_edges; ++e)
        order[e] = (int32_t)e;
    merge_sort(order, tmp, 0, n_edges, w);
    free(tmp);
    return ORACLE_OK;
}

/*
 * The same order computed by several threads (the all-core timing mode, which
 * mirrors a parallel sort followed by a sequential union-find): the index
 * array is cut into n_threads runs, each run is merge-sorted by its own
 * thread, and the runs are merged pairwise, the merges of one round in
 * parallel.  Every merge is the stable merge above, so the result is the same
 * permutation as oracle_edge_order's (the order is total).
 */
struct sort_job {
    int32_t *idx, *tmp;
    int64_t lo, mid, hi;
    const float *w;
};

static void *sort_run(void *arg)
{
    struct sort_job *j = (struct sort_job *)arg;
    merge_sort(j->idx, j->tmp, j->lo, j->hi, j->w);
    return NULL;
}

static void *merge_job(void *arg)
{
    struct sort_job *j = (struct sort_job *)arg;
    merge_runs(j->idx, j->tmp, j->lo, j->mid, j->hi, j->w);
    return NULL;
}

int oracle_edge_order_threads(const float *w, int64_t n_edges, int32_t *order, int n_threads)
{
    if (n_threads <= 1 || n_edges < 2 * (int64_t)n_threads)
        return oracle_edge_order(w, n_edges, order);
    if (n_threads > 256)
        n_threads = 256;
    for (int64_t e = 0; e < n_edges; ++e)
        if (isnan(w[e]))
            return ORACLE_ERR_NAN_WEIGHT;
    int32_t *tmp = (int32_t *)malloc((size_t)n_edges * sizeof(int32_t));
    if (!tmp)
        return ORACLE_ERR_OUT_OF_MEMORY;
    for (int64_t e = 0; e < n_edges; ++e)
        order[e] = (int32_t)e;
    int64_t bound[257];
    for (int t = 0; t <= n_threads; ++t)
        bound[t] = n_edges * t / n_threads;
    struct sort_job jobs[256];
    pthread_t th[256];
    int status = ORACLE_OK;
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = (struct sort_job){order, tmp, bound[t], bound[t], bound[t + 1], w};
        if (pthread_create(&th[t], NULL, sort_run, &jobs[t]) != 0) {
            sort_run(&jobs[t]);
            th[t] = 0;
        }
    }
    for (int t = 0; t < n_threads; ++t)
        if (th[t])
            pthread_join(th[t], NULL);
    /* pairwise merges: after round r, runs of 2^(r+1) original runs are sorted */
    for (int width = 1; width < n_threads; width *= 2) {
        int n_jobs = 0;
        for (int t = 0; t + width < n_threads; t += 2 * width) {
            int hi = t + 2 * width < n_threads ? t + 2 * width : n_threads;
            jobs[n_jobs] = (struct sort_job){order, tmp, bound[t], bound[t + width], bound[hi], w};
            if (pthread_create(&th[n_jobs], NULL, merge_job, &jobs[n_jobs]) != 0) {
                merge_job(&jobs[n_jobs]);
                th[n_jobs] = 0;
            }
            ++n_jobs;
        }
        for (int k = 0; k < n_jobs; ++k)
            if (th[k])
                pthread_join(th[k], NULL);
    }
    free(tmp);
    return status;
}

/*
 * Dendrogram of one tree with n_edges edges and n_edges + 1 vertices.
 * u, v: endpoints in [0, n_edges]; w: weights; all arrays host memory owned
 * by the caller.  Returns 0 or an error code; on error the outputs are
 * unspecified.
 */
static int dendrogram_impl(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                           int32_t *edge_parent, int32_t *vertex_parent, int n_threads);

int oracle_dendrogram(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                      int32_t *edge_parent, int32_t *vertex_parent)
{
    return dendrogram_impl(u, v, w, n_edges, edge_parent, vertex_parent, 1);
}

/* The same dendrogram with the sort on n_threads threads (timing mode). */
int oracle_dendrogram_threads(const int32_t *u, const int32_t *v, const float *w,
                              int64_t n_edges, int32_t *edge_parent, int32_t *vertex_parent,
                              int n_threads)
{
    return dendrogram_impl(u, v, w, n_edges, edge_parent, vertex_parent, n_threads);
}

static int dendrogram_impl(const int32_t *u, const int32_t *v, const float *w, int64_t n_edges,
                           int32_t *edge_parent, int32_t *vertex_parent, int n_threads)
{
    if (n_edges < 0 || n_edges >= INT32_MAX || !vertex_parent)
        return ORACLE_ERR_INVALID_ARGUMENT;
    if (n_edges > 0 && (!u || !v || !w || !edge_parent))
        return ORACLE_ERR_INVALID_ARGUMENT;
    int64_t n = n_edges + 1;
    if (n_edges == 0) {
        vertex_parent[0] = -1;
        return ORACLE_OK;
    }
    for (int64_t e = 0; e < n_edges; ++e) {
        if (isnan(w[e]))
            return ORACLE_ERR_NAN_WEIGHT;
    }
    for (int64_t e = 0; e < n_edges; ++e) {
        if (u[e] < 0 || u[e] >= n || v[e] < 0 || v[e] >= n)
            return ORACLE_ERR_VERTEX_OUT_OF_RANGE;
    }
    for (int64_t e = 0; e < n_edges; ++e) {
        if (u[e] == v[e])
            return ORACLE_ERR_SELF_LOOP;
    }

    int32_t *order = (int32_t *)malloc((size_t)n_edges * sizeof(int32_t));
    int32_t *uf = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *size = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    /* top[c] >= 0: vertex top[c]; top[c] < 0: edge ~top[c] */
    int32_t *top = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int status = ORACLE_OK;
    if (!order || !uf || !size || !top) {
        status = ORACLE_ERR_OUT_OF_MEMORY;
        goto done;
    }
    status = oracle_edge_order_threads(w, n_edges, order, n_threads);
    if (status != ORACLE_OK)
        goto done;

    for (int64_t x = 0; x < n; ++x) {
        uf[x] = (int32_t)x;
        size[x] = 1;
        top[x] = (int32_t)x;
    }
    for (int64_t k = 0; k < n_edges; ++k) {
        int32_t e = order[k];
        int32_t a = find_root(uf, u[e]);
        int32_t b = find_root(uf, v[e]);
        if (a == b) {
            status = ORACLE_ERR_NOT_A_TREE;
            goto done;
        }
        int32_t tops[2] = {top[a], top[b]};
        for (int s = 0; s < 2; ++s) {
            if (tops[s] >= 0)
                vertex_parent[tops[s]] = e;
            else
                edge_parent[~tops[s]] = e;
        }
        /* union by size; the surviving root carries the new top node */
        if (size[a] < size[b]) {
            int32_t t = a;
            a = b;
            b = t;
        }
        uf[b] = a;
        size[a] += size[b];
        top[a] = ~e;
    }
    edge_parent[order[n_edges - 1]] = -1;

done:
    free(order);
    free(uf);
    free(size);
    free(top);
    return status;
}

/*
 * Many independent trees.  Tree t owns edges [edge_offsets[t],
 * edge_offsets[t+1]) and vertices [edge_offsets[t] + t, edge_offsets[t+1] + t
 * + 1); endpoint ids and outputs are local to the tree.  Returns 0 or the
 * first error code (with the failing tree in *bad_tree when not NULL).
 */
int oracle_dendrogram_batched(const int32_t *u, const int32_t *v, const float *w,
                              const int64_t *edge_offsets, int64_t n_trees,
                              int32_t *edge_parent, int32_t *vertex_parent, int64_t *bad_tree)
{
    if (n_trees < 0 || !edge_offsets)
        return ORACLE_ERR_INVALID_ARGUMENT;
    for (int64_t t = 0; t < n_trees; ++t) {
        int64_t e0 = edge_offsets[t];
        int64_t e1 = edge_offsets[t + 1];
        if (e1 < e0)
            return ORACLE_ERR_INVALID_ARGUMENT;
        int st = oracle_dendrogram(u + e0, v + e0, w + e0, e1 - e0, edge_parent + e0,
                                   vertex_parent + e0 + t);
        if (st != ORACLE_OK) {
            if (bad_tree)
                *bad_tree = t;
            return st;
        }
    }
    return ORACLE_OK;
}

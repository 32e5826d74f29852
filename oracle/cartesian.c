/*
 * Closed-form dendrogram of a path tree, used to pin the oracle at full size.
 *
 * TEST INFRASTRUCTURE ONLY (see kruskal.c).  Independent of both the oracle
 * and the CUDA path: it never sorts and never uses union-find.
 *
 * For a path p_0 - p_1 - ... - p_m with edge k joining p_k and p_{k+1},
 * Theorem 1 of the paper (the lowest common dendrogram ancestor of two edges
 * is the heaviest edge on the tree path between them) makes the edge
 * dendrogram the max-Cartesian tree of the edge sequence: the parent of edge
 * k is the lighter of the nearest heavier edge on its left and the nearest
 * heavier edge on its right.  The parent of vertex p_k is the lighter of the
 * path edges k-1 and k (Eq. 1).
 *
 * The order is the one of kruskal.c: weight, then -0.0 before +0.0, then the
 * caller index of the edge.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static int path_lighter(const float *wp, const int32_t *eid, int64_t a, int64_t b)
{
    float wa = wp[a];
    float wb = wp[b];
    if (wa < wb)
        return 1;
    if (wa > wb)
        return 0;
    int sa = signbit(wa) ? 1 : 0;
    int sb = signbit(wb) ? 1 : 0;
    if (sa != sb)
        return sa;
    return eid[a] < eid[b];
}

/*
 * wp[k], eid[k]: weight and caller index of the k-th edge along the path
 * (k = 0..m-1).  Outputs: edge_parent indexed by caller edge index (values:
 * caller edge indices or -1), vertex_parent_path[k] for the path vertex p_k
 * (k = 0..m).  Returns 0, or 7 when out of memory.
 */
int cartesian_path_dendrogram(const float *wp, const int32_t *eid, int64_t m,
                              int32_t *edge_parent, int32_t *vertex_parent_path)
{
    if (m == 0) {
        vertex_parent_path[0] = -1;
        return 0;
    }
    int64_t *stack = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int64_t *left = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!stack || !left) {
        free(stack);
        free(left);
        return 7;
    }
    int64_t top = 0;
    for (int64_t k = 0; k < m; ++k) {
        while (top > 0 && path_lighter(wp, eid, stack[top - 1], k))
            --top;
        left[k] = top > 0 ? stack[top - 1] : -1;
        stack[top++] = k;
    }
    top = 0;
    for (int64_t k = m - 1; k >= 0; --k) {
        while (top > 0 && path_lighter(wp, eid, stack[top - 1], k))
            --top;
        int64_t right = top > 0 ? stack[top - 1] : -1;
        stack[top++] = k;
        int64_t l = left[k];
        int64_t par;
        if (l < 0 && right < 0)
            par = -1;
        else if (l < 0)
            par = right;
        else if (right < 0)
            par = l;
        else
            par = path_lighter(wp, eid, l, right) ? l : right;
        edge_parent[eid[k]] = par < 0 ? -1 : eid[par];
    }
    for (int64_t k = 0; k <= m; ++k) {
        if (k == 0)
            vertex_parent_path[k] = eid[0];
        else if (k == m)
            vertex_parent_path[k] = eid[m - 1];
        else
            vertex_parent_path[k] = path_lighter(wp, eid, k - 1, k) ? eid[k - 1] : eid[k];
    }
    free(stack);
    free(left);
    return 0;
}

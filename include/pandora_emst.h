/*
 * pandora_emst.h - mutual-reachability minimum spanning tree of 3-D points
 * on the GPU: the step before the dendrogram in the HDBSCAN* pipeline of
 * PANDORA (arXiv 2401.06089, Section 6.5, where the spanning tree comes from
 * a Euclidean minimum spanning tree construction and feeds the dendrogram).
 *
 * Definition (minPts as in Section 6.5: the size of the neighbourhood of the
 * density estimate, the point itself counted):
 *   d2(a, b)  = ((dx*dx + dy*dy) + dz*dz), dx = a.x - b.x etc., every
 *               operation a float32 operation rounded to nearest, in that
 *               order (no fused multiply-add);
 *   core2(a)  = the min_pts-th smallest d2(a, p) over all points p,
 *               counting d2(a, a) = 0;
 *   mr2(a, b) = max(core2(a), core2(b), d2(a, b));
 *   edges are totally ordered by (mr2, smaller point id, larger point id),
 * and the result is the minimum spanning tree of the complete graph under
 * that strict total order, which is unique.  The weight reported for an edge
 * is the float32 square root of its mr2 (correctly rounded): the
 * mutual-reachability distance max(core(a), core(b), |a - b|).
 *
 * Arguments: points - device float32 [n_points][3] (x, y, z of point i at
 * 3i .. 3i + 2), owned by the caller; u, v - device int32 [n_points - 1]:
 * the endpoints of every tree edge (u < v), in an unspecified order; w -
 * device float32 [n_points - 1], the edge weights; core_sq - device float32
 * [n_points] receiving core2 of every point, or NULL.  The outputs can be
 * passed to pandora_dendrogram as they are.
 *
 * Limits: 1 <= min_pts <= min(n_points, PANDORA_EMST_MAX_MIN_PTS);
 * n_points <= PANDORA_EMST_MAX_POINTS.  Errors: PANDORA_ERR_INVALID_ARGUMENT
 * (null pointer, n_points < 1, min_pts out of range), PANDORA_ERR_SIZE_LIMIT
 * (too many points), PANDORA_ERR_BAD_POINT (a coordinate is NaN or
 * infinite), PANDORA_ERR_OUT_OF_MEMORY, PANDORA_ERR_ITERATION_LIMIT (a bounded
 * device loop gave up: never expected), PANDORA_ERR_CUDA.  On an error the
 * outputs are unspecified.
 *
 * Blocking: returns when the tree is in u, v, w.  Scratch (about 160 bytes
 * per point) comes from the library's stream-ordered pool on `stream`.
 */
#ifndef PANDORA_EMST_H
#define PANDORA_EMST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PANDORA_EMST_MAX_MIN_PTS 32
#define PANDORA_EMST_MAX_POINTS (1 << 28)

int pandora_mr_emst(const float *points, int64_t n_points, int32_t min_pts, int32_t *u,
                    int32_t *v, float *w, float *core_sq, void *stream);

#ifdef __cplusplus
}
#endif

#endif

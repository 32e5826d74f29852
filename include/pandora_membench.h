/*
 * pandora_membench.h - random-access micro-benchmark of the device memory
 * system, the ceiling against which the dendrogram's level kernels are
 * measured.
 *
 * The paper has no counterpart: this is a measurement utility, not a step of
 * the method.  The contraction levels (Eq. 1, Eq. 2, Section 3.2) read and
 * update 4- and 8-byte words of vertex-indexed arrays at random positions;
 * such an access moves whole DRAM bursts, so the copy bandwidth of HBM is not
 * a ceiling any random-access kernel can reach.  One call launches ONE kernel
 * that performs `n_access` accesses of the chosen kind at positions drawn by
 * a counter-based hash (splitmix64 of `seed + i`), so no index array is read:
 * the kernel measures the random accesses alone.  The caller times the launch
 * (CUDA events on `stream`).
 *
 * Positions: with window >= n_elems (or window <= 0) every access picks a
 * uniform position in [0, n_elems).  With a smaller window the accesses sweep
 * the array window by window in order (access i falls in window
 * i / ceil(n_access / n_windows)), uniform inside the window: the access
 * pattern of a bucketed pass whose bucket fits in L2.
 *
 * Arguments: buf - device array of n_elems elements of the kind's width
 * (4 or 8 bytes), owned by the caller; written by the scatter and atomic
 * kinds.  dst - device array of n_elems 4-byte elements, written by
 * PANDORA_MB_COPY32 only (which reads buf sequentially), else may be NULL.
 * sink - one device 4-byte word the gather kinds may write (keeps their loads
 * alive).  blocks_per_sm - grid size in blocks of 256 threads per SM (1..32).
 *
 * Errors: PANDORA_ERR_INVALID_ARGUMENT for a null buffer, n_elems < 1,
 * n_access < 0, an unknown kind or blocks_per_sm outside 1..32;
 * PANDORA_ERR_CUDA if the launch fails.  Asynchronous: returns after the
 * launch is enqueued.
 */
#ifndef PANDORA_MEMBENCH_H
#define PANDORA_MEMBENCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum pandora_membench_kind {
    PANDORA_MB_GATHER32 = 0,    /* acc ^= buf32[pos]                       */
    PANDORA_MB_GATHER64 = 1,    /* acc ^= buf64[pos]                       */
    PANDORA_MB_SCATTER32 = 2,   /* buf32[pos] = i                          */
    PANDORA_MB_SCATTER64 = 3,   /* buf64[pos] = i                          */
    PANDORA_MB_ATOMICMIN64 = 4, /* atomicMin(buf64 + pos, hash)            */
    PANDORA_MB_COPY32 = 5       /* dst[i] = buf32[i], i < n_elems (sequential) */
};

int pandora_membench(int kind, void *buf, void *dst, void *sink, int64_t n_elems,
                     int64_t n_access, int64_t window, uint64_t seed, int blocks_per_sm,
                     void *stream);

#ifdef __cplusplus
}
#endif

#endif

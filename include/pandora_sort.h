/*
 * pandora_sort.h - the library's stable LSD radix sort of (key, value) pairs.
 *
 * The dendrogram sorts twice: the edges by weight with ties broken by edge
 * index (Section 3.1, "Dendrogram chains and skewness"), and the edges by
 * chain key, ties in rank order, before linking every chain (Section 3.3.3,
 * "Final dendrogram construction").  Both are the same single-pass-per-digit
 * (onesweep) radix sort; this entry point runs its key-value form on a
 * caller's pairs so that the sort can be checked on its own, for every digit
 * plan it uses (three passes of 8 or 9 bits for keys of 25 to 27 bits, the
 * chain keys of 8.4 to 67 million edges; 8-bit digits otherwise).
 *
 * pandora_sort_pairs: keys_out, vals_out = the n pairs (keys_in[i],
 * vals_in[i]) ordered by key; pairs with equal keys keep their input order
 * (stable).  Every key must be below 2^key_bits (1 <= key_bits <= 32): the
 * sort looks at those bits only, and a key with a higher bit set is
 * reported.  All arrays are device arrays of n 4-byte elements owned by the
 * caller; keys_out and vals_out must not overlap the inputs or each other.
 * workspace: device memory of at least pandora_sort_pairs_workspace_size(n,
 * key_bits) bytes, owned by the caller, 16-byte aligned.  The call enqueues
 * its kernels on `stream` (a cudaStream_t; NULL = the legacy default stream),
 * then synchronises the stream and returns the status: PANDORA_OK,
 * PANDORA_ERR_INVALID_ARGUMENT (a null pointer with n > 0, n < 0, n above
 * 2^31 - 1, key_bits outside 1..32, or a key at or above 2^key_bits: the
 * outputs are then unspecified), PANDORA_ERR_WORKSPACE_TOO_SMALL,
 * PANDORA_ERR_ITERATION_LIMIT (a bounded wait gave up; outputs unspecified)
 * or PANDORA_ERR_CUDA.  n == 0 returns PANDORA_OK at once.
 *
 * pandora_sort_pairs_workspace_size: bytes of workspace for n pairs and
 * key_bits; PANDORA_ERR_INVALID_ARGUMENT for n < 0, key_bits outside 1..32
 * or a null result pointer.
 */
#ifndef PANDORA_SORT_H
#define PANDORA_SORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int pandora_sort_pairs_workspace_size(int64_t n, int32_t key_bits, size_t *bytes);

int pandora_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, int64_t n,
                       int32_t key_bits, uint32_t *keys_out, uint32_t *vals_out,
                       void *workspace, size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif

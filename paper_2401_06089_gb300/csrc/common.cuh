// Device-side building blocks shared by the kernels of the dendrogram path.
//
// Written for sm_103a (GB300): 32-lane warps, 152 SMs, 126 MB L2.  Nothing in
// this path is a dense contraction, so nothing here touches the tensor cores;
// every kernel is bound by HBM bandwidth or by L2 latency of random accesses.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pandora.h"

namespace pandora {

using u32 = uint32_t;
using u64 = uint64_t;
using i32 = int32_t;
using i64 = int64_t;

constexpr u32 NONE = 0xFFFFFFFFu;          // "no edge" in minI / chain keys
constexpr int MAX_LEVELS = PANDORA_MAX_LEVELS;
constexpr u32 SPIN_LIMIT = 1u << 22;       // bound of every device-side wait loop

// ---- control block kept at the start of the workspace ----------------------
struct Ctrl {
    int status;               // first device-detected error (pandora_status)
    int pad0;
    u64 count_roots;          // supervertices of the next level
    u64 count_alpha;          // alpha-edges = edges of the next level
    u32 tile_counter[16];     // dynamic tile ids of single-pass kernels
    u32 hist1[4][256];        // digit histograms of the (weight, index) sort
    u32 hist2[4][256];        // digit histograms of the chain-key sort
};

__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// Order-preserving map of an fp32 weight to an unsigned key: unsigned order
// of keys equals IEEE order of non-NaN weights with -0.0 below +0.0.
__device__ __forceinline__ u32 weight_key(float w)
{
    u32 b = __float_as_uint(w);
    return b ^ ((b & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u);
}

__device__ __forceinline__ u32 lanemask_lt()
{
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ u64 ld_relaxed(const u64 *p)
{
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(u64 *p, u64 v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int *p)
{
    return *(const volatile int *)p;
}

__device__ __forceinline__ void st_volatile(int *p, int v)
{
    *(volatile int *)p = v;
}

// Look-back status words: [flag:2 | value:62]; flag 1 = tile aggregate only,
// flag 2 = inclusive prefix through this tile.
constexpr u64 LB_AGG = 1ull << 62;
constexpr u64 LB_INC = 2ull << 62;
constexpr u64 LB_VAL = (1ull << 62) - 1;

// Decoupled look-back for one counter (Merrill & Garland).  Called by ONE
// thread of the block; returns the exclusive prefix of `aggregate` over all
// earlier tiles.  Waits are bounded: on timeout the status word records
// PANDORA_ERR_ITERATION_LIMIT and the partial prefix is returned.
__device__ __forceinline__ u64 lookback_exclusive(u64 *lb, u32 tile, u64 aggregate, int *status)
{
    if (tile == 0) {
        st_relaxed(lb, LB_INC | aggregate);
        return 0;
    }
    st_relaxed(lb + tile, LB_AGG | aggregate);
    u64 excl = 0;
    i64 j = (i64)tile - 1;
    u32 spins = 0;
    while (j >= 0) {
        u64 s = ld_relaxed(lb + j);
        u64 f = s & ~LB_VAL;
        if (f == 0) {
            if (++spins > SPIN_LIMIT) {
                set_status(status, PANDORA_ERR_ITERATION_LIMIT);
                break;
            }
            if (spins > 64)
                __nanosleep(64);
            continue;
        }
        excl += s & LB_VAL;
        if (f == LB_INC)
            break;
        --j;
    }
    st_relaxed(lb + tile, LB_INC | (excl + aggregate));
    return excl;
}

// Tree id of a global edge index in forest mode (binary search of the
// per-tree edge offsets, t such that off[t] <= e < off[t+1]).
__device__ __forceinline__ i64 tree_of_edge(const i64 *__restrict__ off, i64 n_trees, i64 e)
{
    i64 lo = 0, hi = n_trees - 1;
    while (lo < hi) {
        i64 mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= e)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace pandora

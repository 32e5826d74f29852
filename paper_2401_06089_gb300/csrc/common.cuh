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
constexpr int MARK_MAX_BUCKETS = 512;

struct Ctrl {
    int status;                    // first device-detected error (pandora_status)
    int n_levels;                  // contraction levels run; set by the level that
                                   // has no alpha-edge (0 while the loop runs)
    u64 lvl_m[MAX_LEVELS + 1];     // edges of level l (device truth)
    u64 lvl_n[MAX_LEVELS + 1];     // vertices of level l
    u64 n_deep;                    // vertices left to union-find by the bounded walk
    u32 tile_counter[16];          // dynamic tile ids of single-pass kernels
    u32 hist1[4][256];             // digit histograms of the (weight, index) sort
    u32 base1[4][256];             // their exclusive scans (bucket starts)
    u32 hist2[4096];               // digit histograms of the chain-key sort, rows of its digit plan
    u32 base2[4096];               // their exclusive scans
    // bucketed marking (levels with many vertices): incidences per vertex
    // bucket, write cursors, bucket starts
    u32 mark_count[MARK_MAX_BUCKETS];
    u32 mark_cursor[MARK_MAX_BUCKETS];
    u64 mark_base[MARK_MAX_BUCKETS + 1];
    // bucketed link: write cursors of the caller-id buckets
    u32 link_cursor[MARK_MAX_BUCKETS];
};

// Element count produced on the device, clamped to the buffer capacity the
// host sized the launch for (a larger count only arises from invalid input,
// which the producing kernel reports).
__device__ __forceinline__ i64 dev_count(const u64 *d, i64 cap)
{
    const u64 c = *(const volatile u64 *)d;
    return c > (u64)cap ? cap : (i64)c;
}

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
// earlier tiles.  Waits are bounded: a wait longer than `report` spins
// records PANDORA_ERR_ITERATION_LIMIT and goes on (pandora_set_wait_report_limit
// lowers `report` so that tests can see the status without cutting a wait
// short); after SPIN_LIMIT spins the status is recorded and the partial
// prefix is returned, which can only move this tile's outputs to lower,
// still valid positions.
__device__ __forceinline__ u64 lookback_exclusive(u64 *lb, u32 tile, u64 aggregate, int *status,
                                                  u32 report = SPIN_LIMIT)
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
            ++spins;
            if (spins == report + 1u)
                set_status(status, PANDORA_ERR_ITERATION_LIMIT);
            if (spins > SPIN_LIMIT) {
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

// ---- TMA bulk copies (cp.async.bulk) completed on an mbarrier ---------------
__device__ __forceinline__ u32 smem_u32(const void *p)
{
    return (u32)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(u64 *bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u64 *bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned); completion is counted on `bar`
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, u32 bytes, u64 *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`.  On timeout the status word
// records PANDORA_ERR_ITERATION_LIMIT and the wait goes on, bounded again,
// so that the block never leaves while its own copies are still landing in
// its shared memory; returns false if both bounds ran out (the status then
// already says so, and the call's outputs are unspecified).
__device__ __forceinline__ bool mbar_wait_bounded(u64 *bar, u32 parity, int *status)
{
    for (u32 i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    set_status(status, PANDORA_ERR_ITERATION_LIMIT);
    for (u32 i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
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

// Tree id of a level-0 vertex in forest mode: tree t owns the vertices
// [off[t] + t, off[t+1] + t + 1).
__device__ __forceinline__ i64 tree_of_vertex(const i64 *__restrict__ off, i64 n_trees, i64 x)
{
    i64 lo = 0, hi = n_trees - 1;
    while (lo < hi) {
        i64 mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) + mid <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace pandora

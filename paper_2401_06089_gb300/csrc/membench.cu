// Random-access micro-benchmark (include/pandora_membench.h): one kernel per
// call, positions from a counter-based hash, so that the measured time is the
// random accesses alone.  Used to state the ceiling of the level kernels,
// whose random 4- and 8-byte accesses move whole DRAM bursts.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pandora.h"
#include "../../include/pandora_membench.h"

namespace {

using u32 = uint32_t;
using u64 = uint64_t;
using i64 = int64_t;

constexpr int MB_UNROLL = 8;

// splitmix64 finaliser (Steele, Lea and Flood), a bijection of 64-bit words
__device__ __forceinline__ u64 splitmix64(u64 x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

struct Pos {
    i64 n, window, n_windows, per_window;
    u64 seed;
    // position of access i: inside [0, n) by construction (a window's span
    // is clamped to the array's end)
    __device__ __forceinline__ i64 at(i64 i, u64 *h_out) const
    {
        const u64 h = splitmix64(seed + (u64)i);
        *h_out = h;
        if (n_windows <= 1)
            return (i64)__umul64hi(h, (u64)n);
        i64 wi = i / per_window;
        if (wi >= n_windows)
            wi = n_windows - 1;
        const i64 lo = wi * window;
        const i64 span = (n - lo) < window ? (n - lo) : window;
        return lo + (i64)__umul64hi(h, (u64)span);
    }
};

template <int KIND>
__global__ void __launch_bounds__(256) membench_kernel(void *buf, u32 *dst, u32 *sink, Pos p,
                                                       i64 n_access)
{
    if (KIND == PANDORA_MB_COPY32) {
        for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
             i += (i64)gridDim.x * blockDim.x)
            dst[i] = ((const u32 *)buf)[i];
        return;
    }
    const i64 stride = (i64)gridDim.x * blockDim.x * MB_UNROLL;
    u64 acc = 0;
    for (i64 base = ((i64)blockIdx.x * blockDim.x + threadIdx.x) * MB_UNROLL; base < n_access;
         base += stride) {
        i64 pos[MB_UNROLL];
        u64 h[MB_UNROLL];
#pragma unroll
        for (int k = 0; k < MB_UNROLL; ++k)
            pos[k] = base + k < n_access ? p.at(base + k, &h[k]) : -1;
        if (KIND == PANDORA_MB_GATHER32 || KIND == PANDORA_MB_GATHER64) {
            u64 v[MB_UNROLL];
#pragma unroll
            for (int k = 0; k < MB_UNROLL; ++k)
                v[k] = pos[k] < 0 ? 0
                       : KIND == PANDORA_MB_GATHER32 ? (u64)((const u32 *)buf)[pos[k]]
                                                     : ((const u64 *)buf)[pos[k]];
#pragma unroll
            for (int k = 0; k < MB_UNROLL; ++k)
                acc ^= v[k];
        } else {
#pragma unroll
            for (int k = 0; k < MB_UNROLL; ++k) {
                if (pos[k] < 0)
                    continue;
                if (KIND == PANDORA_MB_SCATTER32)
                    ((u32 *)buf)[pos[k]] = (u32)(base + k);
                else if (KIND == PANDORA_MB_SCATTER64)
                    ((u64 *)buf)[pos[k]] = (u64)(base + k);
                else
                    atomicMin((unsigned long long *)buf + pos[k], (unsigned long long)h[k]);
            }
        }
    }
    // an improbable value that both halves can reach: the loads cannot be
    // dropped, and the store practically never happens
    const u32 folded = (u32)acc ^ (u32)(acc >> 32);
    if (folded == 0x9E3779B9u)
        *sink = folded;
}

template <int KIND>
cudaError_t launch(unsigned blocks, cudaStream_t s, void *buf, u32 *dst, u32 *sink, const Pos &p,
                   i64 n_access)
{
    membench_kernel<KIND><<<blocks, 256, 0, s>>>(buf, dst, sink, p, n_access);
    return cudaGetLastError();
}

}  // namespace

extern "C" int pandora_membench(int kind, void *buf, void *dst, void *sink, int64_t n_elems,
                                int64_t n_access, int64_t window, uint64_t seed,
                                int blocks_per_sm, void *stream)
{
    if (!buf || !sink || n_elems < 1 || n_access < 0 || blocks_per_sm < 1 || blocks_per_sm > 32 ||
        kind < PANDORA_MB_GATHER32 || kind > PANDORA_MB_COPY32)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (kind == PANDORA_MB_COPY32 && !dst)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (kind == PANDORA_MB_COPY32)
        n_access = n_elems;
    if (n_access == 0)
        return PANDORA_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    Pos p{};
    p.n = n_elems;
    p.seed = seed;
    p.window = (window <= 0 || window >= n_elems) ? n_elems : window;
    p.n_windows = (n_elems + p.window - 1) / p.window;
    p.per_window = (n_access + p.n_windows - 1) / p.n_windows;
    const i64 per_block = (i64)256 * MB_UNROLL;
    i64 blocks = (n_access + per_block - 1) / per_block;
    const i64 cap = (i64)sms * blocks_per_sm;
    if (blocks > cap)
        blocks = cap;
    cudaStream_t s = (cudaStream_t)stream;
    u32 *d = (u32 *)dst, *k = (u32 *)sink;
    cudaError_t e = cudaSuccess;
    switch (kind) {
    case PANDORA_MB_GATHER32: e = launch<PANDORA_MB_GATHER32>((unsigned)blocks, s, buf, d, k, p, n_access); break;
    case PANDORA_MB_GATHER64: e = launch<PANDORA_MB_GATHER64>((unsigned)blocks, s, buf, d, k, p, n_access); break;
    case PANDORA_MB_SCATTER32: e = launch<PANDORA_MB_SCATTER32>((unsigned)blocks, s, buf, d, k, p, n_access); break;
    case PANDORA_MB_SCATTER64: e = launch<PANDORA_MB_SCATTER64>((unsigned)blocks, s, buf, d, k, p, n_access); break;
    case PANDORA_MB_ATOMICMIN64: e = launch<PANDORA_MB_ATOMICMIN64>((unsigned)blocks, s, buf, d, k, p, n_access); break;
    default: e = launch<PANDORA_MB_COPY32>((unsigned)blocks, s, buf, d, k, p, n_access); break;
    }
    return e == cudaSuccess ? PANDORA_OK : PANDORA_ERR_CUDA;
}

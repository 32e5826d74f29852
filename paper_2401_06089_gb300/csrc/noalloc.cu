// Allocation-free entry point pandora_dendrogram_noalloc (include/pandora.h).
//
// For callers that cannot allocate device memory when they call us (their
// GPU memory belongs to another allocator, or cudaMalloc/cudaFree would
// stall a latency-critical loop), the whole dendrogram pipeline runs on a
// fixed scratch array that is part of the library's device image.  The
// array is 32 MiB on every GPU that loads the library, which bounds the
// input at PANDORA_NOALLOC_MAX_EDGES edges.
#include <mutex>

#include "kernels.cuh"

namespace pandora {
int run_on_workspace(const i32 *u, const i32 *v, const float *w, i64 M, i32 *ep, i32 *vp,
                     void *ws, size_t ws_bytes, cudaStream_t s);
size_t workspace_bytes(i64 M, i64 T);
}  // namespace pandora

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; host code must not use this name as an
// address (it is a host-side stand-in): the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device with that device current.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return PANDORA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PANDORA_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PANDORA_OK;
}

}  // namespace

extern "C" int pandora_dendrogram_noalloc(const int32_t *u, const int32_t *v, const float *w,
                                          int64_t n_edges, int32_t *edge_parent,
                                          int32_t *vertex_parent, void *stream)
{
    using namespace pandora;
    if (n_edges < 0 || !vertex_parent || (n_edges > 0 && (!u || !v || !w || !edge_parent)))
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (n_edges > PANDORA_NOALLOC_MAX_EDGES)
        return PANDORA_ERR_SIZE_LIMIT;
    const size_t need = workspace_bytes(n_edges, 1);
    if (need > kScratchBytes)
        return PANDORA_ERR_SIZE_LIMIT;
    void *ws = nullptr;
    if (int e = scratch_address(&ws))
        return e;
    // The pipeline zeroes its control block, look-back words and counters
    // itself at the start of every call, so stale contents left by an
    // earlier call are never read.
    return run_on_workspace(u, v, w, n_edges, edge_parent, vertex_parent, ws, kScratchBytes,
                            (cudaStream_t)stream);
}

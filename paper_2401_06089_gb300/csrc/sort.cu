// Onesweep LSD radix sort of (key, value...) tuples for sm_103a.
//
// Paper step: the edges are sorted by weight with a consistent tie rule
// (Section 3.1); the chains are sorted again after expansion (Section 3.3.3).
// Both sorts are stable LSD radix sorts over 8-bit digits, so equal keys keep
// their input order: for the weight sort the first value stream is the
// caller edge index and ties therefore resolve by index; for the chain sort
// the input is in ascending rank, so every chain comes out in ascending rank.
//
// One pass = one kernel (Adinets & Merrill's onesweep): a block takes the
// next tile id from an atomic counter, ranks its keys by digit with warp
// ballots (stable: warp w of the tile owns a contiguous run of keys, taken 32
// at a time in order), publishes its per-digit counts and sums the counts of
// all earlier tiles by decoupled look-back (eight predecessor tiles per
// round trip), then scatters keys and each value stream through shared
// memory so that every digit's run is written contiguously.  The per-pass
// digit totals come from one histogram read of all keys before the first
// pass.
//
// The weight sort carries the endpoints (u, v) as two extra value streams:
// moving 8 more bytes per edge through each pass is cheaper than gathering
// them at random afterwards (a random 4-byte read costs a 64-byte DRAM
// burst).
#include "kernels.cuh"

namespace pandora {

namespace {

constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int LB_BATCH = 8;
static_assert(OS_THREADS >= RADIX, "one thread per digit");

// Exclusive scan of one value per thread over the first 256 threads of the
// block (all threads must call; threads >= 256 pass 0 and get garbage).
__device__ __forceinline__ u32 digit_exclusive_scan(u32 x, u32 *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off)
            incl += y;
    }
    if (lane == 31 && warp < RADIX / 32)
        s_warp[warp] = incl;
    __syncthreads();
    u32 prefix = 0;
#pragma unroll
    for (int k = 0; k < RADIX / 32; ++k)
        prefix += (k < warp) ? s_warp[k] : 0u;
    __syncthreads();
    return prefix + incl - x;
}

__global__ void __launch_bounds__(256) hist_weights_kernel(const float *__restrict__ w, i64 n,
                                                           u32 *__restrict__ hist, int *status)
{
    __shared__ u32 s_h[4 * RADIX];
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x)
        s_h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    // every lane runs the same number of iterations so that warp votes are full
    const i64 n_round = (n + 31) & ~(i64)31;
    bool nan_seen = false;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - lane < n_round; i += stride) {
        const bool valid = i < n;
        float x = valid ? w[i] : 0.0f;
        nan_seen |= (x != x);
        u32 k = weight_key(x);
        u32 k0 = __shfl_sync(0xFFFFFFFFu, k, 0);
        u32 vm = __ballot_sync(0xFFFFFFFFu, valid);
        bool uniform = __all_sync(0xFFFFFFFFu, k == k0) && vm == 0xFFFFFFFFu;
        if (uniform) {
            if (lane == 0) {
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    atomicAdd(&s_h[p * RADIX + ((k >> (8 * p)) & 255)], 32u);
            }
        } else if (valid) {
#pragma unroll
            for (int p = 0; p < 4; ++p)
                atomicAdd(&s_h[p * RADIX + ((k >> (8 * p)) & 255)], 1u);
        }
    }
    if (nan_seen)
        set_status(status, PANDORA_ERR_NAN_WEIGHT);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) {
        u32 c = s_h[i];
        if (c)
            atomicAdd(hist + i, c);
    }
}

template <int FLAGS>
__global__ void __launch_bounds__(OS_THREADS, OS_MIN_BLOCKS) onesweep_kernel(const OnesweepParams p)
{
    constexpr bool kAB = (FLAGS & OS_LAST_AB) != 0;
    constexpr bool kUV = (FLAGS & OS_PAYLOAD_UV) != 0;
    __shared__ u32 s_whist[OS_WARPS][RADIX];   // per-warp digit counts, then offsets
    __shared__ u32 s_buf[OS_TILE];             // tile in digit order (keys, then values)
    __shared__ u32 s_buf2[kUV ? OS_TILE : 1];  // v beside u
    __shared__ u32 s_goff[RADIX];              // global position of local position 0, per digit
    __shared__ unsigned char s_dig[OS_TILE];   // digit of each local position
    __shared__ u32 s_local_start[RADIX];
    __shared__ u32 s_warp[RADIX / 32];
    __shared__ u32 s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < OS_WARPS * RADIX; i += OS_THREADS)
        (&s_whist[0][0])[i] = 0;
    if (tid == 0)
        s_tile = atomicAdd(p.tile_counter, 1u);
    // global start of every digit's bucket (exclusive scan of the pass histogram)
    const u32 bin_base = digit_exclusive_scan(tid < RADIX ? p.hist[tid] : 0u, s_warp);
    const u32 tile = s_tile;   // published before the scan's barriers
    const i64 tile_base = (i64)tile * OS_TILE;
    const i64 warp_base = tile_base + (i64)warp * (32 * OS_ITEMS);
    const int shift = p.shift;

    u32 reg[OS_ITEMS];     // keys, later values
    u32 lpos[OS_ITEMS];    // rank within warp and digit, later local position
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        if (idx < p.n)
            reg[it] = (FLAGS & OS_KEY_FROM_W) ? weight_key(p.w_in[idx]) : p.keys_in[idx];
        else
            reg[it] = 0;
    }

    // ---- stable warp-level ranking by digit (ballot multisplit) ------------
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        const bool valid = idx < p.n;
        const u32 d = (reg[it] >> shift) & 255u;
        u32 peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const u32 bit = (d >> b) & 1u;
            const u32 bal = __ballot_sync(0xFFFFFFFFu, bit);
            peers &= bit ? bal : ~bal;
        }
        const int leader = valid ? (__ffs(peers) - 1) : lane;
        u32 base = 0;
        if (valid && lane == leader) {
            base = s_whist[warp][d];
            s_whist[warp][d] = base + __popc(peers);
        }
        __syncwarp();
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        lpos[it] = base + __popc(peers & lt);
    }
    __syncthreads();

    // ---- per-digit totals of the tile; publish for look-back ---------------
    u32 total = 0;
    u64 *lbt = p.lb + (u64)tile * RADIX;
    if (tid < RADIX) {
#pragma unroll
        for (int k = 0; k < OS_WARPS; ++k) {
            const u32 c = s_whist[k][tid];
            s_whist[k][tid] = total;
            total += c;
        }
        st_relaxed(lbt + tid, (tile == 0 ? LB_INC : LB_AGG) | (u64)total);
    }
    const u32 local_start = digit_exclusive_scan(total, s_warp);
    if (tid < RADIX)
        s_local_start[tid] = local_start;
    __syncthreads();

    // ---- keys into shared memory in digit order ----------------------------
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        if (idx < p.n) {
            const u32 d = (reg[it] >> shift) & 255u;
            const u32 pos = s_local_start[d] + s_whist[warp][d] + lpos[it];
            s_buf[pos] = reg[it];
            lpos[it] = pos;
        }
    }

    // ---- decoupled look-back, one thread per digit, 8 tiles per round trip --
    if (tid < RADIX) {
        u64 excl = 0;
        if (tile > 0) {
            i64 j = (i64)tile - 1;
            u32 spins = 0;
            for (;;) {
                u64 s[LB_BATCH];
#pragma unroll
                for (int k = 0; k < LB_BATCH; ++k)
                    s[k] = (j - k >= 0) ? ld_relaxed(p.lb + (u64)(j - k) * RADIX + tid) : LB_INC;
                int consumed = 0;
                bool done = false;
#pragma unroll
                for (int k = 0; k < LB_BATCH; ++k) {
                    if (done || consumed < k)
                        continue;
                    const u64 f = s[k] & ~LB_VAL;
                    if (f == 0)
                        continue;            // not published yet: reload from here
                    excl += s[k] & LB_VAL;
                    consumed = k + 1;
                    if (f == LB_INC)
                        done = true;
                }
                if (done)
                    break;
                j -= consumed;
                if (consumed == 0) {
                    if (++spins > SPIN_LIMIT) {
                        set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
                        break;
                    }
                    if (spins > 16)
                        __nanosleep(32);
                }
            }
            st_relaxed(lbt + tid, LB_INC | (excl + total));
        }
        s_goff[tid] = bin_base + (u32)excl - local_start;   // modulo 2^32
    }
    __syncthreads();

    // ---- write keys, one digit run after another ---------------------------
    const i64 rem = p.n - tile_base;
    const int tile_count = rem < OS_TILE ? (int)rem : OS_TILE;
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
        const int j = k * OS_THREADS + tid;
        if (j < tile_count) {
            const u32 key = s_buf[j];
            const u32 d = (key >> shift) & 255u;
            s_dig[j] = (unsigned char)d;
            if (FLAGS & OS_WRITE_KEYS)
                p.keys_out[s_goff[d] + (u32)j] = key;
        }
    }

    // ---- value stream 0: caller edge index --------------------------------------
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        reg[it] = idx < p.n ? ((FLAGS & OS_GEN_VALS) ? (u32)idx : p.vals_in[idx]) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        if (idx < p.n)
            s_buf[lpos[it]] = reg[it];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
        const int j = k * OS_THREADS + tid;
        if (j < tile_count)
            p.vals_out[s_goff[s_dig[j]] + (u32)j] = s_buf[j];
    }

    // ---- value streams 1, 2: endpoints u, v -----------------------------------
    if (FLAGS & OS_PAYLOAD_UV) {
        __syncthreads();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            u32 *dst = half == 0 ? s_buf : s_buf2;
#pragma unroll
            for (int it = 0; it < OS_ITEMS; ++it) {
                const i64 idx = warp_base + it * 32 + lane;
                if (idx < p.n) {
                    u32 x;
                    if (FLAGS & OS_GEN_VALS) {
                        // first pass: read the caller's endpoints, validate them and
                        // turn tree-local ids into forest ids
                        i32 a = p.u[idx], b = p.v[idx];
                        i64 nv = p.n_vertices, voff = 0;
                        if (FLAGS & OS_FOREST) {
                            const i64 t = tree_of_edge(p.edge_off, p.n_trees, idx);
                            const i64 e0 = __ldg(p.edge_off + t), e1 = __ldg(p.edge_off + t + 1);
                            nv = e1 - e0 + 1;
                            voff = e0 + t;
                        }
                        if (a < 0 || (i64)a >= nv || b < 0 || (i64)b >= nv) {
                            if (half == 0)
                                set_status(p.status, PANDORA_ERR_VERTEX_OUT_OF_RANGE);
                            a = 0;
                            b = 0;
                        } else if (a == b && half == 0) {
                            set_status(p.status, PANDORA_ERR_SELF_LOOP);
                        }
                        x = (u32)((half == 0 ? a : b) + voff);
                    } else {
                        x = half == 0 ? p.pu_in[idx] : p.pv_in[idx];
                    }
                    dst[lpos[it]] = x;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < OS_ITEMS; ++k) {
            const int j = k * OS_THREADS + tid;
            if (j < tile_count) {
                const u32 pos = s_goff[s_dig[j]] + (u32)j;
                if (kAB) {
                    p.ab_out[pos] = make_int2((i32)s_buf[j], (i32)s_buf2[j]);
                } else {
                    p.pu_out[pos] = s_buf[j];
                    p.pv_out[pos] = s_buf2[j];
                }
            }
        }
    }
}

}  // namespace

void launch_hist_weights(const float *w, i64 n, u32 *hist, int *status, cudaStream_t s)
{
    if (n <= 0)
        return;
    i64 blocks = (n + 256 * 16 - 1) / (256 * 16);
    if (blocks > 152 * 8)
        blocks = 152 * 8;
    hist_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(w, n, hist, status);
}

template <int F>
static void launch_os(const OnesweepParams &p, cudaStream_t s)
{
    const i64 tiles = onesweep_tiles(p.n);
    onesweep_kernel<F><<<(unsigned)tiles, OS_THREADS, 0, s>>>(p);
}

void launch_onesweep(int flags, const OnesweepParams &p, cudaStream_t s)
{
    if (p.n <= 0)
        return;
    constexpr int FIRST = OS_KEY_FROM_W | OS_GEN_VALS | OS_PAYLOAD_UV;
    switch (flags) {
    case FIRST | OS_WRITE_KEYS: launch_os<FIRST | OS_WRITE_KEYS>(p, s); break;
    case FIRST | OS_WRITE_KEYS | OS_FOREST: launch_os<FIRST | OS_WRITE_KEYS | OS_FOREST>(p, s); break;
    case FIRST | OS_LAST_AB: launch_os<FIRST | OS_LAST_AB>(p, s); break;
    case FIRST | OS_LAST_AB | OS_FOREST: launch_os<FIRST | OS_LAST_AB | OS_FOREST>(p, s); break;
    case OS_PAYLOAD_UV | OS_WRITE_KEYS: launch_os<OS_PAYLOAD_UV | OS_WRITE_KEYS>(p, s); break;
    case OS_PAYLOAD_UV | OS_LAST_AB: launch_os<OS_PAYLOAD_UV | OS_LAST_AB>(p, s); break;
    case OS_WRITE_KEYS: launch_os<OS_WRITE_KEYS>(p, s); break;
    default: break;
    }
}

}  // namespace pandora

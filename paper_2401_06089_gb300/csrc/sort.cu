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
// next tile id from an atomic counter and at once starts TMA bulk copies
// (cp.async.bulk, completed on mbarriers) of the tile's keys and of every
// value stream into shared memory; it ranks the keys by digit with warp
// ballots as soon as they land (stable: warp w of the tile owns a contiguous
// run of keys, taken 32 at a time in order), publishes its per-digit counts
// and sums the counts of all earlier tiles by decoupled look-back (eight
// predecessor tiles per round trip), then writes keys and each value stream
// through shared memory so that every digit's run is written contiguously.
// The value copies land while the block ranks and looks back, so no DRAM
// latency sits between the look-back and the value writes.  The per-pass
// digit totals come from one histogram read of all keys before the first
// pass.
//
// The weight sort carries the endpoints (u, v) as one extra 8-byte value
// stream (int2; the first pass pairs the caller's two arrays):
// moving 8 more bytes per edge through each pass is cheaper than gathering
// them at random afterwards (a random 4-byte read costs a 64-byte DRAM
// burst).
#include <atomic>
#include <type_traits>

#include "kernels.cuh"
#include "../../include/pandora_sort.h"

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

// Exclusive scan of RD digit counts held DPT consecutive digits per thread
// (thread t owns digits t*DPT .. t*DPT+DPT-1; threads past RD/DPT own none
// and must pass zeros).  All threads of the block must call.
template <int RD>
struct DigitsPerThread {
    static constexpr int value = RD > OS_THREADS ? RD / OS_THREADS : 1;
};

template <int RD>
__device__ __forceinline__ void digits_exclusive_scan(const u32 *x, u32 *out, u32 *s_warp)
{
    constexpr int DPT = DigitsPerThread<RD>::value;
    constexpr int ACTIVE_WARPS = RD / DPT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 sum = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k)
        sum += x[k];
    u32 incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off)
            incl += y;
    }
    if (lane == 31 && warp < ACTIVE_WARPS)
        s_warp[warp] = incl;
    __syncthreads();
    u32 run = 0;
#pragma unroll
    for (int k = 0; k < ACTIVE_WARPS; ++k)
        run += (k < warp) ? s_warp[k] : 0u;
    __syncthreads();
    run += incl - sum;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        out[k] = run;
        run += x[k];
    }
}

// Digit histograms of the weight keys for all four passes, in one read of the
// weights.  Each thread keeps 16 bytes of weights in flight per iteration
// (one float4 when the array is 16-byte aligned) so that enough loads are
// outstanding to stream at DRAM speed, and each warp counts into its own
// copy of the histograms.  Lanes with equal top digits are merged first
// (__match_any_sync): the top digit (sign and high exponent bits) of weights
// in a narrow range takes only a few values, and equal addresses in one
// shared-memory atomic serialise.
constexpr int HIST_WARPS = 8;
__device__ __forceinline__ void hist_count(u32 (*h)[4 * RADIX], int warp, u32 k, bool valid)
{
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (valid)
            atomicAdd(&h[warp][q * RADIX + ((k >> (8 * q)) & 255u)], 1u);
    const u32 d = valid ? k >> 24 : 256u;   // 256: no count
    const u32 peers = __match_any_sync(0xFFFFFFFFu, d);
    if (valid && (threadIdx.x & 31) == (u32)(__ffs(peers) - 1))
        atomicAdd(&h[warp][3 * RADIX + d], (u32)__popc(peers));
}

__global__ void __launch_bounds__(256) hist_weights_kernel(const float *__restrict__ w, i64 n,
                                                           u32 *__restrict__ hist, int *status)
{
    __shared__ u32 s_h[HIST_WARPS][4 * RADIX];
    for (int i = threadIdx.x; i < HIST_WARPS * 4 * RADIX; i += blockDim.x)
        (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    bool nan_seen = false;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    const i64 t0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if ((((uintptr_t)w) & 15) == 0) {
        const float4 *w4 = (const float4 *)w;
        const i64 n4 = n / 4;
        // every lane of a warp runs the same iterations (full warp votes)
        const i64 n4_round = (n4 + 31) & ~(i64)31;
        for (i64 i = t0; i - (threadIdx.x & 31) < n4_round; i += stride) {
            const bool valid = i < n4;
            const float4 x = valid ? w4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            nan_seen |= (x.x != x.x) | (x.y != x.y) | (x.z != x.z) | (x.w != x.w);
            hist_count(s_h, warp, weight_key(x.x), valid);
            hist_count(s_h, warp, weight_key(x.y), valid);
            hist_count(s_h, warp, weight_key(x.z), valid);
            hist_count(s_h, warp, weight_key(x.w), valid);
        }
        // the last n % 4 weights
        if (blockIdx.x == 0 && warp == 0) {
            const i64 i = n4 * 4 + (threadIdx.x & 31);
            const bool valid = i < n;
            const float x = valid ? w[i] : 0.f;
            nan_seen |= valid && (x != x);
            hist_count(s_h, warp, weight_key(x), valid);
        }
    } else {
        const i64 n_round = (n + 31) & ~(i64)31;
        for (i64 i = t0; i - (threadIdx.x & 31) < n_round; i += stride) {
            const bool valid = i < n;
            const float x = valid ? w[i] : 0.f;
            nan_seen |= (x != x);
            hist_count(s_h, warp, weight_key(x), valid);
        }
    }
    if (nan_seen)
        set_status(status, PANDORA_ERR_NAN_WEIGHT);
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) {
        u32 c = 0;
#pragma unroll
        for (int k = 0; k < HIST_WARPS; ++k)
            c += s_h[k][i];
        if (c)
            atomicAdd(hist + i, c);
    }
}

// Digit histograms of 32-bit keys for all four passes (one read of the keys).
__global__ void __launch_bounds__(256) hist_keys_kernel(const u32 *__restrict__ keys, i64 n,
                                                        u32 *__restrict__ hist)
{
    __shared__ u32 s_h[HIST_WARPS][4 * RADIX];
    for (int i = threadIdx.x; i < HIST_WARPS * 4 * RADIX; i += blockDim.x)
        (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    const i64 n_round = (n + 31) & ~(i64)31;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - (threadIdx.x & 31) < n_round;
         i += stride) {
        const bool valid = i < n;
        hist_count(s_h, warp, valid ? keys[i] : 0u, valid);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) {
        u32 c = 0;
#pragma unroll
        for (int k = 0; k < HIST_WARPS; ++k)
            c += s_h[k][i];
        if (c)
            atomicAdd(hist + i, c);
    }
}

// Dynamic shared memory of one onesweep block: the input streams of the tile
// as the TMA lands them (keys; values; u, v), one staging buffer for the
// digit-ordered output, per-warp digit counts and the digit of each output
// position.
// Blocks per SM: the variants that carry the endpoints need 100 KB of shared
// memory and fit two per SM; the others (68 KB) fit three, and are compiled
// for the registers of three.
//
// Digits are DBITS wide (8 or 9; RD = 2^DBITS buckets; the kernel is
// written for up to 10).  Wider digits take fewer passes over keys of 25 to
// 27 bits; they keep 16-bit
// per-warp counts (at most 32 * OS_ITEMS keys of a warp share a digit, and a
// tile's prefix is below OS_TILE) and read each output position's digit back
// from the digit-ordered keys instead of keeping a digit byte, so the chain
// sort's 9-bit variant fits three blocks per SM like the 8-bit one.  Only the
// key-value variant (no carried endpoints) comes in the wide forms.
template <int FLAGS, int DBITS>
struct OsSmem {
    static constexpr int RD = 1 << DBITS;
    static constexpr bool kWide = DBITS > 8;
    using WH = typename std::conditional<kWide, unsigned short, u32>::type;
    static constexpr bool kUV = (FLAGS & OS_PAYLOAD_UV) != 0;
    static_assert(!(kUV && kWide), "wide digits only for the key-value sort");
    static constexpr int kBufs = kUV ? 5 : 3;
    static constexpr size_t kBufBytes = (size_t)OS_TILE * 4;
    static constexpr size_t kWhist = (size_t)kBufs * kBufBytes;
    static constexpr size_t kDig = kWhist + (size_t)OS_WARPS * RD * sizeof(WH);
    static constexpr size_t kBytes = kDig + (kWide ? 0 : OS_TILE);
};
static_assert(32 * OS_ITEMS <= 65535 && OS_TILE <= 65535, "16-bit per-warp digit counts");

template <int FLAGS, int DBITS>
__global__ void __launch_bounds__(OS_THREADS,
                                  (FLAGS & OS_PAYLOAD_UV) || DBITS > 9 ? OS_MIN_BLOCKS : OS_MIN_BLOCKS + 1)
    onesweep_kernel(const OnesweepParams p)
{
    constexpr bool kUV = (FLAGS & OS_PAYLOAD_UV) != 0;
    constexpr bool kGen = (FLAGS & OS_GEN_VALS) != 0;
    using L = OsSmem<FLAGS, DBITS>;
    using WH = typename L::WH;
    constexpr int RD = L::RD;
    constexpr u32 DMASK = (u32)RD - 1u;
    constexpr int DPT = DigitsPerThread<RD>::value;   // digits owned per thread
    constexpr int ACT = RD / DPT;                      // threads that own digits
    extern __shared__ __align__(128) unsigned char smem[];
    // B0 keys in, later values in digit order; B1 values in; B2 keys in
    // digit order; with endpoints (kUV) B3..B4 the endpoints in (the first
    // pass: u in B3 and v in B4 from the caller's arrays; later passes one
    // int2 per element) and B1..B2, once values and keys are out, the
    // endpoints in digit order (int2)
    u32 *B0 = (u32 *)smem;
    u32 *B1 = B0 + OS_TILE;
    u32 *B2 = B1 + OS_TILE;
    u32 *B3 = B2 + OS_TILE;
    u32 *B4 = B3 + OS_TILE;                       // kUV only
    u32 *KD = B2;                                 // keys in digit order
    WH (*s_whist)[RD] = (WH(*)[RD])(smem + L::kWhist);
    unsigned char *s_dig = smem + L::kDig;        // 8-bit digits only
    __shared__ u32 s_goff[RD];                    // global position of local position 0, per digit
    __shared__ u32 s_local_start[RD];
    __shared__ u32 s_warp[OS_WARPS];
    __shared__ u32 s_tile;
    __shared__ __align__(8) u64 s_bar[2];         // [0] keys landed, [1] value streams landed

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < OS_WARPS * RD; i += OS_THREADS)
        (&s_whist[0][0])[i] = 0;
    if (tid == 0) {
        s_tile = atomicAdd(p.tile_counter, 1u);
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const u32 tile = s_tile;
    const i64 tile_base = (i64)tile * OS_TILE;
    const i64 rem = p.n - tile_base;
    const int tile_count = rem < OS_TILE ? (int)rem : OS_TILE;
    // whole 16-byte chunks go by TMA; the last (tile_count % 4) elements of
    // the array by plain loads (a bulk copy must not read past its end)
    const int n_bulk = tile_count & ~3;
    // A bulk copy needs 16-byte aligned source and destination (the smem
    // buffers are; tile_base * 4 is a multiple of 16 KB).  Each stream whose
    // base address is not aligned -- possible for caller arrays -- is read
    // with plain loads instead.
    const void *ksrc = (FLAGS & OS_KEY_FROM_W) ? (const void *)(p.w_in + tile_base)
                                               : (const void *)(p.keys_in + tile_base);
    const void *vsrc = kGen ? nullptr : (const void *)(p.vals_in + tile_base);
    const void *usrc = !kUV ? nullptr
                            : kGen ? (const void *)(p.u + tile_base) : (const void *)(p.uv_in + tile_base);
    const void *wsrc = kUV && kGen ? (const void *)(p.v + tile_base) : nullptr;
    const bool k_bulk = (((uintptr_t)ksrc) & 15) == 0;
    const bool v_bulk = !kGen && (((uintptr_t)vsrc) & 15) == 0;
    const bool uv_bulk = kUV && ((((uintptr_t)usrc | (uintptr_t)wsrc) & 15) == 0);
    if (tid == 0) {
        const u32 bytes = (u32)n_bulk * 4;
        mbar_arrive_expect_tx(&s_bar[0], k_bulk ? bytes : 0u);
        if (k_bulk && bytes)
            tma_load_1d(B0, ksrc, bytes, &s_bar[0]);
        mbar_arrive_expect_tx(&s_bar[1], (v_bulk ? bytes : 0u) + (uv_bulk ? 2u * bytes : 0u));
        if (bytes) {
            if (v_bulk)
                tma_load_1d(B1, vsrc, bytes, &s_bar[1]);
            if (uv_bulk) {
                if (kGen) {
                    tma_load_1d(B3, usrc, bytes, &s_bar[1]);
                    tma_load_1d(B4, wsrc, bytes, &s_bar[1]);
                } else {
                    tma_load_1d(B3, usrc, 2u * bytes, &s_bar[1]);   // int2 per element
                }
            }
        }
    }
    // tails and streams that are not bulk-copied: plain loads into ranges the
    // copies do not touch
    for (int i = (k_bulk ? n_bulk : 0) + tid; i < tile_count; i += OS_THREADS)
        B0[i] = (FLAGS & OS_KEY_FROM_W) ? __float_as_uint(p.w_in[tile_base + i]) : p.keys_in[tile_base + i];
    if (!kGen)
        for (int i = (v_bulk ? n_bulk : 0) + tid; i < tile_count; i += OS_THREADS)
            B1[i] = p.vals_in[tile_base + i];
    if (kUV) {
        for (int i = (uv_bulk ? n_bulk : 0) + tid; i < tile_count; i += OS_THREADS) {
            if (kGen) {
                B3[i] = (u32)p.u[tile_base + i];
                B4[i] = (u32)p.v[tile_base + i];
            } else {
                ((int2 *)B3)[i] = p.uv_in[tile_base + i];
            }
        }
    }
    // global start of every owned digit's bucket: scanned once per pass when
    // the caller provides it, else here
    u32 bin_base[DPT];
    if (p.bin_base) {
#pragma unroll
        for (int k = 0; k < DPT; ++k)
            bin_base[k] = tid < ACT ? p.bin_base[tid * DPT + k] : 0u;
    } else {
        u32 hx[DPT];
#pragma unroll
        for (int k = 0; k < DPT; ++k)
            hx[k] = tid < ACT ? p.hist[tid * DPT + k] : 0u;
        digits_exclusive_scan<RD>(hx, bin_base, s_warp);
    }
    mbar_wait_bounded(&s_bar[0], 0, p.status);
    __syncthreads();   // plain-loaded tail elements visible to all

    const int wbase = warp * (32 * OS_ITEMS);   // this warp's run inside the tile
    const int shift = p.shift;
    auto key_at = [&](int i) -> u32 {
        const u32 x = B0[i];
        return (FLAGS & OS_KEY_FROM_W) ? weight_key(__uint_as_float(x)) : x;
    };

    // ---- stable warp-level ranking by digit (ballot multisplit) ------------
    u32 lpos[OS_ITEMS];    // rank within warp and digit, later local position
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const int i = wbase + it * 32 + lane;
        const bool valid = i < tile_count;
        const u32 d = valid ? (key_at(i) >> shift) & DMASK : 0u;
        u32 peers = __ballot_sync(0xFFFFFFFFu, valid);
#pragma unroll
        for (int b = 0; b < DBITS; ++b) {
            const u32 bit = (d >> b) & 1u;
            const u32 bal = __ballot_sync(0xFFFFFFFFu, bit);
            peers &= bit ? bal : ~bal;
        }
        const int leader = valid ? (__ffs(peers) - 1) : lane;
        u32 base = 0;
        if (valid && lane == leader) {
            base = s_whist[warp][d];
            s_whist[warp][d] = (WH)(base + __popc(peers));
        }
        __syncwarp();
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        lpos[it] = base + __popc(peers & lt);
    }
    __syncthreads();

    // ---- per-digit totals of the tile; publish for look-back ---------------
    u32 total[DPT];
    u64 *lbt = p.lb + (u64)tile * RD;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        total[k] = 0;
        if (tid < ACT) {
            const int d = tid * DPT + k;
#pragma unroll
            for (int w = 0; w < OS_WARPS; ++w) {
                const u32 c = s_whist[w][d];
                s_whist[w][d] = (WH)total[k];
                total[k] += c;
            }
            st_relaxed(lbt + d, (tile == 0 ? LB_INC : LB_AGG) | (u64)total[k]);
        }
    }
    u32 local_start[DPT];
    digits_exclusive_scan<RD>(total, local_start, s_warp);
    if (tid < ACT) {
#pragma unroll
        for (int k = 0; k < DPT; ++k)
            s_local_start[tid * DPT + k] = local_start[k];
    }
    __syncthreads();

    // ---- keys into KD in digit order ------------------------------------------
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const int i = wbase + it * 32 + lane;
        if (i < tile_count) {
            const u32 key = key_at(i);
            const u32 d = (key >> shift) & DMASK;
            const u32 pos = s_local_start[d] + s_whist[warp][d] + lpos[it];
            KD[pos] = key;
            if (!L::kWide)
                s_dig[pos] = (unsigned char)d;
            lpos[it] = pos;
        }
    }

    // ---- decoupled look-back, per owned digit, 8 tiles per round trip -------
#pragma unroll
    for (int kd = 0; kd < DPT; ++kd) {
        if (tid >= ACT)
            break;
        const int dg = tid * DPT + kd;
        u64 excl = 0;
        if (tile > 0) {
            i64 j = (i64)tile - 1;
            u32 spins = 0;
            for (;;) {
                u64 sv[LB_BATCH];
#pragma unroll
                for (int k = 0; k < LB_BATCH; ++k)
                    sv[k] = (j - k >= 0) ? ld_relaxed(p.lb + (u64)(j - k) * RD + dg) : LB_INC;
                int consumed = 0;
                bool done = false;
#pragma unroll
                for (int k = 0; k < LB_BATCH; ++k) {
                    if (done || consumed < k)
                        continue;
                    const u64 f = sv[k] & ~LB_VAL;
                    if (f == 0)
                        continue;            // not published yet: reload from here
                    excl += sv[k] & LB_VAL;
                    consumed = k + 1;
                    if (f == LB_INC)
                        done = true;
                }
                if (done)
                    break;
                j -= consumed;
                if (consumed == 0) {
                    ++spins;
                    if (spins == p.report_limit + 1u)
                        set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
                    if (spins > SPIN_LIMIT) {
                        set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
                        break;
                    }
                    if (spins > 16)
                        __nanosleep(32);
                }
            }
            st_relaxed(lbt + dg, LB_INC | (excl + total[kd]));
        }
        s_goff[dg] = bin_base[kd] + (u32)excl - local_start[kd];   // modulo 2^32
    }
    mbar_wait_bounded(&s_bar[1], 0, p.status);   // value streams landed
    __syncthreads();

    // ---- write keys (KD); values, stream 0, into B0 in digit order ------------
    // digit of output position j (KD keeps the keys in digit order)
    auto dig_at = [&](int j) -> u32 { return L::kWide ? (KD[j] >> shift) & DMASK : (u32)s_dig[j]; };
    if (FLAGS & OS_WRITE_KEYS) {
        for (int j = tid; j < tile_count; j += OS_THREADS)
            p.keys_out[s_goff[dig_at(j)] + (u32)j] = KD[j];
    }
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const int i = wbase + it * 32 + lane;
        if (i < tile_count)
            B0[lpos[it]] = kGen ? (u32)(tile_base + i) : B1[i];
    }
    __syncthreads();

    // ---- write values (B0); endpoints into B1..B2 in digit order --------------
    for (int j = tid; j < tile_count; j += OS_THREADS)
        p.vals_out[s_goff[dig_at(j)] + (u32)j] = B0[j];
    if (kUV) {
#pragma unroll
        for (int it = 0; it < OS_ITEMS; ++it) {
            const int i = wbase + it * 32 + lane;
            if (i < tile_count) {
                u32 xa, xb;
                if (kGen) {
                    xa = B3[i];
                    xb = B4[i];
                } else {
                    const int2 e = ((const int2 *)B3)[i];
                    xa = (u32)e.x;
                    xb = (u32)e.y;
                }
                if (kGen) {
                    // first pass: validate the caller's endpoints and turn
                    // tree-local ids into forest ids
                    i32 a = (i32)xa, b = (i32)xb;
                    i64 nv = p.n_vertices, voff = 0;
                    if (FLAGS & OS_FOREST) {
                        const i64 e = tile_base + i;
                        const i64 t = tree_of_edge(p.edge_off, p.n_trees, e);
                        const i64 e0 = __ldg(p.edge_off + t), e1 = __ldg(p.edge_off + t + 1);
                        nv = e1 - e0 + 1;
                        voff = e0 + t;
                        if (e0 < 0 || e1 > p.n || e < e0 || e >= e1) {
                            // offsets that are not a partition of [0, M) (an
                            // asynchronous call cannot stop at the host check):
                            // keep every id inside the forest
                            set_status(p.status, PANDORA_ERR_INVALID_ARGUMENT);
                            nv = 0;
                            voff = 0;
                        }
                    }
                    if (a < 0 || (i64)a >= nv || b < 0 || (i64)b >= nv) {
                        set_status(p.status, PANDORA_ERR_VERTEX_OUT_OF_RANGE);
                        a = 0;
                        b = 0;
                    } else if (a == b) {
                        set_status(p.status, PANDORA_ERR_SELF_LOOP);
                    }
                    xa = (u32)(a + voff);
                    xb = (u32)(b + voff);
                }
                ((int2 *)B1)[lpos[it]] = make_int2((i32)xa, (i32)xb);
            }
        }
        __syncthreads();
        // the last pass writes the level-0 edge array, the others the next
        // pass's endpoint stream: both an int2 per edge
        for (int j = tid; j < tile_count; j += OS_THREADS)
            p.uv_out[s_goff[s_dig[j]] + (u32)j] = ((const int2 *)B1)[j];
    }
}

// Exclusive scan of each 256-digit histogram row (one block per row).
__global__ void __launch_bounds__(RADIX) hist_scan_kernel(const u32 *hist, u32 *base)
{
    __shared__ u32 s_warp[RADIX / 32];
    const u32 x = hist[blockIdx.x * RADIX + threadIdx.x];
    base[blockIdx.x * RADIX + threadIdx.x] = digit_exclusive_scan(x, s_warp);
}

// Exclusive scan of the histogram row of every pass of a digit plan (one
// block of 1024 threads per pass, one thread per digit).
__global__ void __launch_bounds__(1024) hist_scan_plan_kernel(const u32 *hist, u32 *base,
                                                              const DigitPlan plan)
{
    __shared__ u32 s_warp[32];
    const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rd = 1 << plan.width[q];
    const int d = threadIdx.x;
    const u32 x = d < rd ? hist[plan.off[q] + d] : 0u;
    u32 incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    u32 pre = 0;
    for (int k = 0; k < warp; ++k)
        pre += s_warp[k];
    if (d < rd)
        base[plan.off[q] + d] = pre + incl - x;
}

// Digit histograms of 32-bit keys for every pass of a digit plan (one read
// of the keys); a key at or above 2^key_bits is reported.
__global__ void __launch_bounds__(256) hist_keys_plan_kernel(const u32 *__restrict__ keys, i64 n,
                                                             const DigitPlan plan, int key_bits,
                                                             u32 *__restrict__ hist, int *status)
{
    __shared__ u32 s_h[DIGIT_PLAN_HIST];
    const int h_total = plan.off[plan.n - 1] + (1 << plan.width[plan.n - 1]);
    for (int i = threadIdx.x; i < h_total; i += blockDim.x)
        s_h[i] = 0;
    __syncthreads();
    bool bad = false;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
        const u32 k = keys[i];
        bad |= key_bits < 32 && (k >> key_bits) != 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (q < plan.n)
                atomicAdd(&s_h[plan.off[q] + ((k >> plan.shift[q]) & ((1u << plan.width[q]) - 1u))], 1u);
    }
    if (bad)
        set_status(status, PANDORA_ERR_INVALID_ARGUMENT);
    __syncthreads();
    for (int i = threadIdx.x; i < h_total; i += blockDim.x)
        if (s_h[i])
            atomicAdd(hist + i, s_h[i]);
}

}  // namespace

void launch_hist_scan(const u32 *hist, u32 *base, int rows, cudaStream_t s)
{
    hist_scan_kernel<<<rows, RADIX, 0, s>>>(hist, base);
}

DigitPlan digit_plan(int bits)
{
    DigitPlan pl{};
    if (bits <= 0)
        return pl;
    if (bits <= 24 || bits > 27) {
        pl.n = (bits + 7) / 8;
        for (int q = 0; q < pl.n; ++q)
            pl.width[q] = 8;
    } else {
        // three passes, the bits spread as evenly as possible (8 or 9 each)
        pl.n = 3;
        for (int q = 0; q < 3; ++q)
            pl.width[q] = bits / 3 + (q < bits % 3 ? 1 : 0);
    }
    for (int q = 0; q < pl.n; ++q) {
        pl.shift[q] = q == 0 ? 0 : pl.shift[q - 1] + pl.width[q - 1];
        pl.off[q] = q == 0 ? 0 : pl.off[q - 1] + (1 << pl.width[q - 1]);
    }
    return pl;
}

void launch_hist_scan_plan(const u32 *hist, u32 *base, const DigitPlan &plan, cudaStream_t s)
{
    if (plan.n > 0)
        hist_scan_plan_kernel<<<plan.n, 1024, 0, s>>>(hist, base, plan);
}

void launch_hist_keys(const u32 *keys, i64 n, u32 *hist, cudaStream_t s)
{
    if (n <= 0)
        return;
    i64 blocks = (n + 256 * 16 - 1) / (256 * 16);
    if (blocks > 152 * 4)
        blocks = 152 * 4;
    hist_keys_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys, n, hist);
}

void launch_hist_weights(const float *w, i64 n, u32 *hist, int *status, cudaStream_t s)
{
    if (n <= 0)
        return;
    i64 blocks = (n + 256 * 16 - 1) / (256 * 16);
    if (blocks > 152 * 4)
        blocks = 152 * 4;
    hist_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(w, n, hist, status);
}

template <int F, int DBITS = 8>
static void launch_os(const OnesweepParams &p, cudaStream_t s)
{
    constexpr size_t bytes = OsSmem<F, DBITS>::kBytes;
    // opt in to more than 48 KB of dynamic shared memory, once per device
    static std::atomic<unsigned long long> done_mask{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done_mask.load() & bit)) {
        cudaFuncSetAttribute(onesweep_kernel<F, DBITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
        done_mask.fetch_or(bit);
    }
    const i64 tiles = p.grid_tiles > 0 ? p.grid_tiles : onesweep_tiles(p.n);
    onesweep_kernel<F, DBITS><<<(unsigned)tiles, OS_THREADS, bytes, s>>>(p);
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
    case OS_WRITE_KEYS:
        if (p.dbits == 9)
            launch_os<OS_WRITE_KEYS, 9>(p, s);
        else
            launch_os<OS_WRITE_KEYS>(p, s);
        break;
    default: break;
    }
}

// ---- the sort on its own (include/pandora_sort.h) ---------------------------
namespace {

struct SortCtrl {
    int status;
    u32 tile_counter[3];
    u32 hist[DIGIT_PLAN_HIST];
    u32 base[DIGIT_PLAN_HIST];
};

struct SortLayout {
    size_t ctrl, tmp_keys, tmp_vals, lb, total;
};

SortLayout sort_layout(i64 n, const DigitPlan &plan)
{
    int widest = 8;
    for (int q = 0; q < plan.n; ++q)
        widest = widest > plan.width[q] ? widest : plan.width[q];
    SortLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    L.ctrl = take(sizeof(SortCtrl));
    L.tmp_keys = take((size_t)n * 4);
    L.tmp_vals = take((size_t)n * 4);
    L.lb = take((size_t)onesweep_tiles(n) * ((size_t)1 << widest) * 8);
    L.total = off;
    return L;
}

}  // namespace

}  // namespace pandora

using namespace pandora;

extern "C" int pandora_sort_pairs_workspace_size(int64_t n, int32_t key_bits, size_t *bytes)
{
    if (!bytes || n < 0 || key_bits < 1 || key_bits > 32)
        return PANDORA_ERR_INVALID_ARGUMENT;
    *bytes = sort_layout(n, digit_plan(key_bits)).total;
    return PANDORA_OK;
}

extern "C" int pandora_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, int64_t n,
                                  int32_t key_bits, uint32_t *keys_out, uint32_t *vals_out,
                                  void *workspace, size_t workspace_bytes, void *stream)
{
    if (n < 0 || n > (int64_t)0x7FFFFFFF || key_bits < 1 || key_bits > 32)
        return PANDORA_ERR_INVALID_ARGUMENT;
    if (n == 0)
        return PANDORA_OK;
    if (!keys_in || !vals_in || !keys_out || !vals_out || !workspace)
        return PANDORA_ERR_INVALID_ARGUMENT;
    const DigitPlan plan = digit_plan(key_bits);
    const SortLayout L = sort_layout(n, plan);
    if (workspace_bytes < L.total || ((uintptr_t)workspace & 15) != 0)
        return workspace_bytes < L.total ? PANDORA_ERR_WORKSPACE_TOO_SMALL : PANDORA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *ws = (unsigned char *)workspace;
    SortCtrl *ctrl = (SortCtrl *)(ws + L.ctrl);
    u32 *tk = (u32 *)(ws + L.tmp_keys), *tv = (u32 *)(ws + L.tmp_vals);
    u64 *lb = (u64 *)(ws + L.lb);
    if (cudaMemsetAsync(ctrl, 0, sizeof(SortCtrl), s) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    i64 blocks = (n + 256 * 16 - 1) / (256 * 16);
    if (blocks > 152 * 4)
        blocks = 152 * 4;
    hist_keys_plan_kernel<<<(unsigned)blocks, 256, 0, s>>>(keys_in, n, plan, key_bits, ctrl->hist,
                                                           &ctrl->status);
    launch_hist_scan_plan(ctrl->hist, ctrl->base, plan, s);
    // ping-pong so that the last pass writes the caller's outputs
    const u32 *ik = keys_in, *iv = vals_in;
    for (int q = 0; q < plan.n; ++q) {
        const bool to_out = ((plan.n - 1 - q) & 1) == 0;
        OnesweepParams P{};
        P.report_limit = wait_report_limit();
        P.n = n;
        P.shift = plan.shift[q];
        P.dbits = plan.width[q];
        P.hist = ctrl->hist + plan.off[q];
        P.bin_base = ctrl->base + plan.off[q];
        P.lb = lb;
        P.tile_counter = &ctrl->tile_counter[0];
        P.status = &ctrl->status;
        P.keys_in = ik;
        P.vals_in = iv;
        P.keys_out = to_out ? keys_out : tk;
        P.vals_out = to_out ? vals_out : tv;
        if (cudaMemsetAsync(lb, 0, (size_t)onesweep_tiles(n) * ((size_t)1 << P.dbits) * 8, s) != cudaSuccess ||
            cudaMemsetAsync(&ctrl->tile_counter[0], 0, 4, s) != cudaSuccess)
            return PANDORA_ERR_CUDA;
        launch_onesweep(OS_WRITE_KEYS, P, s);
        ik = P.keys_out;
        iv = P.vals_out;
    }
    int status = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PANDORA_ERR_CUDA;
    return status;
}

// Onesweep LSD radix sort of (key, value) pairs for sm_103a.
//
// Paper step: the edges are sorted by weight with a consistent tie rule
// (Section 3.1); the chains are sorted again after expansion (Section 3.3.3).
// Both sorts are stable LSD radix sorts over 8-bit digits, so equal keys keep
// their input order: for the weight sort the value is the caller edge index
// and ties therefore resolve by index, for the chain sort the input is in
// ascending rank so every chain comes out in ascending rank.
//
// One pass = one kernel (Adinets & Merrill's onesweep): a block takes the
// next tile id from an atomic counter, ranks its 4096 keys by digit with
// warp ballots (stable: warp w of the tile owns a contiguous run of 512
// keys, processed 32 at a time in order), publishes its per-digit counts and
// finds the counts of all earlier tiles by decoupled look-back, then
// scatters keys and values through shared memory so that each digit's run is
// written contiguously.  The per-pass digit totals come from one histogram
// read of all keys done before the first pass.
#include "kernels.cuh"

namespace pandora {

namespace {

constexpr int OS_WARPS = OS_THREADS / 32;
static_assert(OS_THREADS == RADIX, "one thread per digit");

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ u32 block_exclusive_scan_256(u32 x, u32 *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        u32 y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off)
            incl += y;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();
    u32 prefix = 0;
#pragma unroll
    for (int k = 0; k < OS_WARPS; ++k)
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
__global__ void __launch_bounds__(OS_THREADS) onesweep_kernel(const OnesweepParams p)
{
    __shared__ u32 s_whist[OS_WARPS][RADIX];   // per-warp digit counts, then offsets
    __shared__ u32 s_buf[OS_TILE];             // tile in digit order (keys, then values)
    __shared__ u32 s_goff[RADIX];              // global position of local position 0, per digit
    __shared__ u32 s_local_start[RADIX];
    __shared__ u32 s_warp[OS_WARPS];
    __shared__ u32 s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < OS_WARPS * RADIX; i += OS_THREADS)
        (&s_whist[0][0])[i] = 0;
    if (tid == 0)
        s_tile = atomicAdd(p.tile_counter, 1u);
    // global start of every digit's bucket (exclusive scan of the pass histogram)
    const u32 bin_base = block_exclusive_scan_256(p.hist[tid], s_warp);
    const u32 tile = s_tile;   // published before the scan's barriers
    const i64 tile_base = (i64)tile * OS_TILE;
    const i64 warp_base = tile_base + (i64)warp * (32 * OS_ITEMS);
    const int shift = p.shift;

    u32 reg[OS_ITEMS];     // keys, later values
    u32 lpos[OS_ITEMS];    // rank within warp and digit, later local position
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        if (idx < p.n) {
            if (FLAGS & OS_KEY_FROM_W)
                reg[it] = weight_key(p.w_in[idx]);
            else
                reg[it] = p.keys_in[idx];
        } else {
            reg[it] = 0;
        }
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
#pragma unroll
    for (int k = 0; k < OS_WARPS; ++k) {
        const u32 c = s_whist[k][tid];
        s_whist[k][tid] = total;
        total += c;
    }
    u64 *lbt = p.lb + (u64)tile * RADIX;
    st_relaxed(lbt + tid, (tile == 0 ? LB_INC : LB_AGG) | (u64)total);
    const u32 local_start = block_exclusive_scan_256(total, s_warp);
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
    // values into registers while the look-back runs
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        if (FLAGS & OS_GEN_VALS)
            reg[it] = (u32)idx;
        else
            reg[it] = idx < p.n ? p.vals_in[idx] : 0u;
    }

    // ---- decoupled look-back, one thread per digit -------------------------
    u64 excl = 0;
    if (tile > 0) {
        i64 j = (i64)tile - 1;
        u32 spins = 0;
        while (j >= 0) {
            const u64 s = ld_relaxed(p.lb + (u64)j * RADIX + tid);
            const u64 f = s & ~LB_VAL;
            if (f == 0) {
                if (++spins > SPIN_LIMIT) {
                    set_status(p.status, PANDORA_ERR_ITERATION_LIMIT);
                    break;
                }
                if (spins > 32)
                    __nanosleep(32);
                continue;
            }
            excl += s & LB_VAL;
            if (f == LB_INC)
                break;
            --j;
        }
        st_relaxed(lbt + tid, LB_INC | (excl + total));
    }
    s_goff[tid] = bin_base + (u32)excl - local_start;   // modulo 2^32
    __syncthreads();

    // ---- write keys, one digit run after another ---------------------------
    const i64 rem = p.n - tile_base;
    const int tile_count = rem < OS_TILE ? (int)rem : OS_TILE;
    u32 dj[OS_ITEMS];
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
        const int j = k * OS_THREADS + tid;
        if (j < tile_count) {
            const u32 key = s_buf[j];
            dj[k] = (key >> shift) & 255u;
            if (FLAGS & OS_WRITE_KEYS)
                p.keys_out[s_goff[dj[k]] + (u32)j] = key;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const i64 idx = warp_base + it * 32 + lane;
        if (idx < p.n)
            s_buf[lpos[it]] = reg[it];
    }
    __syncthreads();

    // ---- write values (and, on the last weight pass, the endpoints) --------
#pragma unroll
    for (int k = 0; k < OS_ITEMS; ++k) {
        const int j = k * OS_THREADS + tid;
        if (j < tile_count) {
            const u32 val = s_buf[j];
            const u32 pos = s_goff[dj[k]] + (u32)j;
            p.vals_out[pos] = val;
            if (FLAGS & OS_GATHER) {
                i32 a = __ldg(p.u + val);
                i32 b = __ldg(p.v + val);
                i64 nv = p.n_vertices;
                i64 voff = 0;
                if (FLAGS & OS_FOREST) {
                    const i64 t = tree_of_edge(p.edge_off, p.n_trees, (i64)val);
                    const i64 e0 = __ldg(p.edge_off + t), e1 = __ldg(p.edge_off + t + 1);
                    nv = e1 - e0 + 1;
                    voff = e0 + t;
                }
                if (a < 0 || (i64)a >= nv || b < 0 || (i64)b >= nv) {
                    set_status(p.status, PANDORA_ERR_VERTEX_OUT_OF_RANGE);
                    a = 0;
                    b = 0;
                } else if (a == b) {
                    set_status(p.status, PANDORA_ERR_SELF_LOOP);
                }
                p.ab_out[pos] = make_int2((i32)(a + voff), (i32)(b + voff));
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
    switch (flags) {
    // weight sort: first, middle, last pass and single pass (one or forest)
    case OS_KEY_FROM_W | OS_GEN_VALS | OS_WRITE_KEYS: launch_os<OS_KEY_FROM_W | OS_GEN_VALS | OS_WRITE_KEYS>(p, s); break;
    case OS_WRITE_KEYS: launch_os<OS_WRITE_KEYS>(p, s); break;
    case OS_GATHER: launch_os<OS_GATHER>(p, s); break;
    case OS_GATHER | OS_FOREST: launch_os<OS_GATHER | OS_FOREST>(p, s); break;
    case OS_KEY_FROM_W | OS_GEN_VALS | OS_GATHER: launch_os<OS_KEY_FROM_W | OS_GEN_VALS | OS_GATHER>(p, s); break;
    case OS_KEY_FROM_W | OS_GEN_VALS | OS_GATHER | OS_FOREST: launch_os<OS_KEY_FROM_W | OS_GEN_VALS | OS_GATHER | OS_FOREST>(p, s); break;
    default: break;
    }
}

}  // namespace pandora

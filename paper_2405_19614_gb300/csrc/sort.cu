// One stable 8-bit counting pass of (uint32 key, uint32 value) pairs, onesweep
// style: a block ranks a 4096-key tile in shared memory, finds the tile's
// global offsets by a decoupled look-back over its predecessors, and scatters
// through shared memory so that the global writes are coalesced.  Tile ids
// come from an atomic counter, so every predecessor of a tile is already
// running and the look-back always makes progress; each wait is still bounded
// and reports GS_ERR_TIMEOUT instead of hanging.  The digit histograms are
// built by the kernels that produce the keys.
#include "sort.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = kSortTileKeys / kSortThreads;  // 16
constexpr uint32_t kLbAgg = 1u << 30;   // tile aggregate published
constexpr uint32_t kLbInc = 2u << 30;   // inclusive prefix published
constexpr uint32_t kLbMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;  // spins (32 ns sleeps) before a look-back wait gives up
#ifndef GS_SORT_LOOKBACK
#define GS_SORT_LOOKBACK 4
#endif
#ifndef GS_SORT_MIN_BLOCKS
#define GS_SORT_MIN_BLOCKS 4
#endif
constexpr int kLookback = GS_SORT_LOOKBACK;  // predecessors read at once

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Lanes of the warp whose 8-bit digit equals this lane's: the intersection,
// over the digit's bits, of the lanes that agree on each bit (eight ballots;
// cheaper here than the hardware match, which ran on a narrow pipe).
__device__ __forceinline__ uint32_t match_digit(uint32_t d)
{
#ifdef GS_SORT_HW_MATCH
    return __match_any_sync(kFullMask, d);
#endif
    uint32_t peers = kFullMask;
    #pragma unroll
    for (int b = 0; b < 8; b++) {
        const uint32_t ones = __ballot_sync(kFullMask, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? ones : ~ones;
    }
    return peers;
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *tmp /* [8] */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    uint32_t wbase = 0;
    #pragma unroll
    for (int w = 0; w < kSortWarps; w++) wbase += (w < warp) ? tmp[w] : 0u;
    __syncthreads();
    return wbase + inc - x;
}

struct SortSmem {
    uint32_t keys[kSortTileKeys];
    uint32_t vals[kSortTileKeys];
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t tile_prefix[kRadix];
    uint32_t digit_out[kRadix];
    uint32_t tmp[kSortWarps];
    uint32_t tile_id;
};

// Several blocks per SM: the ranking and scatter wait mostly on shared
// memory, so occupancy is what hides it; values stay out of registers until
// the staging.
template <int MODE>
__global__ void __launch_bounds__(kSortThreads, GS_SORT_MIN_BLOCKS) onesweep_kernel(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *n_p, uint32_t cap, const uint32_t *__restrict__ hist,
    uint32_t *lb, uint32_t *lb_next, uint32_t *block_counter, int shift, SortExpand ex, uint32_t *status,
    uint32_t spin_limit)
{
    __shared__ SortSmem S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = min(*n_p, cap);
    const uint32_t num_tiles = (n + kSortTileKeys - 1) / kSortTileKeys;
    // persistent: a block takes the next tile once it has finished the last,
    // so every tile a look-back waits on is held by a running block
    for (;;) {
        if (tid == 0) S.tile_id = atomicAdd(block_counter, 1u);
        for (int k = tid; k < kSortWarps * kRadix; k += kSortThreads) (&S.warp_hist[0][0])[k] = 0;
        __syncthreads();
        const uint32_t tile = S.tile_id;
        if (tile >= num_tiles) return;
        if (lb_next) lb_next[tile * kRadix + tid] = 0;  // the next pass starts from a clean slot

        uint32_t key[kSortItems], rank[kSortItems];
        const uint32_t base = tile * kSortTileKeys + warp * (32 * kSortItems) + lane;
        #pragma unroll
        for (int i = 0; i < kSortItems; i++) {
            const uint32_t idx = base + i * 32;
            key[i] = idx < n ? kin[idx] : ~0u;  // past n: ranks after every valid key of digit 255, lands past n
        }
        // stable rank within the warp, items in (i, lane) order
        const uint32_t lt_mask = (1u << lane) - 1u;
        #pragma unroll
        for (int i = 0; i < kSortItems; i++) {
            const uint32_t d = (key[i] >> shift) & 0xffu;
            const uint32_t peers = match_digit(d);
            const int leader = __ffs(peers) - 1;
            uint32_t prev = 0;
            if (lane == leader) {
                prev = S.warp_hist[warp][d];
                S.warp_hist[warp][d] = prev + (uint32_t)__popc(peers);
            }
            prev = __shfl_sync(kFullMask, prev, leader);
            rank[i] = prev + (uint32_t)__popc(peers & lt_mask);
            __syncwarp();
        }
        __syncthreads();

        // thread = digit: offsets of each warp within the tile's digit run
        const uint32_t d = tid;
        uint32_t count = 0;
        #pragma unroll
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = S.warp_hist[w][d];
            S.warp_hist[w][d] = count;
            count += c;
        }
        st_relaxed(lb + tile * kRadix + d, (tile == 0 ? kLbInc : kLbAgg) | count);
        const uint32_t tile_prefix = block_exclusive_scan(count, S.tmp);
        S.tile_prefix[d] = tile_prefix;
        __syncthreads();

        // stage the tile in digit order (so that the global writes are
        // coalesced) before the look-back, which then has the registers
        #pragma unroll
        for (int i = 0; i < kSortItems; i++) {
            const uint32_t dd = (key[i] >> shift) & 0xffu;
            rank[i] += S.tile_prefix[dd] + S.warp_hist[warp][dd];  // now the position in the tile
            S.keys[rank[i]] = key[i];
        }
        #pragma unroll
        for (int i = 0; i < kSortItems; i++) {
            const uint32_t idx = base + i * 32;
            S.vals[rank[i]] = idx < n ? vin[idx] : 0u;
        }

        // decoupled look-back over the predecessors' per-digit counts, reading
        // kLookback of them at a time: aggregates are summed up to the first
        // inclusive prefix; an entry not yet published is read again
        uint32_t prefix = 0;
        if (tile > 0) {
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            bool done = false;
            while (!done) {
                uint32_t x[kLookback];
                #pragma unroll
                for (int u = 0; u < kLookback; u++)
                    x[u] = j - u >= 0 ? ld_relaxed(lb + (uint32_t)(j - u) * kRadix + d) : kLbInc;
                int used = 0;
                #pragma unroll
                for (int u = 0; u < kLookback; u++) {
                    const uint32_t f = x[u] & ~kLbMask;
                    if (f == 0) break;  // not published yet
                    prefix += x[u] & kLbMask;
                    used = u + 1;
                    if (f == kLbInc) {
                        done = true;
                        break;
                    }
                }
                j -= used;
                if (j < 0) done = true;
                if (!done && used < kLookback) {  // entry j not published yet
                    if (++spins > spin_limit) {
                        raise_status(status, GS_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            st_relaxed(lb + tile * kRadix + d, kLbInc | (prefix + count));
        }
        const uint32_t gbase = block_exclusive_scan(hist[d], S.tmp);
        S.digit_out[d] = gbase + prefix;
        __syncthreads();

        if (MODE == kSortExpand) {
            // gathers eight at a time ahead of their writes
            constexpr int kGroup = 8;
            #pragma unroll 1
            for (int i0 = 0; i0 < kSortItems; i0 += kGroup) {
                uint2 rec[kGroup];
                uint32_t out[kGroup];
                #pragma unroll
                for (int i = 0; i < kGroup; i++) {
                    const int k = tid + (i0 + i) * kSortThreads;
                    const uint32_t dd = (S.keys[k] >> shift) & 0xffu;
                    out[i] = S.digit_out[dd] + ((uint32_t)k - S.tile_prefix[dd]);
                    rec[i] = out[i] < n ? ex.rec[S.vals[k]] : make_uint2(0u, 0u);
                }
                #pragma unroll
                for (int i = 0; i < kGroup; i++) {
                    if (out[i] >= n) continue;
                    const int k = tid + (i0 + i) * kSortThreads;
                    ex.keys[out[i]] = ((uint64_t)S.keys[k] << 32) | rec[i].x;
                    ex.vals[out[i]] = rec[i].y % ex.n;
                }
            }
        } else {
            for (int k = tid; k < kSortTileKeys; k += kSortThreads) {
                const uint32_t kk = S.keys[k];
                const uint32_t dd = (kk >> shift) & 0xffu;
                const uint32_t out = S.digit_out[dd] + ((uint32_t)k - S.tile_prefix[dd]);
                if (out >= n) continue;
                if (MODE == kSortPaired) {
                    reinterpret_cast<uint2 *>(kout)[out] = make_uint2(kk, S.vals[k]);
                } else {
                    kout[out] = kk;
                    vout[out] = S.vals[k];
                }
            }
        }
        __syncthreads();  // the tile's shared state is read before the next tile overwrites it
    }
}

template <int MODE>
static void launch_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                        const uint32_t *n_dev, int64_t cap, const uint32_t *hist, uint32_t *lb, uint32_t *lb_next,
                        uint32_t *block_counter, int shift, const SortExpand &ex, uint32_t *status, cudaStream_t s,
                        uint32_t spin_limit = kSpinLimit)
{
    static int per_sm = 0;  // resident blocks per SM (the same on every GB300)
    if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_kernel<MODE>, kSortThreads, 0);
    const int64_t tiles = (cap + kSortTileKeys - 1) / kSortTileKeys;
    const int64_t slots = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(tiles < slots ? tiles : slots);
    onesweep_kernel<MODE><<<grid, kSortThreads, 0, s>>>(kin, vin, kout, vout, n_dev, (uint32_t)cap, hist, lb,
                                                         lb_next, block_counter, shift, ex, status, spin_limit);
}

gs_status_t onesweep_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                          const uint32_t *n_dev, int64_t cap, const uint32_t *hist, uint32_t *lb,
                          uint32_t *lb_next, uint32_t *block_counter, int shift, int mode, const SortExpand *expand,
                          uint32_t *status, cudaStream_t s)
{
    if (cap < 1 || cap > 0xffffffffll) return GS_ERR_INVALID_ARG;
    const SortExpand none = {};
    switch (mode) {
    case kSortPlain:
        launch_pass<kSortPlain>(kin, vin, kout, vout, n_dev, cap, hist, lb, lb_next, block_counter, shift, none,
                                status, s);
        break;
    case kSortPaired:
        launch_pass<kSortPaired>(kin, vin, kout, vout, n_dev, cap, hist, lb, lb_next, block_counter, shift, none,
                                 status, s);
        break;
    case kSortExpand:
        if (!expand) return GS_ERR_INVALID_ARG;
        launch_pass<kSortExpand>(kin, vin, kout, vout, n_dev, cap, hist, lb, lb_next, block_counter, shift, *expand,
                                 status, s);
        break;
    default: return GS_ERR_INVALID_ARG;
    }
    return launch_status();
}

// Check of the asynchronous timeout path: two 4096-key tiles of pseudo-random
// keys sorted by their low byte.  The fill kernel writes the keys, values,
// digit histogram and key count, and starts the tile counter at 1 when tile 0
// is to be withheld, so that no block ever publishes tile 0.
constexpr int kCheckKeys = 2 * kSortTileKeys;
struct CheckLayout {
    static constexpr size_t kout = 0, vout = 4 * kCheckKeys, kin = 8 * kCheckKeys, vin = 12 * kCheckKeys,
                            hist = 16 * kCheckKeys, counter = hist + 4 * kRadix, n = counter + 4,
                            lb = align256(n + 4), bytes = lb + onesweep_lookback_bytes(kCheckKeys);
};

__global__ void check_fill_kernel(unsigned char *ws, int withhold_first_tile)
{
    uint32_t *kin = reinterpret_cast<uint32_t *>(ws + CheckLayout::kin);
    uint32_t *vin = reinterpret_cast<uint32_t *>(ws + CheckLayout::vin);
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + CheckLayout::hist);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kCheckKeys) return;
    const uint32_t k = (uint32_t)i * 2654435761u;  // multiplicative hash of the index
    kin[i] = k;
    vin[i] = (uint32_t)i;
    atomicAdd(&hist[k & 0xffu], 1u);
    if (i == 0) {
        *reinterpret_cast<uint32_t *>(ws + CheckLayout::counter) = withhold_first_tile ? 1u : 0u;
        *reinterpret_cast<uint32_t *>(ws + CheckLayout::n) = (uint32_t)kCheckKeys;
    }
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_check_lookback_timeout_workspace_size(void) { return CheckLayout::bytes; }

extern "C" gs_status_t gs_check_lookback_timeout(uint32_t spin_limit, int32_t withhold_first_tile, uint32_t *status,
                                                 void *workspace, size_t workspace_bytes, void *stream)
{
    if (!status || !workspace || workspace_bytes < CheckLayout::bytes ||
        (reinterpret_cast<uintptr_t>(workspace) & 255))
        return GS_ERR_INVALID_ARG;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStream_t s = as_stream(stream);
    // histogram, counters and look-back flags start at zero
    if (cudaMemsetAsync(ws + CheckLayout::hist, 0, CheckLayout::bytes - CheckLayout::hist, s) != cudaSuccess)
        return GS_ERR_CUDA;
    check_fill_kernel<<<kCheckKeys / 256, 256, 0, s>>>(ws, withhold_first_tile != 0);
    const SortExpand none = {};
    auto u32 = [&](size_t off) { return reinterpret_cast<uint32_t *>(ws + off); };
    launch_pass<kSortPlain>(u32(CheckLayout::kin), u32(CheckLayout::vin), u32(CheckLayout::kout),
                            u32(CheckLayout::vout), u32(CheckLayout::n), kCheckKeys, u32(CheckLayout::hist),
                            u32(CheckLayout::lb), nullptr, u32(CheckLayout::counter), 0, none, status, s,
                            spin_limit ? spin_limit : kSpinLimit);
    return launch_status();
}

// a3. Stable LSD radix sort of (uint64 key, uint32 value) pairs, onesweep
// style: one pass over the keys builds the histograms of every 8-bit digit,
// then one kernel per digit ranks a 4096-key tile in shared memory, finds the
// tile's global offsets by a decoupled look-back over its predecessors, and
// scatters.  Tile ids come from an atomic counter, so every predecessor of a
// tile is already running and the look-back always makes progress; each wait
// is still bounded and reports GS_ERR_TIMEOUT instead of hanging.
//
// Front-to-back order within each tile (Sec. 3.4 "Differentiable
// Rasterization") comes from the keys: (tile << 32) | bits(depth).
#include "common.cuh"
#include "sort.cuh"

namespace gs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kRadix = 256;
constexpr uint32_t kLbAgg = 1u << 30;   // tile aggregate published
constexpr uint32_t kLbInc = 2u << 30;   // inclusive prefix published
constexpr uint32_t kLbMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

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

__global__ void __launch_bounds__(256) sort_hist_kernel(const uint64_t *__restrict__ keys,
                                                        const uint32_t *n_pairs_p, uint32_t cap,
                                                        int n_passes, uint32_t *hist, uint32_t *lb0)
{
    __shared__ uint32_t sh[kMaxSortPasses][kRadix];
    for (int k = threadIdx.x; k < kMaxSortPasses * kRadix; k += blockDim.x) (&sh[0][0])[k] = 0;
    __syncthreads();
    const uint32_t n = min(*n_pairs_p, cap);
    const uint32_t num_tiles = (n + kSortTile - 1) / kSortTile;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (uint32_t k = gtid; k < num_tiles * kRadix; k += stride) lb0[k] = 0;
    const int lane = threadIdx.x & 31;
    for (uint32_t base = gtid - lane; base < n; base += stride) {
        const uint32_t i = base + lane;
        const bool valid = i < n;
        const uint64_t key = valid ? keys[i] : 0ull;
        for (int p = 0; p < n_passes; p++) {
            const uint32_t d = valid ? (uint32_t)((key >> (8 * p)) & 0xff) : 256u;
            const uint32_t peers = __match_any_sync(kFullMask, d);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&sh[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_passes * kRadix; k += blockDim.x) {
        const uint32_t c = (&sh[0][0])[k];
        if (c) atomicAdd(hist + k, c);
    }
}

struct SortSmem {
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t warp_hist[kSortWarps][kRadix];
    uint32_t tile_prefix[kRadix];
    uint32_t digit_out[kRadix];
    uint32_t tmp[kSortWarps];
    uint32_t tile_id;
};

__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(
    const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *n_pairs_p, uint32_t cap, const uint32_t *__restrict__ hist,
    uint32_t *lb, uint32_t *lb_next, uint32_t *tile_counter, int shift, uint32_t *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = min(*n_pairs_p, cap);
    const uint32_t num_tiles = (n + kSortTile - 1) / kSortTile;
    if (tid == 0) S.tile_id = atomicAdd(tile_counter, 1u);
    for (int k = tid; k < kSortWarps * kRadix; k += kSortThreads) (&S.warp_hist[0][0])[k] = 0;
    __syncthreads();
    const uint32_t tile = S.tile_id;
    if (tile >= num_tiles) return;
    if (lb_next) lb_next[tile * kRadix + tid] = 0;  // the next pass starts from a clean slot

    uint64_t key[kSortItems];
    uint32_t val[kSortItems], rank[kSortItems];
    const uint32_t base = tile * kSortTile + warp * (32 * kSortItems) + lane;
    #pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        const uint32_t idx = base + i * 32;
        if (idx < n) {
            key[i] = kin[idx];
            val[i] = vin[idx];
        } else {
            key[i] = ~0ull;  // ranks after every valid key of digit 255, lands past n
            val[i] = 0;
        }
    }
    // stable rank within the warp, items in (i, lane) order
    const uint32_t lt_mask = (1u << lane) - 1u;
    #pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        const uint32_t d = (uint32_t)(key[i] >> shift) & 0xffu;
        const uint32_t peers = __match_any_sync(kFullMask, d);
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

    // decoupled look-back over the predecessors' per-digit counts
    uint32_t prefix = 0;
    if (tile > 0) {
        int64_t j = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (j >= 0) {
            const uint32_t x = ld_relaxed(lb + (uint32_t)j * kRadix + d);
            const uint32_t f = x & ~kLbMask;
            if (f == 0) {
                if (++spins > kSpinLimit) {
                    raise_status(status, GS_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            prefix += x & kLbMask;
            if (f == kLbInc) break;
            --j;
        }
        st_relaxed(lb + tile * kRadix + d, kLbInc | (prefix + count));
    }
    const uint32_t gbase = block_exclusive_scan(hist[d], S.tmp);
    S.digit_out[d] = gbase + prefix;
    __syncthreads();

    // stage the tile in digit order so that the global writes are coalesced
    #pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        const uint32_t dd = (uint32_t)(key[i] >> shift) & 0xffu;
        const uint32_t pos = S.tile_prefix[dd] + S.warp_hist[warp][dd] + rank[i];
        S.keys[pos] = key[i];
        S.vals[pos] = val[i];
    }
    __syncthreads();
    for (int k = tid; k < kSortTile; k += kSortThreads) {
        const uint64_t kk = S.keys[k];
        const uint32_t dd = (uint32_t)(kk >> shift) & 0xffu;
        const uint32_t out = S.digit_out[dd] + ((uint32_t)k - S.tile_prefix[dd]);
        if (out < n) {
            kout[out] = kk;
            vout[out] = S.vals[k];
        }
    }
}

size_t sort_workspace_bytes(int64_t cap)
{
    const int64_t tiles = (cap + kSortTile - 1) / kSortTile + 1;
    size_t b = 0;
    b += align256(sizeof(uint32_t) * kMaxSortPasses * kRadix);  // histograms
    b += align256(sizeof(uint32_t) * kMaxSortPasses);           // tile counters
    b += 2 * align256(sizeof(uint32_t) * (size_t)tiles * kRadix);  // two look-back regions
    return b;
}

int sort_passes(int n_bits) { return (n_bits + 7) / 8; }

gs_status_t radix_sort_pairs(uint64_t *keys_a, uint32_t *vals_a, uint64_t *keys_b, uint32_t *vals_b,
                             const uint32_t *n_pairs, int64_t cap, int n_bits, void *ws, uint32_t *status,
                             cudaStream_t s)
{
    const int P = sort_passes(n_bits);
    if (P < 1 || P > kMaxSortPasses) return GS_ERR_INVALID_ARG;
    const int64_t tiles = (cap + kSortTile - 1) / kSortTile + 1;
    unsigned char *p = static_cast<unsigned char *>(ws);
    uint32_t *hist = reinterpret_cast<uint32_t *>(p);
    p += align256(sizeof(uint32_t) * kMaxSortPasses * kRadix);
    uint32_t *counters = reinterpret_cast<uint32_t *>(p);
    p += align256(sizeof(uint32_t) * kMaxSortPasses);
    uint32_t *lb[2];
    lb[0] = reinterpret_cast<uint32_t *>(p);
    p += align256(sizeof(uint32_t) * (size_t)tiles * kRadix);
    lb[1] = reinterpret_cast<uint32_t *>(p);

    if (cudaMemsetAsync(hist, 0, (char *)(counters + kMaxSortPasses) - (char *)hist, s) != cudaSuccess)
        return GS_ERR_CUDA;
    const int sms = num_sms();
    sort_hist_kernel<<<sms * 4, 256, 0, s>>>(keys_a, n_pairs, (uint32_t)cap, P, hist, lb[0]);

    static bool attr_set = false;
    const int smem = (int)sizeof(SortSmem);
    if (!attr_set) {
        if (cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return GS_ERR_CUDA;
        attr_set = true;
    }
    const unsigned grid = (unsigned)((cap + kSortTile - 1) / kSortTile);
    uint64_t *kin = keys_a, *kout = keys_b;
    uint32_t *vin = vals_a, *vout = vals_b;
    for (int pass = 0; pass < P; pass++) {
        onesweep_kernel<<<grid, kSortThreads, smem, s>>>(kin, vin, kout, vout, n_pairs, (uint32_t)cap,
                                                         hist + pass * kRadix, lb[pass & 1],
                                                         pass + 1 < P ? lb[(pass + 1) & 1] : nullptr,
                                                         counters + pass, 8 * pass, status);
        uint64_t *tk = kin;
        kin = kout;
        kout = tk;
        uint32_t *tv = vin;
        vin = vout;
        vout = tv;
    }
    return launch_status();
}

}  // namespace gs

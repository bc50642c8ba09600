// a2 - a4. Binning of projected Gaussians into 16x16 tiles in front-to-back
// order (Sec. 3.4 "Differentiable Rasterization": the Gaussians of each tile
// are arranged by depth before alpha blending).
//
// The result is the list a stable sort of the 64-bit keys (global tile << 32)
// | bits(depth), values = Gaussian index, would give: per tile, entries by
// depth, equal depths in index order.  It is built in two small sorts instead
// of one wide one:
//   1. the drawn (view, Gaussian) records are compacted and sorted by depth
//      (four 8-bit passes over 32-bit keys; ties stay in record order);
//   2. every record emits one (tile id, depth rank) pair per tile it touches,
//      in depth order, so the pair list is already in front-to-back order;
//   3. a stable sort of the pairs by tile id alone (ceil(log2 tiles / 8)
//      passes over 32-bit keys, two for up to 65,536 tiles) gives the final
//      order; its last pass writes the 64-bit keys and the values from the
//      depth rank;
//   4. each tile's [start, end) from the sorted keys.
// Steps 1 and 2 build the digit histograms of the passes that follow, so no
// pass needs a histogram kernel.  Emission is load-balanced: a block scans its
// records' tile counts in shared memory and consecutive threads take
// consecutive pairs, finding their record by binary search.
#include "binning.cuh"
#include "common.cuh"
#include "sort.cuh"

namespace gs {

__device__ __forceinline__ uint64_t block_exclusive_scan_u64(uint64_t x, uint64_t *tmp /* [8] */, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFullMask, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) tmp[warp] = inc;
    __syncthreads();
    uint64_t wbase = 0, all = 0;
    #pragma unroll
    for (int w = 0; w < kEmitThreads / 32; w++) {
        wbase += (w < warp) ? tmp[w] : 0ull;
        all += tmp[w];
    }
    __syncthreads();
    if (total) *total = all;
    return wbase + inc - x;
}

__device__ __forceinline__ void clear_hist(uint32_t (*h)[kRadix], int n_passes)
{
    for (int k = threadIdx.x; k < n_passes * kRadix; k += blockDim.x) (&h[0][0])[k] = 0;
}

__device__ __forceinline__ void flush_hist(uint32_t (*h)[kRadix], int n_passes, uint32_t *global)
{
    for (int k = threadIdx.x; k < n_passes * kRadix; k += blockDim.x) {
        const uint32_t c = (&h[0][0])[k];
        if (c) atomicAdd(global + k, c);
    }
}

// 1a. Drawn records (tiles_touched > 0) of each block of kEmitChunk records.
__global__ void __launch_bounds__(kEmitThreads) vis_count_kernel(const uint32_t *__restrict__ tt, int64_t total,
                                                                 uint64_t *block_sums)
{
    __shared__ uint64_t tmp[kEmitThreads / 32];
    const int64_t first = (int64_t)blockIdx.x * kEmitChunk + threadIdx.x;
    uint64_t s = 0;
    #pragma unroll
    for (int k = 0; k < kEmitItems; k++) {
        const int64_t o = first + k * kEmitThreads;
        if (o < total && tt[o] > 0) s++;
    }
    uint64_t all;
    block_exclusive_scan_u64(s, tmp, &all);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = all;
}

// One block: exclusive scan of the block sums in place, 16 consecutive sums
// per thread per round (all loads in flight at once); the grand total goes to
// *count, flagged when it exceeds cap.
constexpr int kScanPer = 16;

// When n_items_dev is set, only the first ceil(*n_items_dev / chunk) sums are
// scanned (the others belong to chunks past the drawn records and are neither
// written nor read).
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint64_t *sums, int64_t nb, int64_t cap, uint32_t *count,
                                                         uint32_t *status, const uint32_t *n_items_dev, int chunk)
{
    if (n_items_dev) {
        const int64_t used = ((int64_t)*n_items_dev + chunk - 1) / chunk;
        nb = used < nb ? used : nb;
    }
    __shared__ uint64_t tmp[32];
    __shared__ uint64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024 * kScanPer) {
        const int64_t first = base + (int64_t)threadIdx.x * kScanPer;
        uint64_t v[kScanPer], x = 0;
        #pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            v[k] = first + k < nb ? sums[first + k] : 0ull;
            x += v[k];
        }
        uint64_t inc = x;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFullMask, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) tmp[warp] = inc;
        __syncthreads();
        uint64_t wbase = 0, all = 0;
        for (int w = 0; w < 32; w++) {
            wbase += (w < warp) ? tmp[w] : 0ull;
            all += tmp[w];
        }
        uint64_t run = carry + wbase + inc - x;
        #pragma unroll
        for (int k = 0; k < kScanPer; k++) {
            if (first + k < nb) sums[first + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t total = carry;
        *count = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
        if (total > (uint64_t)cap) raise_status(status, GS_ERR_CAPACITY);
    }
}

// 1b. Compaction of the drawn records in record order: (depth bits, record
// id), and the histograms of the four depth digits.
__global__ void __launch_bounds__(kEmitThreads) vis_compact_kernel(const float *__restrict__ rec,
                                                                   const uint32_t *__restrict__ tt, int64_t total,
                                                                   const uint64_t *__restrict__ block_off,
                                                                   uint32_t *rz, uint32_t *rid, uint32_t *hist)
{
    __shared__ uint64_t tmp[kEmitThreads / 32];
    __shared__ uint32_t h[kDepthPasses][kRadix];
    clear_hist(h, kDepthPasses);
    // records first + 8 t .. first + 8 t + 7 belong to thread t, so the
    // compacted order is the record order
    const int64_t first = (int64_t)blockIdx.x * kEmitChunk + (int64_t)threadIdx.x * kEmitItems;
    bool vis[kEmitItems];
    uint64_t s = 0;
    static_assert(kEmitItems == 8, "two 16-byte loads a thread");
    if (first + kEmitItems <= total && (reinterpret_cast<uintptr_t>(tt) & 15) == 0) {
        // the thread's eight counts as two 16-byte loads (the warp's loads are
        // one contiguous kilobyte)
        const uint4 a = reinterpret_cast<const uint4 *>(tt + first)[0];
        const uint4 b = reinterpret_cast<const uint4 *>(tt + first)[1];
        const uint32_t t8[kEmitItems] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        #pragma unroll
        for (int k = 0; k < kEmitItems; k++) {
            vis[k] = t8[k] > 0;
            s += vis[k];
        }
    } else {
        #pragma unroll
        for (int k = 0; k < kEmitItems; k++) {
            const int64_t o = first + k;
            vis[k] = o < total && tt[o] > 0;
            s += vis[k];
        }
    }
    uint32_t z[kEmitItems];
    #pragma unroll
    for (int k = 0; k < kEmitItems; k++) z[k] = vis[k] ? __float_as_uint(rec[12 * (first + k) + 2]) : 0u;
    uint64_t pos = block_off[blockIdx.x] + block_exclusive_scan_u64(s, tmp, nullptr);
    #pragma unroll
    for (int k = 0; k < kEmitItems; k++) {
        if (vis[k]) {
            rz[pos] = z[k];
            rid[pos] = (uint32_t)(first + k);
            pos++;
        }
        count_digits_warp(h, z[k], vis[k], kDepthPasses);
    }
    __syncthreads();
    flush_hist(h, kDepthPasses, hist);
}

// Record ids and tile counts of the depth-sorted records j < n_vis of a
// block's chunk (thread t holds j = first + 2 t, first + 2 t + 1); recs holds
// (depth bits, record id) pairs.
__device__ __forceinline__ void chunk_counts(const uint2 *__restrict__ recs, const uint32_t *__restrict__ tt,
                                             uint32_t n_vis, uint32_t chunk, uint32_t (&r)[kPairItems],
                                             uint32_t (&c)[kPairItems])
{
    const int64_t first = (int64_t)chunk * kPairChunk + (int64_t)threadIdx.x * kPairItems;
    #pragma unroll
    for (int k = 0; k < kPairItems; k++) {
        const int64_t j = first + k;
        r[k] = j < n_vis ? recs[j].y : 0u;
        c[k] = j < n_vis ? tt[r[k]] : 0u;
    }
}

// 2a. Pairs of each block of kPairChunk depth-sorted records.
// Persistent over the chunks of the drawn records (their number is known
// only here): a grid sized to the GPU, not to every record slot, most of which
// are undrawn on a multi-view batch.
__global__ void __launch_bounds__(kEmitThreads) pair_count_kernel(const uint2 *__restrict__ recs,
                                                                  const uint32_t *__restrict__ tt,
                                                                  const uint32_t *n_vis_p, uint64_t *block_sums)
{
    __shared__ uint64_t tmp[kEmitThreads / 32];
    const uint32_t n_vis = *n_vis_p;
    const uint32_t n_chunks = (n_vis + kPairChunk - 1) / kPairChunk;
    for (uint32_t chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
        uint32_t r[kPairItems], c[kPairItems];
        chunk_counts(recs, tt, n_vis, chunk, r, c);
        uint64_t s = 0;
        #pragma unroll
        for (int k = 0; k < kPairItems; k++) s += c[k];
        uint64_t all;
        block_exclusive_scan_u64(s, tmp, &all);
        if (threadIdx.x == 0) block_sums[chunk] = all;
    }
}

// Index of the (k + 1)-th set bit of m (m has more than k set bits).
__device__ __forceinline__ int nth_set_bit(unsigned long long m, uint32_t k)
{
    for (uint32_t i = 0; i < k; i++) m &= m - 1ull;
    return __ffsll((long long)m) - 1;
}

// 2b. Emission of (tile id, depth rank) pairs in depth order, and the
// histograms of the tile-id digits.  A record's pairs are the tiles its mask
// keeps (rectangles of up to 64 tiles) or every tile of its rectangle.
__global__ void __launch_bounds__(kEmitThreads) pair_emit_kernel(const uint2 *__restrict__ recs,
                                                                 const uint2 *__restrict__ rect,
                                                                 const unsigned long long *__restrict__ tmask,
                                                                 const uint32_t *__restrict__ tt,
                                                                 const uint32_t *n_vis_p, uint32_t n, ViewTable vt,
                                                                 const uint64_t *__restrict__ block_off, int64_t cap,
                                                                 uint32_t *tk, uint32_t *tv, uint32_t *hist,
                                                                 int tile_passes)
{
    __shared__ uint64_t tmp[kEmitThreads / 32];
    __shared__ uint32_t s_excl[kPairChunk + 1];
    __shared__ uint32_t s_r0[kPairChunk], s_r1[kPairChunk];
    __shared__ unsigned long long s_m[kPairChunk];
    __shared__ uint16_t s_v[kPairChunk];
    __shared__ uint32_t h[kMaxTilePasses][kRadix];
    constexpr int kRun = 8;  // consecutive pairs a thread emits per round
    __shared__ uint32_t s_tk[kEmitThreads * kRun], s_tv[kEmitThreads * kRun];
    const uint32_t n_vis = *n_vis_p;
    const uint32_t n_chunks = (n_vis + kPairChunk - 1) / kPairChunk;
    if (blockIdx.x >= n_chunks) return;  // no drawn record: nothing to emit
    clear_hist(h, tile_passes);
    // persistent over the drawn records' chunks (see pair_count_kernel); the
    // digit histograms gather over all of a block's chunks
    for (uint32_t chunk = blockIdx.x; chunk < n_chunks; chunk += gridDim.x) {
    __syncthreads();  // the previous chunk's shared arrays have been read
    uint32_t r[kPairItems], c[kPairItems];
    chunk_counts(recs, tt, n_vis, chunk, r, c);
    uint64_t sum = 0;
    #pragma unroll
    for (int k = 0; k < kPairItems; k++) sum += c[k];
    uint64_t block_total;
    uint64_t run = block_exclusive_scan_u64(sum, tmp, &block_total);
    #pragma unroll
    for (int k = 0; k < kPairItems; k++) {
        const int q = threadIdx.x * kPairItems + k;
        s_excl[q] = (uint32_t)run;
        run += c[k];
        if (c[k]) {
            const uint2 rr = rect[r[k]];
            s_r0[q] = rr.x;
            s_r1[q] = rr.y;
            s_m[q] = tmask[r[k]];
            s_v[q] = (uint16_t)(r[k] / n);
        }
    }
    if (threadIdx.x == 0) s_excl[kPairChunk] = (uint32_t)block_total;
    __syncthreads();
    const uint64_t base = block_off[chunk];
    const uint32_t j0 = chunk * kPairChunk;
    const uint32_t nq = (uint32_t)block_total;
    // each thread makes kRun consecutive pairs: one search for the first, then
    // a walk along the rectangle's rows (and on to the next records); the
    // round's pairs go out through shared memory so the writes are coalesced
    for (uint32_t q0 = 0; q0 < nq; q0 += kEmitThreads * kRun) {  // block-uniform trip count
        const uint32_t qs = q0 + threadIdx.x * kRun;
        uint32_t tile[kRun];
        bool valid[kRun];
        #pragma unroll
        for (int j = 0; j < kRun; j++) {
            tile[j] = 0;
            valid[j] = false;
        }
        if (qs < nq) {
            // last record i with s_excl[i] <= qs (records of zero count share their successor's offset)
            int lo = 0, hi = kPairChunk;  // invariant: s_excl[lo] <= qs < s_excl[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_excl[mid] <= qs) lo = mid; else hi = mid;
            }
            uint32_t x0, x1, w, tx, row, row0, tiles_x;
            unsigned long long rem;  // kept tiles after the current one (masked records)
            bool masked;
            auto place = [&](uint32_t idx) {  // the idx-th tile of the rectangle, row-major
                const uint32_t ky = idx / w;
                tx = x0 + (idx - ky * w);
                row = row0 + ky * tiles_x;
            };
            auto enter = [&](int rec, uint32_t k) {  // record rec, its k-th pair
                const uint32_t r0 = s_r0[rec], r1 = s_r1[rec];
                x0 = r0 & 0xffff;
                x1 = r1 & 0xffff;
                w = x1 - x0 + 1;
                const uint32_t h = (r1 >> 16) - (r0 >> 16) + 1;
                const ViewInfo &V = vt.v[s_v[rec]];
                tiles_x = (uint32_t)V.tiles_x;
                row0 = (uint32_t)V.tile_base + (r0 >> 16) * tiles_x;
                masked = w * h <= 64;
                uint32_t idx = k;
                rem = 0ull;
                if (masked) {
                    const unsigned long long m = s_m[rec];
                    idx = (uint32_t)nth_set_bit(m, k);
                    rem = idx < 63 ? m & ~((2ull << idx) - 1ull) : 0ull;
                }
                place(idx);
            };
            enter(lo, qs - s_excl[lo]);
            #pragma unroll
            for (int j = 0; j < kRun; j++) {
                const uint32_t q = qs + j;
                if (q >= nq) break;
                if (base + q >= (uint64_t)cap) break;  // dropped: the capacity bit is already set
                if (q >= s_excl[lo + 1]) {  // on to the next record with pairs
                    do {
                        lo++;
                    } while (q >= s_excl[lo + 1]);
                    enter(lo, 0);
                }
                tile[j] = row + tx;
                valid[j] = true;
                s_tk[threadIdx.x * kRun + j] = tile[j];
                s_tv[threadIdx.x * kRun + j] = j0 + (uint32_t)lo;
                if (masked) {
                    if (rem) {
                        place((uint32_t)(__ffsll((long long)rem) - 1));
                        rem &= rem - 1ull;
                    }
                } else if (++tx > x1) {
                    tx = x0;
                    row += tiles_x;
                }
            }
        }
        #pragma unroll
        for (int j = 0; j < kRun; j++) count_digits_warp(h, tile[j], valid[j], tile_passes);
        __syncthreads();
        const uint32_t m = min((uint32_t)(kEmitThreads * kRun), nq - q0);
        for (uint32_t i = threadIdx.x; i < m; i += kEmitThreads) {
            const uint64_t pos = base + q0 + i;
            if (pos >= (uint64_t)cap) break;
            tk[pos] = s_tk[i];
            tv[pos] = s_tv[i];
        }
        __syncthreads();
    }
    }  // chunks
    __syncthreads();
    flush_hist(h, tile_passes, hist);
}

// 4. Each tile's [start, end) from the sorted keys (tiles without pairs keep
// the [0, 0) they were cleared to).
__global__ void __launch_bounds__(256) ranges_kernel(const uint64_t *__restrict__ keys, const uint32_t *n_pairs_p,
                                                     uint32_t cap, uint32_t *ranges)
{
    const uint32_t n = min(*n_pairs_p, cap);
    const uint32_t stride = gridDim.x * blockDim.x;
    #pragma unroll 4
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t t = (uint32_t)(keys[i] >> 32);
        const uint32_t tp = i > 0 ? (uint32_t)(keys[i - 1] >> 32) : ~0u;
        if (tp != t) {
            ranges[2 * t] = i;
            if (i > 0) ranges[2 * tp + 1] = i;
        }
        if (i == n - 1) ranges[2 * t + 1] = n;
    }
}

static int bits_for(int64_t x)  // bits needed to represent x >= 0
{
    int b = 0;
    while (b < 63 && (int64_t(1) << b) <= x) b++;
    return b;
}

struct BinWorkspace {
    uint64_t *block_sums;
    uint32_t *small;  // n_vis, pass counters, depth and tile histograms (cleared together)
    uint32_t *rz[2], *rid[2];
    uint2 *recs;  // depth-sorted (depth bits, record id)
    uint32_t *lb[2];
    uint32_t *pk, *pv;  // pair buffer
    size_t lb_bytes, small_bytes, bytes;
};

static BinWorkspace carve(void *base, int64_t n_records, int64_t cap)
{
    const BinOffsets o = bin_offsets(n_records, cap);
    unsigned char *p = static_cast<unsigned char *>(base);
    BinWorkspace w;
    w.block_sums = reinterpret_cast<uint64_t *>(p + o.block_sums);
    w.small = reinterpret_cast<uint32_t *>(p + o.small);
    w.small_bytes = o.small_bytes;
    for (int i = 0; i < 2; i++) {
        w.rz[i] = reinterpret_cast<uint32_t *>(p + o.rz[i]);
        w.rid[i] = reinterpret_cast<uint32_t *>(p + o.rid[i]);
        w.lb[i] = reinterpret_cast<uint32_t *>(p + o.lb[i]);
    }
    w.recs = reinterpret_cast<uint2 *>(p + o.recs);
    w.lb_bytes = o.lb_bytes;
    w.pk = reinterpret_cast<uint32_t *>(p + o.pk);
    w.pv = reinterpret_cast<uint32_t *>(p + o.pv);
    w.bytes = o.bytes;
    return w;
}

}  // namespace gs

using namespace gs;

extern "C" size_t gs_bin_sort_workspace_size(int64_t n_records, int64_t pair_capacity, int64_t n_tiles_total)
{
    (void)n_tiles_total;
    if (n_records < 0 || pair_capacity < 1) return 0;
    return bin_offsets(n_records > 0 ? n_records : 1, pair_capacity).bytes;
}

extern "C" gs_status_t gs_bin_sort(const gs_projected_t *proj, int64_t n, const gs_view_t *views, int32_t n_views,
                                   gs_bins_t *bins, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!proj || !bins || n < 0) return GS_ERR_INVALID_ARG;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    const int64_t cap = bins->capacity;
    if (cap < 1 || cap >= (int64_t(1) << 30)) return GS_ERR_INVALID_ARG;
    if (!bins->keys || !bins->vals || !bins->ranges || !bins->n_pairs || !bins->status || !workspace)
        return GS_ERR_INVALID_ARG;
    const int64_t total = (int64_t)n_views * n;
    if (total >= (int64_t(1) << 32)) return GS_ERR_INVALID_ARG;  // record ids are 32-bit
    BinWorkspace w = carve(workspace, total > 0 ? total : 1, cap);
    if (workspace_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return GS_ERR_INVALID_ARG;
    const int tile_passes = (bits_for(vt.n_tiles_total - 1) + 7) / 8 > 0 ? (bits_for(vt.n_tiles_total - 1) + 7) / 8 : 1;
    if (tile_passes > kMaxTilePasses) return GS_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(bins->ranges, 0, sizeof(uint32_t) * 2 * (size_t)vt.n_tiles_total, s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (total == 0) {
        if (cudaMemsetAsync(bins->n_pairs, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
        return GS_OK;
    }
    if (!proj->rec || !proj->rect || !proj->tiles_touched || !proj->tile_mask) return GS_ERR_INVALID_ARG;

    uint32_t *n_vis = w.small;
    uint32_t *counters = w.small + 1;  // one per pass
    uint32_t *hist_depth = counters + kDepthPasses + kMaxTilePasses;
    uint32_t *hist_tile = hist_depth + kDepthPasses * kRadix;
    if (cudaMemsetAsync(w.small, 0, w.small_bytes, s) != cudaSuccess) return GS_ERR_CUDA;
    if (cudaMemsetAsync(w.lb[0], 0, w.lb_bytes, s) != cudaSuccess) return GS_ERR_CUDA;

    // 1. drawn records sorted by depth
    const unsigned nb = (unsigned)((total + kEmitChunk - 1) / kEmitChunk);
    vis_count_kernel<<<nb, kEmitThreads, 0, s>>>(proj->tiles_touched, total, w.block_sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(w.block_sums, nb, total, n_vis, bins->status, nullptr, 1);
    vis_compact_kernel<<<nb, kEmitThreads, 0, s>>>(proj->rec, proj->tiles_touched, total, w.block_sums, w.rz[0],
                                                   w.rid[0], hist_depth);
    for (int p = 0; p < kDepthPasses; p++) {
        const int a = p & 1;
        const bool last = p + 1 == kDepthPasses;  // writes (depth bits, record id) pairs
        st = onesweep_pass(w.rz[a], w.rid[a], last ? reinterpret_cast<uint32_t *>(w.recs) : w.rz[a ^ 1],
                           w.rid[a ^ 1], n_vis, total, hist_depth + p * kRadix, w.lb[a], last ? nullptr : w.lb[a ^ 1],
                           counters + p, 8 * p, last ? kSortPaired : kSortPlain, nullptr, bins->status, s);
        if (st != GS_OK) return st;
    }

    // 2. pairs in depth order; the last tile pass reads the workspace buffer,
    // so emission goes where the pass count puts it (the key array doubles
    // as the other buffer)
    uint32_t *buf_k[2] = {w.pk, reinterpret_cast<uint32_t *>(bins->keys)};
    uint32_t *buf_v[2] = {w.pv, reinterpret_cast<uint32_t *>(bins->keys) + cap};
    const int e = (tile_passes & 1) ? 0 : 1;
    // chunks of the drawn records: at most np, known on the device only; both
    // kernels are persistent over them with grids sized to the GPU
    const unsigned np = (unsigned)((total + kPairChunk - 1) / kPairChunk);
    const unsigned pgrid = (unsigned)(np < (unsigned)num_sms() * 8u ? np : (unsigned)num_sms() * 8u);
    pair_count_kernel<<<pgrid, kEmitThreads, 0, s>>>(w.recs, proj->tiles_touched, n_vis, w.block_sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(w.block_sums, np, cap, bins->n_pairs, bins->status, n_vis, kPairChunk);
    pair_emit_kernel<<<pgrid, kEmitThreads, 0, s>>>(w.recs, reinterpret_cast<const uint2 *>(proj->rect),
                                                  reinterpret_cast<const unsigned long long *>(proj->tile_mask),
                                                 proj->tiles_touched, n_vis, (uint32_t)n, vt, w.block_sums, cap,
                                                 buf_k[e], buf_v[e], hist_tile, tile_passes);
    st = launch_status();
    if (st != GS_OK) return st;

    // 3. stable passes over the tile id; the last writes keys and values
    if (cudaMemsetAsync(w.lb[0], 0, w.lb_bytes, s) != cudaSuccess) return GS_ERR_CUDA;
    const SortExpand ex = {bins->keys, bins->vals, w.recs, (uint32_t)n};
    int src = e;
    for (int p = 0; p < tile_passes; p++) {
        const bool last = p + 1 == tile_passes;
        const int a = p & 1;
        st = onesweep_pass(buf_k[src], buf_v[src], buf_k[src ^ 1], buf_v[src ^ 1], bins->n_pairs, cap,
                           hist_tile + p * kRadix, w.lb[a], last ? nullptr : w.lb[a ^ 1],
                           counters + kDepthPasses + p, 8 * p, last ? kSortExpand : kSortPlain, &ex, bins->status, s);
        if (st != GS_OK) return st;
        src ^= 1;
    }

    // 4. tile ranges
    const int64_t rb = (cap + 255) / 256, rmax = (int64_t)num_sms() * 16;
    ranges_kernel<<<(unsigned)(rb < rmax ? rb : rmax), 256, 0, s>>>(bins->keys, bins->n_pairs, (uint32_t)cap, bins->ranges);
    return launch_status();
}

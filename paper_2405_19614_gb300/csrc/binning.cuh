// Block shapes of the binning kernels and the layout of gs_bin_sort's
// workspace, shared by binning.cu and the allocation-free entry point (which
// sizes its fixed scratch array from this layout at compile time).
#pragma once

#include <cstddef>
#include <cstdint>

#include "sort.cuh"

namespace gs {

constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitChunk = kEmitThreads * kEmitItems;  // records per block, compaction
constexpr int kPairItems = 2;
constexpr int kPairChunk = kEmitThreads * kPairItems;  // sorted records per block, pair emission
constexpr int kDepthPasses = 4;
constexpr int kMaxTilePasses = 4;
constexpr int kSmallWords = 1 + kDepthPasses + kMaxTilePasses + (kDepthPasses + kMaxTilePasses) * kRadix;

// Byte offsets of the workspace regions for n_records (view, Gaussian)
// records and a pair capacity cap, each region 256-byte aligned: scan block
// sums; the small counters and histograms; two ping-pong buffers of the drawn
// records' depth keys and ids; their depth-sorted (depth, id) pairs; two
// look-back regions; the (tile id, depth rank) pair buffer.
struct BinOffsets {
    size_t block_sums = 0, small = 0, small_bytes = 0;
    size_t rz[2] = {0, 0}, rid[2] = {0, 0};
    size_t recs = 0, lb_bytes = 0;
    size_t lb[2] = {0, 0};
    size_t pk = 0, pv = 0, bytes = 0;
};

constexpr BinOffsets bin_offsets(int64_t n_records, int64_t cap)
{
    BinOffsets o;
    const int64_t nb = (n_records + kPairChunk - 1) / kPairChunk + 1;  // the larger of the two block counts
    size_t off = 0;
    o.block_sums = off;
    off += align256(sizeof(uint64_t) * (size_t)nb);
    o.small = off;
    o.small_bytes = sizeof(uint32_t) * kSmallWords;
    off += align256(o.small_bytes);
    for (int i = 0; i < 2; i++) {
        o.rz[i] = off;
        off += align256(sizeof(uint32_t) * (size_t)n_records);
        o.rid[i] = off;
        off += align256(sizeof(uint32_t) * (size_t)n_records);
    }
    o.recs = off;
    off += align256(2 * sizeof(uint32_t) * (size_t)n_records);
    o.lb_bytes = onesweep_lookback_bytes(n_records > cap ? n_records : cap);
    for (int i = 0; i < 2; i++) {
        o.lb[i] = off;
        off += o.lb_bytes;
    }
    o.pk = off;
    off += align256(sizeof(uint32_t) * (size_t)cap);
    o.pv = off;
    off += align256(sizeof(uint32_t) * (size_t)cap);
    o.bytes = off;
    return o;
}

}  // namespace gs

// Internal interface of the onesweep radix sort (sort.cu).
#pragma once

#include "common.cuh"

namespace gs {

constexpr int kMaxSortPasses = 8;

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Workspace bytes for a sort of up to cap pairs.
size_t sort_workspace_bytes(int64_t cap);

// Number of 8-bit digit passes for n_bits significant key bits.
int sort_passes(int n_bits);

// Sorts min(*n_pairs, cap) pairs starting in (keys_a, vals_a), ping-ponging
// with (keys_b, vals_b); the result lands in _a when the number of passes is
// even and in _b when it is odd.
gs_status_t radix_sort_pairs(uint64_t *keys_a, uint32_t *vals_a, uint64_t *keys_b, uint32_t *vals_b,
                             const uint32_t *n_pairs, int64_t cap, int n_bits, void *ws, uint32_t *status,
                             cudaStream_t s);

}  // namespace gs

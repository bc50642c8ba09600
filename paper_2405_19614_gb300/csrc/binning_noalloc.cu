// Allocation-free variant of gs_bin_sort (the paper has no counterpart; this is
// a service for callers that cannot allocate device memory).
//
// gs_bin_sort needs a scratch workspace (the scans' block sums, the drawn
// records' depth keys and ids with their second sort buffer, the look-back
// flags and histograms of the radix passes, and the second pair buffer).  Normally the caller allocates
// it.  Some callers cannot: code that is capturing a CUDA graph cannot call
// cudaMalloc in the middle of the capture, a fixed-rate tracking loop on a robot cannot afford the device
// synchronisation an allocation may cause, and some host frameworks own every
// byte of device memory and hand a plugin only its inputs and outputs.  For
// them this file keeps the scratch in one file-scope device array of fixed
// size, reserved when the library is loaded on a GPU and held until the
// process exits.
//
// Limits: at most kNoAllocMaxRecords (view, Gaussian) records (n_views * n)
// and a pair capacity of at most kNoAllocMaxPairs (2,097,152 each); larger
// calls are rejected with GS_ERR_CAPACITY before anything is enqueued.  The
// array is exactly the workspace gs_bin_sort needs at both limits (about
// 65 MiB), computed at compile time from the same layout, so every call
// within the limits fits.
//
// Sharing: every call uses the same array and it keeps the previous call's
// contents.  Everything the sort needs at zero is cleared inside the call, so
// successive calls on one stream are independent; calls that can overlap on
// the GPU (different streams, or different host threads without ordering)
// race on the array and must not be issued.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current (host code cannot use
// the array's name as a device pointer).  Make that first call before any
// stream capture begins, so the capture only records kernel launches.
#include <mutex>

#include "binning.cuh"
#include "common.cuh"

namespace gs {

constexpr int64_t kNoAllocMaxRecords = int64_t(1) << 21;  // 2,097,152 records
constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 21;    // 2,097,152 pairs
// the workspace layout is monotone in both sizes, so its size at the limits
// bounds every call within them
constexpr size_t kNoAllocScratchBytes = bin_offsets(kNoAllocMaxRecords, kNoAllocMaxPairs).bytes;
static_assert(kNoAllocScratchBytes <= (size_t(66) << 20), "the fixed scratch array stays about 65 MiB");
static_assert(kNoAllocScratchBytes % 256 == 0, "whole 256-byte regions");

static __device__ __align__(256) unsigned char g_bin_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
static void *g_scratch_ptr[kNoAllocMaxDevices];
static std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once).
static gs_status_t scratch_for_current_device(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return GS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess || !p) return GS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" gs_status_t gs_bin_sort_noalloc(const gs_projected_t *proj, int64_t n, const gs_view_t *views,
                                           int32_t n_views, gs_bins_t *bins, void *stream)
{
    if (!proj || !bins || n < 0 || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    const int64_t records = (int64_t)n_views * n;
    if (records > kNoAllocMaxRecords || bins->capacity > kNoAllocMaxPairs) return GS_ERR_CAPACITY;
    ViewTable vt;
    gs_status_t st = make_view_table(views, n_views, &vt);
    if (st != GS_OK) return st;
    const size_t need = gs_bin_sort_workspace_size(records, bins->capacity, vt.n_tiles_total);
    if (need == 0) return GS_ERR_INVALID_ARG;
    if (need > kNoAllocScratchBytes) return GS_ERR_CAPACITY;
    void *scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != GS_OK) return st;
    return gs_bin_sort(proj, n, views, n_views, bins, scratch, kNoAllocScratchBytes, stream);
}

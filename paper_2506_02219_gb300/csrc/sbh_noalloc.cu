// sbh_noalloc.cu -- sbh_morton_sort_noalloc: the Morton ordering step of the tree build for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or any allocating routine: real-time loops where the
// implicit synchronisation of an allocation is not acceptable, and host applications that hand a
// library a fixed device-memory budget up front and own every allocation themselves. For them
// this entry point orders points exactly as sbh_build does (same codes, same stable order) using
// only the caller's input and output buffers plus one scratch array of fixed size that lives in
// this library's static device memory.
//
// The scratch array is a file-scope __device__ array; every GPU that loads the library holds it
// until the process exits. Host code cannot use the array's name as a device address, so every
// call looks up its address with cudaGetSymbolAddress in the current device's context (a lookup,
// no allocation). The address is not cached: it belongs to the context it was taken in, and a
// cudaDeviceReset or another context on the same device would leave a cached one stale. The first
// call on a device also loads this module's device code there.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "sbh.h"
#include "sbh_build.cuh"
#include "sbh_sort.cuh"

namespace sbh {

namespace {

constexpr int64_t kNoAllocMaxPoints = SBH_NOALLOC_MAX_POINTS;
constexpr int kNoAllocMaxTiles = (int)((kNoAllocMaxPoints + kSortTile - 1) / kSortTile);

constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// layout of the scratch array
constexpr size_t kOffKeys = 0;                                                            // u64 [max]
constexpr size_t kOffVals = kOffKeys + round256(sizeof(uint64_t) * kNoAllocMaxPoints);    // i32 [max]
constexpr size_t kOffHist = kOffVals + round256(sizeof(int32_t) * kNoAllocMaxPoints);     // i32 [256 x tiles]
constexpr size_t kHistInts = (size_t)256 * kNoAllocMaxTiles;
constexpr size_t kScanTempInts = kHistInts / 2048 + 16;                                   // >= scan_temp_ints
constexpr size_t kOffScan = kOffHist + round256(sizeof(int) * kHistInts);
constexpr size_t kOffBounds = kOffScan + round256(sizeof(int) * kScanTempInts);          // i32 [8]
constexpr size_t kOffCtrl = kOffBounds + round256(sizeof(int) * 8);                       // TreeCtrl [2]
constexpr size_t kScratchBytes = kOffCtrl + round256(2 * sizeof(TreeCtrl));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

}  // namespace

}  // namespace sbh

extern "C" {

sbh_status sbh_morton_sort_noalloc(const float* points, int64_t n, uint64_t* codes, int32_t* perm, void* stream)
{
    using namespace sbh;
    set_error_message("");
    if (n < 1 || n > kNoAllocMaxPoints) {
        set_error_message("sbh_morton_sort_noalloc: n = %lld outside [1, %lld] (SBH_NOALLOC_MAX_POINTS)", (long long)n,
                          (long long)kNoAllocMaxPoints);
        return SBH_EINVAL;
    }
    if (!points || !codes || !perm) {
        set_error_message("sbh_morton_sort_noalloc: points, codes and perm must be non-NULL");
        return SBH_EINVAL;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        set_error_message("sbh_morton_sort_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return SBH_ECUDA;
    }
    unsigned char* base = (unsigned char*)p;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* keys_tmp = (uint64_t*)(base + kOffKeys);
    int32_t* vals_tmp = (int32_t*)(base + kOffVals);
    int* hist = (int*)(base + kOffHist);
    int* scan_tmp = (int*)(base + kOffScan);
    int* bounds = (int*)(base + kOffBounds);
    TreeCtrl* ctrl = (TreeCtrl*)(base + kOffCtrl);

    const unsigned grid = (unsigned)((n + 255) / 256 < 2432 ? (n + 255) / 256 : 2432);
    k_bounds_init<<<1, 32, 0, s>>>(bounds);  // every call starts the min/max from scratch
    note_launch();
    // the weight count of k_bounds is not used here; the points array stands in for the weights
    // (it has 3n floats, so the n reads stay inside it)
    k_bounds<<<grid, 256, 0, s>>>(points, points, n, bounds);
    note_launch();
    k_root_cube<<<1, 32, 0, s>>>(bounds, ctrl, ctrl + 1);
    note_launch();
    // ping-pong between the caller's outputs and the scratch copy: 8 passes end in the outputs
    uint64_t* k0 = codes;
    int32_t* v0 = perm;
    uint64_t* k1 = keys_tmp;
    int32_t* v1 = vals_tmp;
    k_morton<<<grid, 256, 0, s>>>(points, n, ctrl, k0, v0);
    note_launch();
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t nhist = (int64_t)256 * ntiles;
    for (int pass = 0; pass < 8; ++pass) {
        k_radix_hist<<<ntiles, kSortThreads, 0, s>>>(k0, n, 8 * pass, ntiles, hist);
        note_launch();
        scan_exclusive(hist, hist, nhist, scan_tmp, s);
        k_radix_scatter<<<ntiles, kSortThreads, 0, s>>>(k0, v0, n, 8 * pass, ntiles, hist, k1, v1);
        note_launch();
        uint64_t* tk = k0; k0 = k1; k1 = tk;
        int32_t* tv = v0; v0 = v1; v1 = tv;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error_message("sbh_morton_sort_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
        return SBH_ECUDA;
    }
    return SBH_OK;
}

}  // extern "C"

// sbh_sort.cuh -- the Morton-code and radix-sort kernels of the tree build (defined in
// sbh_build.cu), declared for the other translation units that launch them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_internal.cuh"

namespace sbh {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// scratch: [0..2] per-axis min (ordered int), [3..5] max, [6] bad coordinates, [7] bad weights
__global__ void k_bounds_init(int* scratch);
__global__ void k_bounds(const float* __restrict__ pts, const float* __restrict__ w, int64_t n,
                         int* __restrict__ scratch);
__global__ void k_root_cube(const int* __restrict__ scratch, TreeCtrl* c4, TreeCtrl* c2);
__global__ void k_morton(const float* __restrict__ pts, int64_t n, const TreeCtrl* __restrict__ c4,
                         uint64_t* __restrict__ code, int32_t* __restrict__ idx);
__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int ntiles,
                             int* __restrict__ hist);
__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n,
                                int shift, int ntiles, const int* __restrict__ offsets,
                                uint64_t* __restrict__ kout, int32_t* __restrict__ vout);

}  // namespace sbh

// sbh_build.cuh -- the library-owned tree object and the host-side build steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_internal.cuh"

namespace sbh {

// Device arrays of one tree (capacity `cap` nodes; at most 2n - 1 are used).
struct DeviceTree {
    int64_t cap = 0;
    int max_level = 0;   // 10 (64-ary) or 20 (8-ary)
    int level_shift = 0; // log2 of the per-dimension branching d: 2 or 1
    float4* pm = nullptr;
    float4* dip = nullptr;
    float4* pmd = nullptr;   // [cap][2]: pm and dip interleaved (the estimator's tree with normals)
    float* cdf = nullptr;
    uint8_t* gd = nullptr;
    int32_t* fc = nullptr;
    uint32_t* meta = nullptr;
    int32_t* nb = nullptr;
    int32_t* ne = nullptr;
    int32_t* parent = nullptr;
    int32_t* skip = nullptr;
    int32_t* minl = nullptr;
    double* agg = nullptr;   // [cap][8] FP64: m, m p (3), m n (3), 0
    TreeCtrl* ctrl = nullptr;
    bool built = false;

    TreeView view() const
    {
        TreeView v;
        v.pm = pm; v.dip = dip; v.pmd = pmd; v.cdf = cdf; v.gd = gd; v.fc = fc; v.meta = meta; v.nb = nb; v.ne = ne;
        v.skip = skip; v.ctrl = ctrl;
        return v;
    }
};

// stream-ordered device allocation: the library's memory pool or the caller's allocator
cudaError_t dalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);
void set_allocator(sbh_alloc_fn a, sbh_free_fn f, void* ctx);
void set_memory_limit(uint64_t bytes);
uint64_t memory_in_use();

int64_t scan_temp_ints(int64_t n);
void scan_exclusive(const int* in, int* out, int64_t n, int* temp, cudaStream_t s);

}  // namespace sbh

// The opaque tree handle of the C ABI.
struct sbh_tree {
    int64_t n = 0;
    int32_t leaf_size = 1;
    int32_t has_normals = 0;
    int device = 0;
    cudaStream_t stream = nullptr;   // stream of the last build step
    uint64_t* code = nullptr;        // sorted Morton codes
    int32_t* perm = nullptr;         // input index of each sorted point
    float4* spw = nullptr;           // sorted (x, y, z, m)
    float4* snrm = nullptr;          // sorted normals or nullptr
    uint8_t* lcp4 = nullptr;         // shared code digits of neighbours, 6-bit digits
    uint8_t* lcp2 = nullptr;         // the same, 3-bit digits
    sbh::DeviceTree t4;              // 64-ary tree (estimator)
    sbh::DeviceTree t2;              // 8-ary tree (Barnes-Hut), built on demand
    sbh::TreeCtrl host_ctrl4;        // host copy of t4.ctrl, read when sbh_build finishes
};

namespace sbh {
// Enqueue the topology, aggregate and packing steps of one tree on `s`.
cudaError_t build_tree(sbh_tree* T, DeviceTree& D, const uint8_t* lcp, int max_level, int level_shift,
                       bool with_skip, cudaStream_t s);
// Enqueue validation (sets *bad on the host after a sync), root cube, codes, sort and gather.
cudaError_t build_sorted(sbh_tree* T, const float* pts, const float* w, const float* nrm, cudaStream_t s,
                         int* bad_points, int* bad_weights);
cudaError_t alloc_tree(DeviceTree& D, int64_t n, bool with_dip, bool with_skip, bool with_rec, cudaStream_t s);
void free_tree(DeviceTree& D, cudaStream_t s);
}  // namespace sbh

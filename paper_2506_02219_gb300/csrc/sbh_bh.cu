// sbh_bh.cu -- deterministic Barnes-Hut (Madan et al. 2025, Sec. 3.1, Eq. 2, Algorithm 1) on
// the 8-ary tree, the GPU baseline the estimator is compared with.
//
// A node is used whole -- m_a f(p_a, q) added -- when it is a source point or its far-field ratio
// ||q - p_a|| / |B_a| >= beta; otherwise the walk enters its first child. The walk is stackless:
// after a node is used it continues at skip[node], the next node of a depth-first order after
// that node's subtree (its next sibling, else its parent's skip). With warp voting the 32 queries
// of a warp walk together: a node is opened when any of them needs it, so every lane reads the
// same node (one broadcast load) and no lane diverges; the sum only gets more accurate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_eval.cuh"

namespace sbh {

template <int KIND>
__device__ __forceinline__ void bh_add(const TreeView& T, int32_t v, float4 p, float3 q, const KernelParams& kp,
                                       float& acc, ExpAcc& ex)
{
    if constexpr (KIND == SBH_COULOMB) acc += term_coulomb(p, q, kp.eps2);
    else if constexpr (KIND == SBH_WINDING) acc += term_winding(p, __ldg(&T.dip[v]), q);
    else if constexpr (KIND == SBH_AFFINE) acc += term_affine(p, q, kp.g);
    else {
        const float d = dist_fast(p, q);
        ex.lower(d, kp.alpha);
        ex.acc = fmaf(p.w, ex.scale(d, kp.alpha), ex.acc);
    }
}

template <int KIND, bool VOTE>
__global__ void __launch_bounds__(256) k_bh_eval(TreeView T, const float* __restrict__ Q, int64_t nq, KernelParams kp,
                                                 float beta, float* __restrict__ out)
{
    __shared__ float sdiam[kDiamLevels];
    if (threadIdx.x < kDiamLevels) sdiam[threadIdx.x] = T.ctrl->diam[threadIdx.x];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int32_t n_nodes = T.ctrl->n_nodes;
    // the loop bound is warp-uniform so that voting warps stay converged
    const int64_t warp_base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31);
    for (int64_t jb = warp_base; jb < nq; jb += stride) {
        const int64_t j = jb + (threadIdx.x & 31);
        const bool active = j < nq;
        const float3 q = active ? make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]) : make_float3(0.f, 0.f, 0.f);
        float acc = 0.0f;
        ExpAcc ex;
        ex.init(3.0e38f);
        int32_t v = 0;
        // a depth-first walk enters every node at most once; the bound only guards a damaged tree
        int32_t budget = n_nodes + 1;
        if (VOTE || active) {
            while (v >= 0 && budget-- > 0) {
                const float4 p = __ldg(&T.pm[v]);
                const uint32_t m = __ldg(&T.meta[v]);
                bool use = meta_kind(m) == kPoint;
                if (!use) use = __fdiv_rn(dist_rn(p.x, p.y, p.z, q), sdiam[meta_level(m)]) >= beta;
                if (VOTE) use = __all_sync(0xFFFFFFFFu, use || !active);
                if (use) {
                    if (active) bh_add<KIND>(T, v, p, q, kp, acc, ex);
                    v = __ldg(&T.skip[v]);
                } else {
                    v = __ldg(&T.fc[v]);
                }
            }
        }
        if (v >= 0) acc = ex.acc = __int_as_float(0x7FC00000);  // walk did not finish: NaN
        if (active) {
            if constexpr (KIND == SBH_SMOOTHDIST)
                out[j] = ex.acc > 0.0f ? ex.ref - __logf(ex.acc) / kp.alpha : __int_as_float(0x7F800000);
            else out[j] = acc;
        }
    }
}

template <int KIND>
static void launch_bh_kind(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, float beta,
                           int vote, float* out, cudaStream_t s, unsigned blocks)
{
    if (vote) k_bh_eval<KIND, true><<<blocks, 256, 0, s>>>(T, Q, nq, kp, beta, out);
    else k_bh_eval<KIND, false><<<blocks, 256, 0, s>>>(T, Q, nq, kp, beta, out);
    note_launch();
}

cudaError_t launch_bh_eval(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, float beta,
                           int warp_vote, float* out, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    int64_t blocks = (nq + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 64;
    if (blocks > cap) blocks = cap;
    switch (kp.kind) {
    case SBH_COULOMB: launch_bh_kind<SBH_COULOMB>(T, Q, nq, kp, beta, warp_vote, out, s, (unsigned)blocks); break;
    case SBH_WINDING: launch_bh_kind<SBH_WINDING>(T, Q, nq, kp, beta, warp_vote, out, s, (unsigned)blocks); break;
    case SBH_SMOOTHDIST: launch_bh_kind<SBH_SMOOTHDIST>(T, Q, nq, kp, beta, warp_vote, out, s, (unsigned)blocks); break;
    case SBH_AFFINE: launch_bh_kind<SBH_AFFINE>(T, Q, nq, kp, beta, warp_vote, out, s, (unsigned)blocks); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sbh

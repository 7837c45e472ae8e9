// sbh_brute.cu -- the exact kernel sum F(q) = sum_i m_i f(p_i, q) (Madan et al. 2025, Eq. 1) by
// tiled brute force: each block stages a tile of sources in shared memory and every thread sums
// the tile for its query (the classic all-pairs layout the paper uses for ground truth, Sec. 4.3).
// With fp64_accum each tile's FP32 partial sum is added into an FP64 accumulator, which keeps
// the rounding error of million-term sums at the level of one tile; this is the error reference.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_eval.cuh"

namespace sbh {

constexpr int kBruteThreads = 256;
constexpr int kBruteTile = 256;

template <int KIND, bool FP64>
__global__ void __launch_bounds__(kBruteThreads) k_brute(const float* __restrict__ P, const float* __restrict__ W,
                                                         const float* __restrict__ N, int64_t n,
                                                         const float* __restrict__ Q, int64_t nq, KernelParams kp,
                                                         float* __restrict__ out)
{
    __shared__ float4 spm[kBruteTile];
    __shared__ float4 sdp[KIND == SBH_WINDING ? kBruteTile : 1];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = j < nq;
    const float3 q = active ? make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]) : make_float3(0.f, 0.f, 0.f);
    double acc64 = 0.0;
    float acc32 = 0.0f;
    // smooth distance: sum = (acc64 + part) * exp(-alpha * ref), ref = smallest distance so far
    float ref = 3.0e38f;
    for (int64_t t0 = 0; t0 < n; t0 += kBruteTile) {
        const int cnt = (n - t0) < kBruteTile ? (int)(n - t0) : kBruteTile;
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int64_t i = t0 + threadIdx.x;
            spm[threadIdx.x] = make_float4(P[3 * i], P[3 * i + 1], P[3 * i + 2], W[i]);
            if constexpr (KIND == SBH_WINDING) {
                const float w = W[i];
                sdp[threadIdx.x] = make_float4(w * N[3 * i], w * N[3 * i + 1], w * N[3 * i + 2], 0.0f);
            }
        }
        __syncthreads();
        float part = 0.0f;
        if constexpr (KIND == SBH_SMOOTHDIST) {
            for (int k = 0; k < cnt; ++k) {
                const float4 p = spm[k];
                const float d = dist_fast(p, q);
                if (d < ref) {
                    const float f = __expf(-kp.alpha * (ref - d));
                    part *= f;
                    if (FP64) acc64 *= (double)f; else acc32 *= f;
                    ref = d;
                }
                part = fmaf(p.w, __expf(-kp.alpha * (d - ref)), part);
            }
        } else {
#pragma unroll 8
            for (int k = 0; k < cnt; ++k) {
                const float4 p = spm[k];
                if constexpr (KIND == SBH_COULOMB) part += term_coulomb(p, q, kp.eps2);
                else if constexpr (KIND == SBH_WINDING) part += term_winding(p, sdp[k], q);
                else part += term_affine(p, q, kp.g);
            }
        }
        if (FP64) acc64 += (double)part; else acc32 += part;
    }
    if (!active) return;
    const double total = FP64 ? acc64 : (double)acc32;
    if constexpr (KIND == SBH_SMOOTHDIST)
        out[j] = total > 0.0 ? (float)((double)ref - log(total) / (double)kp.alpha) : __int_as_float(0x7F800000);
    else out[j] = (float)total;
}

template <int KIND>
static void launch_brute_kind(const float* P, const float* W, const float* N, int64_t n, const float* Q, int64_t nq,
                              const KernelParams& kp, int fp64, float* out, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((nq + kBruteThreads - 1) / kBruteThreads);
    if (fp64) k_brute<KIND, true><<<blocks, kBruteThreads, 0, s>>>(P, W, N, n, Q, nq, kp, out);
    else k_brute<KIND, false><<<blocks, kBruteThreads, 0, s>>>(P, W, N, n, Q, nq, kp, out);
    note_launch();
}

cudaError_t launch_brute(const float* P, const float* W, const float* N, int64_t n, const float* Q, int64_t nq,
                         const KernelParams& kp, int fp64_accum, float* out, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    switch (kp.kind) {
    case SBH_COULOMB: launch_brute_kind<SBH_COULOMB>(P, W, N, n, Q, nq, kp, fp64_accum, out, s); break;
    case SBH_WINDING: launch_brute_kind<SBH_WINDING>(P, W, N, n, Q, nq, kp, fp64_accum, out, s); break;
    case SBH_SMOOTHDIST: launch_brute_kind<SBH_SMOOTHDIST>(P, W, N, n, Q, nq, kp, fp64_accum, out, s); break;
    case SBH_AFFINE: launch_brute_kind<SBH_AFFINE>(P, W, N, n, Q, nq, kp, fp64_accum, out, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sbh

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

// The exact sum and its query gradient: per tile FP32 partials of the value and of the three
// gradient components, added into FP64 accumulators (the smooth distance in the frame
// exp(-alpha ref) of the smallest distance so far, as above). Outputs follow sbh_eval_grad:
// the smooth distance returns d = ref - log(acc) / alpha and grad d = -grad acc / (alpha acc).
template <int KIND>
__global__ void __launch_bounds__(kBruteThreads) k_brute_grad(const float* __restrict__ P, const float* __restrict__ W,
                                                              const float* __restrict__ N, int64_t n,
                                                              const float* __restrict__ Q, int64_t nq, KernelParams kp,
                                                              float* __restrict__ out, float* __restrict__ grad)
{
    __shared__ float4 spm[kBruteTile];
    __shared__ float4 sdp[KIND == SBH_WINDING ? kBruteTile : 1];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = j < nq;
    const float3 q = active ? make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]) : make_float3(0.f, 0.f, 0.f);
    double a64 = 0.0, g64[3] = {0.0, 0.0, 0.0};
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
        float v = 0.0f, g[3] = {0.0f, 0.0f, 0.0f};
        for (int k = 0; k < cnt; ++k) {
            const float4 pm = spm[k];
            const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
            if constexpr (KIND == SBH_COULOMB) {
                const float e = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kp.eps2)));
                const float ir = rsqrt_ftz(e);
                const float t = pm.w * ir;
                const float c = t * ir * ir;
                v += t;
                g[0] = fmaf(c, dx, g[0]); g[1] = fmaf(c, dy, g[1]); g[2] = fmaf(c, dz, g[2]);
            } else if constexpr (KIND == SBH_WINDING) {
                const float4 D = sdp[k];
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 >= kMinNormal) {
                    const float ir = rsqrt_ftz(r2);
                    const float ir3 = ir * ir * ir;
                    const float dn = fmaf(dx, D.x, fmaf(dy, D.y, dz * D.z));
                    v = fmaf(kInv4Pi * dn, ir3, v);
                    const float c = 3.0f * kInv4Pi * dn * ir3 * ir * ir;
                    const float b = -kInv4Pi * ir3;
                    g[0] += fmaf(b, D.x, c * dx); g[1] += fmaf(b, D.y, c * dy); g[2] += fmaf(b, D.z, c * dz);
                }
            } else if constexpr (KIND == SBH_SMOOTHDIST) {
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float ir = rsqrt_ftz(fmaxf(r2, 1e-37f));
                const float r = r2 * ir;
                if (r < ref) {
                    const float f = __expf(-kp.alpha * (ref - r));
                    const double f64 = (double)f;
                    v *= f; g[0] *= f; g[1] *= f; g[2] *= f;
                    a64 *= f64; g64[0] *= f64; g64[1] *= f64; g64[2] *= f64;
                    ref = r;
                }
                const float t = pm.w * __expf(-kp.alpha * (r - ref));
                v += t;
                if (r2 > 0.0f) {
                    const float c = kp.alpha * t * ir;
                    g[0] = fmaf(c, dx, g[0]); g[1] = fmaf(c, dy, g[1]); g[2] = fmaf(c, dz, g[2]);
                }
            } else {
                v = fmaf(pm.w, 1.0f + fmaf(kp.g[0], dx, fmaf(kp.g[1], dy, kp.g[2] * dz)), v);
                g[0] -= pm.w * kp.g[0]; g[1] -= pm.w * kp.g[1]; g[2] -= pm.w * kp.g[2];
            }
        }
        a64 += (double)v;
        g64[0] += (double)g[0]; g64[1] += (double)g[1]; g64[2] += (double)g[2];
    }
    if (!active) return;
    if constexpr (KIND == SBH_SMOOTHDIST) {
        const bool pos = a64 > 0.0;
        out[j] = pos ? (float)((double)ref - log(a64) / (double)kp.alpha) : __int_as_float(0x7F800000);
        const double c = pos ? -1.0 / ((double)kp.alpha * a64) : 0.0;
        for (int a = 0; a < 3; ++a) grad[3 * j + a] = pos ? (float)(c * g64[a]) : __int_as_float(0x7FC00000);
    } else {
        out[j] = (float)a64;
        for (int a = 0; a < 3; ++a) grad[3 * j + a] = (float)g64[a];
    }
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

cudaError_t launch_brute_grad(const float* P, const float* W, const float* N, int64_t n, const float* Q, int64_t nq,
                              const KernelParams& kp, float* out, float* grad, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    const unsigned b = (unsigned)((nq + kBruteThreads - 1) / kBruteThreads);
    switch (kp.kind) {
    case SBH_COULOMB: k_brute_grad<SBH_COULOMB><<<b, kBruteThreads, 0, s>>>(P, W, N, n, Q, nq, kp, out, grad); break;
    case SBH_WINDING: k_brute_grad<SBH_WINDING><<<b, kBruteThreads, 0, s>>>(P, W, N, n, Q, nq, kp, out, grad); break;
    case SBH_SMOOTHDIST: k_brute_grad<SBH_SMOOTHDIST><<<b, kBruteThreads, 0, s>>>(P, W, N, n, Q, nq, kp, out, grad); break;
    case SBH_AFFINE: k_brute_grad<SBH_AFFINE><<<b, kBruteThreads, 0, s>>>(P, W, N, n, Q, nq, kp, out, grad); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace sbh

// sbh_learned.cuh -- the learned child proposal: parameter layout, features, FP16-weight inference
// and the learned pick (device, inline: used by the estimator kernels), and the host-side training
// steps (sbh_learned.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_internal.cuh"

struct sbh_tree;

namespace sbh {

constexpr int kMlpParams = 1313;  // W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3

constexpr int kIn = 6, kH = 32;
constexpr int oW1 = 0, ob1 = kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH, ob3 = ow3 + kH;
static_assert(ob3 + 1 == kMlpParams, "parameter layout");
constexpr int kMaxLearnedChildren = 64;
constexpr float kMixEps = 0.1f;

// features of child c of node T at q (see the oracle for the same definition in FP64)
__device__ __forceinline__ void child_features(const TreeView& T, const float* diam, uint32_t mT, float4 pT,
                                               int32_t c, float4 pc, uint32_t mc, float3 q, bool dipole, float x[6])
{
    const float BT = diam[meta_level(mT)], Bc = diam[meta_level(mc)];
    const float tx = pT.x - q.x, ty = pT.y - q.y, tz = pT.z - q.z;
    const float vx = pc.x - q.x, vy = pc.y - q.y, vz = pc.z - q.z;
    const float dT = sqrtf(tx * tx + ty * ty + tz * tz) + 1e-6f * BT;
    const float dc = sqrtf(vx * vx + vy * vy + vz * vz) + 1e-6f * Bc;
    x[0] = logf(dc / Bc);
    x[1] = logf(pc.w / pT.w);
    x[2] = logf(Bc / BT);
    x[3] = logf(dc / dT);
    x[4] = 0.0f;
    x[5] = 0.0f;
    if (dipole) {
        const float4 N = __ldg(&T.dip[c]);
        const float nn = sqrtf(N.x * N.x + N.y * N.y + N.z * N.z);
        x[4] = nn / pc.w;
        x[5] = nn > 0.0f ? (vx * N.x + vy * N.y + vz * N.z) / (dc * nn) : 0.0f;
    }
}

// score of one feature row with FP16 weights, FP32 accumulation
__device__ __forceinline__ float score16(const __half* w, const float x[6])
{
    float h1[kH];
#pragma unroll
    for (int i = 0; i < kH; ++i) {
        float z = __half2float(w[ob1 + i]);
#pragma unroll
        for (int k = 0; k < kIn; ++k) z = fmaf(__half2float(w[oW1 + i * kIn + k]), x[k], z);
        h1[i] = fmaxf(z, 0.0f);
    }
    float s = __half2float(w[ob3]);
#pragma unroll 4
    for (int i = 0; i < kH; ++i) {
        float z = __half2float(w[ob2 + i]);
#pragma unroll
        for (int k = 0; k < kH; ++k) z = fmaf(__half2float(w[oW2 + i * kH + k]), h1[k], z);
        s = fmaf(__half2float(w[ow3 + i]), fmaxf(z, 0.0f), s);
    }
    return s;
}

// ------------------------------------------------------------------------------------------------
// the learned pick, used by the one-lane-per-query estimator kernel
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int learned_pick(const TreeView& T, const __half* w, const float* diam, int32_t node, uint32_t mT,
                            float4 pT, float3 q, bool dipole, uint32_t x, float* prob)
{
    const int32_t f = __ldg(&T.fc[node]);
    const int nc = (int)meta_nchild(mT);
    const float u = unit24(x);
    if (nc > kMaxLearnedChildren) {  // mass-proportional pick
        int lo = 0, hi = nc - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(&T.cdf[f + mid]) <= u) lo = mid + 1;
            else hi = mid;
        }
        *prob = __ldg(&T.pm[f + lo]).w / pT.w;
        return lo;
    }
    float s[kMaxLearnedChildren];
    float mx = -3.0e38f;
    for (int c = 0; c < nc; ++c) {
        const float4 pc = __ldg(&T.pm[f + c]);
        float xf[6];
        child_features(T, diam, mT, pT, f + c, pc, __ldg(&T.meta[f + c]), q, dipole, xf);
        s[c] = score16(w, xf);
        mx = fmaxf(mx, s[c]);
    }
    float Z = 0.0f;
    for (int c = 0; c < nc; ++c) {
        s[c] = __expf(s[c] - mx);
        Z += s[c];
    }
    const float iz = (1.0f - kMixEps) / Z, im = kMixEps / pT.w;
    float cum = 0.0f;
    int pick = nc - 1;
    float pp = 0.0f;
    for (int c = 0; c < nc; ++c) {
        const float pc = fmaf(s[c], iz, __ldg(&T.pm[f + c]).w * im);
        cum += pc;
        if (u < cum) { pick = c; pp = pc; break; }
        pp = pc;
    }
    *prob = pp;
    return pick;
}

// device state of one network
struct MlpState {
    float* w = nullptr;     // FP32 master weights
    __half* wh = nullptr;   // FP16 copy used for inference
    float* m = nullptr;     // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;
    int64_t step = 0;
};

cudaError_t mlp_alloc(MlpState& M, cudaStream_t s);
void mlp_release(MlpState& M, cudaStream_t s);
cudaError_t mlp_sync_half(MlpState& M, cudaStream_t s);
cudaError_t mlp_scores(const MlpState& M, const float* feats, int64_t n, float* out, cudaStream_t s);
cudaError_t mlp_loss_grad(MlpState& M, const float* feats, const float* targets, const int64_t* off, int64_t n_sets,
                          cudaStream_t s);
cudaError_t mlp_adam_step(MlpState& M, float lr, cudaStream_t s);
cudaError_t mlp_dataset(const sbh_tree* tree, const float* Q, int nq, const int32_t* set_node, int n_node_sets,
                        const int64_t* set_off, const KernelParams& kp, float* feats, float* targets, cudaStream_t s);

}  // namespace sbh

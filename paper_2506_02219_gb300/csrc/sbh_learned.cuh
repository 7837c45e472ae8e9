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
constexpr float kScoreClamp = 40.0f;  // scores are clamped to [-40, 40]: the softmax needs no max subtraction

// The network is used at node T when T has 2..64 children and the query is nearer than `near`
// cell diagonals to T's centre (FP32: d_T < near * |B_T|); elsewhere the pick is by mass.
__device__ __forceinline__ bool learned_gate(int nc, float dT, float near, float BT)
{
    return nc >= 2 && nc <= kMaxLearnedChildren && dT < __fmul_rn(near, BT);
}

__device__ __forceinline__ float clamp_score(float s) { return fminf(fmaxf(s, -kScoreClamp), kScoreClamp); }

// features of a child (centre and mass pc, cell diagonal Bc, dipole sum N) of node T (pT, BT) at q
// (see the oracle for the same definition in FP64)
__device__ __forceinline__ void features_of(float BT, float Bc, float4 pT, float4 pc, float4 N, float3 q, bool dipole,
                                            float x[6])
{
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
        const float nn = sqrtf(N.x * N.x + N.y * N.y + N.z * N.z);
        x[4] = nn / pc.w;
        x[5] = nn > 0.0f ? (vx * N.x + vy * N.y + vz * N.z) / (dc * nn) : 0.0f;
    }
}

__device__ __forceinline__ void child_features(const TreeView& T, const float* diam, uint32_t mT, float4 pT,
                                               int32_t c, float4 pc, uint32_t mc, float3 q, bool dipole, float x[6])
{
    const float4 N = dipole ? __ldg(&T.dip[c]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    features_of(diam[meta_level(mT)], diam[meta_level(mc)], pT, pc, N, q, dipole, x);
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
                                            float4 pT, float dT, float near, float3 q, bool dipole, uint32_t x,
                                            float* prob)
{
    const int32_t f = __ldg(&T.fc[node]);
    const int nc = (int)meta_nchild(mT);
    const float u = unit24(x);
    if (!learned_gate(nc, dT, near, diam[meta_level(mT)])) {  // mass-proportional pick
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
    float Z = 0.0f;
    for (int c = 0; c < nc; ++c) {
        const float4 pc = __ldg(&T.pm[f + c]);
        float xf[6];
        child_features(T, diam, mT, pT, f + c, pc, __ldg(&T.meta[f + c]), q, dipole, xf);
        s[c] = __expf(clamp_score(score16(w, xf)));
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

// ------------------------------------------------------------------------------------------------
// Warp-cooperative scoring on the tensor cores (mma.sync m16n8k16, FP16 operands, FP32
// accumulation). A chunk is 32 feature rows in shared memory, FP16, 16 columns: the six features,
// a 1 that carries the first layer's bias, zeros. Layer 1 is [32 x 16] x [16 x 32]; its ReLU'd
// FP32 accumulators are packed to FP16 in place as the A operand of layer 2 ([32 x 32] x
// [32 x 32]; the m16n8 accumulator layout of two adjacent n-tiles is the m16k16 operand layout);
// layer 2's accumulators start at b2, and the output s = b3 + sum_n w3_n relu(z2_n) is reduced
// across the four lanes that hold a row. The weight operands are held in shared memory in
// fragment order so every lane loads its registers without bank conflicts.
// ------------------------------------------------------------------------------------------------
struct __align__(16) MlpFrag {
    uint32_t b1[4][2][32];     // layer 1: [n-tile][register][lane]
    uint32_t b2[2][4][2][32];  // layer 2: [k-step][n-tile][register][lane]
    float bias2[kH];
    float w3[kH];
    float b3;
};

constexpr int kChunkWords = 8;  // one FP16 row of 16 columns

// Fill the fragments from the FP16 weights (all threads of the block; sync afterwards).
__device__ __forceinline__ void mlp_frag_fill(const __half* __restrict__ wh, MlpFrag& F)
{
    // B[k][n] of layer 1: W1[n][k] for k < 6, b1[n] for k = 6, 0 above
    auto B1 = [&](int k, int n) -> __half {
        return k < kIn ? wh[oW1 + n * kIn + k] : (k == kIn ? wh[ob1 + n] : __float2half_rn(0.0f));
    };
    for (int i = threadIdx.x; i < 4 * 2 * 32; i += blockDim.x) {
        const int lane = i & 31, reg = (i >> 5) & 1, nt = i >> 6;
        const int g = lane >> 2, t = lane & 3;
        const int k = 2 * t + 8 * reg, n = nt * 8 + g;
        const __half2 h = __halves2half2(B1(k, n), B1(k + 1, n));
        F.b1[nt][reg][lane] = *reinterpret_cast<const uint32_t*>(&h);
    }
    // B[k][n] of layer 2: W2[n][k]
    for (int i = threadIdx.x; i < 2 * 4 * 2 * 32; i += blockDim.x) {
        const int lane = i & 31, reg = (i >> 5) & 1, nt = (i >> 6) & 3, ks = i >> 8;
        const int g = lane >> 2, t = lane & 3;
        const int k = ks * 16 + 2 * t + 8 * reg, n = nt * 8 + g;
        const __half2 h = __halves2half2(wh[oW2 + n * kH + k], wh[oW2 + n * kH + k + 1]);
        F.b2[ks][nt][reg][lane] = *reinterpret_cast<const uint32_t*>(&h);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        F.bias2[i] = __half2float(wh[ob2 + i]);
        F.w3[i] = __half2float(wh[ow3 + i]);
    }
    if (threadIdx.x == 0) F.b3 = __half2float(wh[ob3]);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_relu_half2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(fmaxf(lo, 0.0f), fmaxf(hi, 0.0f));
    return *reinterpret_cast<const uint32_t*>(&h);
}

// One FP16 feature row (6 features, the bias 1, zeros) as 8 words.
__device__ __forceinline__ void store_feature_row(uint32_t* row, const float x[6], bool live)
{
    const __half2 h0 = __floats2half2_rn(x[0], x[1]), h1 = __floats2half2_rn(x[2], x[3]);
    const __half2 h2 = __floats2half2_rn(x[4], x[5]), h3 = __floats2half2_rn(1.0f, 0.0f);
    uint4 v0, v1 = make_uint4(0u, 0u, 0u, 0u);
    v0.x = *reinterpret_cast<const uint32_t*>(&h0);
    v0.y = *reinterpret_cast<const uint32_t*>(&h1);
    v0.z = *reinterpret_cast<const uint32_t*>(&h2);
    v0.w = *reinterpret_cast<const uint32_t*>(&h3);
    if (!live) v0 = make_uint4(0u, 0u, 0u, 0u);
    reinterpret_cast<uint4*>(row)[0] = v0;
    reinterpret_cast<uint4*>(row)[1] = v1;
}

// The weight operands of one lane, held in registers while a warp scores several chunks.
struct MlpRegs {
    uint32_t b1[4][2];
    uint32_t b2[2][4][2];
    float bias2[4][2];
    float w3[4][2];
    float b3;
};

__device__ __forceinline__ void load_mlp_regs(const MlpFrag& F, MlpRegs& R)
{
    const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        R.b1[nt][0] = F.b1[nt][0][lane];
        R.b1[nt][1] = F.b1[nt][1][lane];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            R.b2[ks][nt][0] = F.b2[ks][nt][0][lane];
            R.b2[ks][nt][1] = F.b2[ks][nt][1][lane];
        }
        const int n0 = nt * 8 + 2 * t;
        R.bias2[nt][0] = F.bias2[n0];
        R.bias2[nt][1] = F.bias2[n0 + 1];
        R.w3[nt][0] = F.w3[n0];
        R.w3[nt][1] = F.w3[n0 + 1];
    }
    R.b3 = F.b3;
}

// Scores of the 32 rows of chunk A ([32][kChunkWords] words, written by the warp, __syncwarp'd);
// returns the score of row `lane` to that lane. `sc` is 32 floats of scratch.
__device__ __forceinline__ float score_chunk(const MlpRegs& W, const uint32_t* A, float* sc)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mb = 0; mb < 2; ++mb) {
        const uint32_t* r0 = A + (mb * 16 + g) * kChunkWords;
        const uint32_t* r1 = r0 + 8 * kChunkWords;
        const uint32_t a[4] = {r0[t], r1[t], r0[4 + t], r1[4 + t]};
        float c1[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            c1[nt][0] = c1[nt][1] = c1[nt][2] = c1[nt][3] = 0.0f;
            mma16816(c1[nt], a, W.b1[nt][0], W.b1[nt][1]);
        }
        uint32_t a2[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            a2[ks][0] = pack_relu_half2(c1[2 * ks][0], c1[2 * ks][1]);
            a2[ks][1] = pack_relu_half2(c1[2 * ks][2], c1[2 * ks][3]);
            a2[ks][2] = pack_relu_half2(c1[2 * ks + 1][0], c1[2 * ks + 1][1]);
            a2[ks][3] = pack_relu_half2(c1[2 * ks + 1][2], c1[2 * ks + 1][3]);
        }
        float s_lo = 0.0f, s_hi = 0.0f;  // rows g and g + 8 of the m-block
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            float c2[4] = {W.bias2[nt][0], W.bias2[nt][1], W.bias2[nt][0], W.bias2[nt][1]};
            mma16816(c2, a2[0], W.b2[0][nt][0], W.b2[0][nt][1]);
            mma16816(c2, a2[1], W.b2[1][nt][0], W.b2[1][nt][1]);
            s_lo = fmaf(W.w3[nt][0], fmaxf(c2[0], 0.0f), fmaf(W.w3[nt][1], fmaxf(c2[1], 0.0f), s_lo));
            s_hi = fmaf(W.w3[nt][0], fmaxf(c2[2], 0.0f), fmaf(W.w3[nt][1], fmaxf(c2[3], 0.0f), s_hi));
        }
        s_lo += __shfl_xor_sync(0xFFFFFFFFu, s_lo, 1);
        s_lo += __shfl_xor_sync(0xFFFFFFFFu, s_lo, 2);
        s_hi += __shfl_xor_sync(0xFFFFFFFFu, s_hi, 1);
        s_hi += __shfl_xor_sync(0xFFFFFFFFu, s_hi, 2);
        if (t == 0) {
            sc[mb * 16 + g] = s_lo + W.b3;
            sc[mb * 16 + g + 8] = s_hi + W.b3;
        }
    }
    __syncwarp();
    const float r = sc[lane];
    __syncwarp();
    return r;
}

// The same scores with the weight operands read from the block's shared-memory fragments at each
// use instead of held in registers (every lane reads its own word of a fragment: no bank
// conflicts; the biases and output weights are broadcasts). For kernels whose other state leaves
// no room for the 41 registers of MlpRegs.
__device__ __forceinline__ float score_chunk_shared(const MlpFrag& F, const uint32_t* A, float* sc)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int mb = 0; mb < 2; ++mb) {
        const uint32_t* r0 = A + (mb * 16 + g) * kChunkWords;
        const uint32_t* r1 = r0 + 8 * kChunkWords;
        const uint32_t a[4] = {r0[t], r1[t], r0[4 + t], r1[4 + t]};
        uint32_t a2[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            float c0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            mma16816(c0, a, F.b1[2 * ks][0][lane], F.b1[2 * ks][1][lane]);
            mma16816(c1, a, F.b1[2 * ks + 1][0][lane], F.b1[2 * ks + 1][1][lane]);
            a2[ks][0] = pack_relu_half2(c0[0], c0[1]);
            a2[ks][1] = pack_relu_half2(c0[2], c0[3]);
            a2[ks][2] = pack_relu_half2(c1[0], c1[1]);
            a2[ks][3] = pack_relu_half2(c1[2], c1[3]);
        }
        float s_lo = 0.0f, s_hi = 0.0f;  // rows g and g + 8 of the m-block
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int n0 = nt * 8 + 2 * t;
            const float bb0 = F.bias2[n0], bb1 = F.bias2[n0 + 1];
            float c2[4] = {bb0, bb1, bb0, bb1};
            mma16816(c2, a2[0], F.b2[0][nt][0][lane], F.b2[0][nt][1][lane]);
            mma16816(c2, a2[1], F.b2[1][nt][0][lane], F.b2[1][nt][1][lane]);
            const float w0 = F.w3[n0], w1 = F.w3[n0 + 1];
            s_lo = fmaf(w0, fmaxf(c2[0], 0.0f), fmaf(w1, fmaxf(c2[1], 0.0f), s_lo));
            s_hi = fmaf(w0, fmaxf(c2[2], 0.0f), fmaf(w1, fmaxf(c2[3], 0.0f), s_hi));
        }
        s_lo += __shfl_xor_sync(0xFFFFFFFFu, s_lo, 1);
        s_lo += __shfl_xor_sync(0xFFFFFFFFu, s_lo, 2);
        s_hi += __shfl_xor_sync(0xFFFFFFFFu, s_hi, 1);
        s_hi += __shfl_xor_sync(0xFFFFFFFFu, s_hi, 2);
        if (t == 0) {
            sc[mb * 16 + g] = s_lo + F.b3;
            sc[mb * 16 + g + 8] = s_hi + F.b3;
        }
    }
    __syncwarp();
    const float r = sc[lane];
    __syncwarp();
    return r;
}

// device state of one network
struct MlpState {
    float* w = nullptr;     // FP32 master weights
    __half* wh = nullptr;   // FP16 copy used for inference
    float* m = nullptr;     // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;
    float* part = nullptr;  // per-block partial gradients of the last loss evaluation
    int part_blocks = 0;    // blocks part holds room for (8 per SM of the device it was made on)
    int64_t step = 0;
};

cudaError_t mlp_alloc(MlpState& M, cudaStream_t s);
void mlp_release(MlpState& M, cudaStream_t s);
cudaError_t mlp_sync_half(MlpState& M, cudaStream_t s);
cudaError_t mlp_scores(const MlpState& M, const float* feats, int64_t n, float* out, cudaStream_t s);
cudaError_t mlp_loss_grad(MlpState& M, const float* feats, const float* targets, const int64_t* off, int64_t n_sets,
                          cudaStream_t s);
cudaError_t mlp_adam_step(MlpState& M, float lr, cudaStream_t s);
// training sets visited by Algorithm 2's own paths: base == nullptr counts per query, else writes
cudaError_t mlp_visit(const TreeView& T, const float* Q, int nq, int samples, uint64_t seed, float near,
                      int max_per_query, int32_t* count, const int64_t* base, int32_t* set_q, int32_t* set_node,
                      cudaStream_t s);
cudaError_t mlp_set_rows(const TreeView& T, const int32_t* set_node, int64_t n_sets, int64_t* rows, cudaStream_t s);
cudaError_t mlp_dataset(const sbh_tree* tree, const float* Q, const int32_t* set_q, const int32_t* set_node,
                        int64_t n_sets, const int64_t* set_off, const KernelParams& kp, float* feats, float* targets,
                        cudaStream_t s);

}  // namespace sbh

// sbh_learned.cu -- the learned child proposal: a 6-32-32-1 ReLU network that scores each child
// of a node from query-relative geometry, trained on the residuals met by the estimator's own
// traversals, and used in place of the mass-proportional pick of Algorithm 2.
//
// The paper samples the path index in proportion to mass and names importance sampling as future
// work (Sec. 3.3); this is the project's extension. At a node T with 2..64 children whose centre
// is nearer to the query than `near` cell diagonals, the proposal is
//   pi_c = (1 - eps) softmax(clamp(s))_c + eps m_c / m_T,   eps = 0.1, scores clamped to [-40, 40];
// elsewhere pi_c = m_c / m_T. Every child keeps a probability > 0, so the estimator stays unbiased
// with p(I in T) the product of the pi's along the path. Training: every training query walks
// Algorithm 2's own paths, each decision node within reach becomes a set, and its children's
// targets are |R_c(q)|, the exact residual of the child's subtree (its exact sum minus its
// centre-of-mass term), the per-level proposal that minimises the variance of the child's
// contribution; cross-entropy to the normalised targets, Adam on FP32 master weights, an FP16
// copy for inference. The estimator scores on the tensor cores (sbh_eval_batched.cu).
//
// Parameter layout (1313 values): W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_build.cuh"
#include "sbh_learned.cuh"

namespace sbh {

namespace {

// Scores of feature rows with the estimator's tensor-core scorer: one warp per chunk of 32 rows.
constexpr int kScoreWarps = 8;

__global__ void __launch_bounds__(32 * kScoreWarps) k_scores(const __half* __restrict__ wg,
                                                            const float* __restrict__ feats, int64_t n,
                                                            float* __restrict__ out)
{
    __shared__ MlpFrag F;
    __shared__ __align__(16) uint32_t A[kScoreWarps][32 * kChunkWords];
    __shared__ float sc[kScoreWarps][32];
    mlp_frag_fill(wg, F);
    __syncthreads();
    MlpRegs R;
    load_mlp_regs(F, R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunks = (n + 31) / 32;
    for (int64_t c = (int64_t)blockIdx.x * kScoreWarps + warp; c < chunks; c += (int64_t)gridDim.x * kScoreWarps) {
        const int64_t r = c * 32 + lane;
        const bool live = r < n;
        float x[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (live)
            for (int k = 0; k < 6; ++k) x[k] = feats[6 * r + k];
        store_feature_row(&A[warp][lane * kChunkWords], x, live);
        __syncwarp();
        const float s = score_chunk(R, A[warp], sc[warp]);
        if (live) out[r] = s;
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------------
// training sets from the estimator's own traversals: every training query walks the paths of
// Algorithm 2 (mass-proportional picks, Eq. 5 roulette; its own random stream) and records each
// node it takes a decision at where the network would be used. Pass 0 counts per query, pass 1
// writes (query, node) at the query's offset. At most max_per_query sets per query.
// ------------------------------------------------------------------------------------------------
template <int PASS>
__global__ void __launch_bounds__(256) k_visit(TreeView T, const float* __restrict__ Q, int nq, int samples, uint2 key,
                                               float near, int max_per_query, int32_t* __restrict__ count,
                                               const int64_t* __restrict__ base, int32_t* __restrict__ set_q,
                                               int32_t* __restrict__ set_node)
{
    __shared__ float diam[kDiamLevels];
    if (threadIdx.x < kDiamLevels) diam[threadIdx.x] = T.ctrl->diam[threadIdx.x];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    const float3 q = make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]);
    const int32_t first_sub = T.ctrl->first_sub;
    const int n_sub = T.ctrl->n_sub;
    int n = 0;
    for (int ai = 0; ai < n_sub && n < max_per_query; ++ai) {
        const int32_t a = first_sub + ai;
        const float4 pa = __ldg(&T.pm[a]);
        const uint32_t ma = __ldg(&T.meta[a]);
        if (meta_kind(ma) == kPoint) continue;
        for (int s = 0; s < samples && n < max_per_query; ++s) {
            int32_t node = a;
            uint32_t mT = ma;
            float dT = dist_rn(pa.x, pa.y, pa.z, q);
            uint4 blk = make_uint4(0u, 0u, 0u, 0u);
            for (uint32_t depth = 0; meta_kind(mT) != kPoint && depth < (uint32_t)kMaxDepth; ++depth) {
                const int nc = (int)meta_nchild(mT);
                if (learned_gate(nc, dT, near, diam[meta_level(mT)])) {
                    if (PASS == 1) {
                        set_q[base[j] + n] = j;
                        set_node[base[j] + n] = node;
                    }
                    if (++n >= max_per_query) break;
                }
                // the estimator's stream layout: one block serves depths 2i and 2i + 1
                if ((depth & 1u) == 0u) blk = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)ai, (uint32_t)s, depth), key);
                const uint2 x = (depth & 1u) ? make_uint2(blk.z, blk.w) : make_uint2(blk.x, blk.y);
                const int32_t f = __ldg(&T.fc[node]);
                const float u = unit24(x.x);
                int lo = 0, hi = nc - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(&T.cdf[f + mid]) <= u) lo = mid + 1;
                    else hi = mid;
                }
                const int32_t c = f + lo;
                const float4 pc = __ldg(&T.pm[c]);
                const uint32_t mc = __ldg(&T.meta[c]);
                const float dc = dist_rn(pc.x, pc.y, pc.z, q);
                float p;
                if (!rr_continue(0, unit24(x.y), dT, diam[meta_level(mT)], meta_level(mT), dc, meta_level(mc), p)) break;
                node = c;
                mT = mc;
                dT = dc;
            }
        }
    }
    if (PASS == 0) count[j] = n;
}

__global__ void k_set_rows(TreeView T, const int32_t* __restrict__ set_node, int64_t n_sets, int64_t* __restrict__ rows)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_sets) rows[i] = (int64_t)meta_nchild(__ldg(&T.meta[set_node[i]]));
}

// ------------------------------------------------------------------------------------------------
// training set: for every training query and every subdomain a with 2..64 children, one decision
// set = the children of a, features and |exact residual| targets (FP64 sums over the child's
// points, in Morton order)
// ------------------------------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ double point_value(float4 p, const float4* nrm, int64_t i, float3 q, const KernelParams& kp)
{
    const double dx = (double)p.x - q.x, dy = (double)p.y - q.y, dz = (double)p.z - q.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if constexpr (KIND == SBH_COULOMB) return (double)p.w / sqrt(r2 + (double)kp.eps2);
    else if constexpr (KIND == SBH_WINDING) {
        if (r2 == 0.0) return 0.0;
        const float4 n = nrm[i];
        return (double)p.w * (dx * n.x + dy * n.y + dz * n.z) / (4.0 * 3.141592653589793 * r2 * sqrt(r2));
    } else if constexpr (KIND == SBH_SMOOTHDIST) {
        return (double)p.w * exp(-(double)kp.alpha * sqrt(r2));
    } else {
        return (double)p.w * (1.0 + kp.g[0] * dx + kp.g[1] * dy + kp.g[2] * dz);
    }
}

template <int KIND>
__device__ __forceinline__ double node_value64(const TreeView& T, int32_t v, float4 pm, float3 q, const KernelParams& kp)
{
    const double dx = (double)pm.x - q.x, dy = (double)pm.y - q.y, dz = (double)pm.z - q.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if constexpr (KIND == SBH_COULOMB) return (double)pm.w / sqrt(r2 + (double)kp.eps2);
    else if constexpr (KIND == SBH_WINDING) {
        if (r2 == 0.0) return 0.0;
        const float4 N = __ldg(&T.dip[v]);
        return (dx * N.x + dy * N.y + dz * N.z) / (4.0 * 3.141592653589793 * r2 * sqrt(r2));
    } else if constexpr (KIND == SBH_SMOOTHDIST) {
        return (double)pm.w * exp(-(double)kp.alpha * sqrt(r2));
    } else {
        return (double)pm.w * (1.0 + kp.g[0] * dx + kp.g[1] * dy + kp.g[2] * dz);
    }
}

// one warp per decision set s = (query set_q[s], node set_node[s]); rows set_off[s] ..
template <int KIND>
__global__ void k_dataset(TreeView T, const float4* __restrict__ spw, const float4* __restrict__ snrm,
                          const float* __restrict__ Q, const int32_t* __restrict__ set_q,
                          const int32_t* __restrict__ set_node, int64_t n_sets, const int64_t* __restrict__ set_off,
                          KernelParams kp, float* __restrict__ feats, float* __restrict__ targets)
{
    __shared__ float diam[kDiamLevels];
    if (threadIdx.x < kDiamLevels) diam[threadIdx.x] = T.ctrl->diam[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < n_sets;
         s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t j = set_q[s];
        const int32_t a = set_node[s];
        const float3 q = make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]);
        const uint32_t ma = __ldg(&T.meta[a]);
        const float4 pa = __ldg(&T.pm[a]);
        const int32_t f = __ldg(&T.fc[a]);
        const int nc = (int)meta_nchild(ma);
        const int64_t r0 = set_off[s];
        for (int c = 0; c < nc; ++c) {
            const int32_t ch = f + c;
            const int32_t b = __ldg(&T.nb[ch]), e = __ldg(&T.ne[ch]);
            double sum = 0.0;
            for (int32_t i = b + lane; i < e; i += 32) sum += point_value<KIND>(spw[i], snrm, i, q, kp);
            for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
            if (lane == 0) {
                const float4 pc = __ldg(&T.pm[ch]);
                const double r = sum - node_value64<KIND>(T, ch, pc, q, kp);
                targets[r0 + c] = (float)fabs(r);
                float x[6];
                child_features(T, diam, ma, pa, ch, pc, __ldg(&T.meta[ch]), q, KIND == SBH_WINDING, x);
                for (int k = 0; k < 6; ++k) feats[6 * (r0 + c) + k] = x[k];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// loss and gradient: mean over sets of the cross-entropy between softmax(scores) and the set's
// normalised targets. One warp per set, lane i = hidden unit i of both layers. Each warp keeps its
// partial gradient (per lane: its rows of W1 and W2 and its biases), the block adds its warps'
// partials in warp order and writes one row per block; k_sum_blocks adds the rows in block order.
// No atomics: the gradient, and so the whole training, is the same bit for bit on every run.
// ------------------------------------------------------------------------------------------------
constexpr int kTrainWarps = 4;
constexpr int kPartStride = kMlpParams + 1;  // a block's row: the gradient, then its loss

__global__ void __launch_bounds__(32 * kTrainWarps) k_loss_grad(const float* __restrict__ wg,
                                                               const float* __restrict__ feats,
                                                               const float* __restrict__ targets,
                                                               const int64_t* __restrict__ off, int64_t n_sets,
                                                               float inv_sets, float* __restrict__ part)
{
    __shared__ float w[kMlpParams];
    __shared__ float sc[kTrainWarps][kMaxLearnedChildren];
    __shared__ float wpart[kTrainWarps][kPartStride];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = wg[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float gW1[kIn] = {0, 0, 0, 0, 0, 0}, gW2[kH], gb1 = 0, gb2 = 0, gw3 = 0, gb3 = 0, lsum = 0;
    for (int k = 0; k < kH; ++k) gW2[k] = 0.0f;
    const float b1 = w[ob1 + lane], b2 = w[ob2 + lane], w3 = w[ow3 + lane], b3 = w[ob3];

    for (int64_t s = (int64_t)blockIdx.x * kTrainWarps + warp; s < n_sets; s += (int64_t)gridDim.x * kTrainWarps) {
        const int64_t r0 = off[s];
        const int nc = (int)(off[s + 1] - r0);
        if (nc < 2 || nc > kMaxLearnedChildren) continue;
        // forward: scores
        float tmax = 0.0f;
        for (int c = 0; c < nc; ++c) {
            const float* x = feats + 6 * (r0 + c);
            float z = b1;
            for (int k = 0; k < kIn; ++k) z = fmaf(w[oW1 + lane * kIn + k], x[k], z);
            const float h1 = fmaxf(z, 0.0f);
            float z2 = b2;
            for (int k = 0; k < kH; ++k) z2 = fmaf(w[oW2 + lane * kH + k], __shfl_sync(0xFFFFFFFFu, h1, k), z2);
            float t = w3 * fmaxf(z2, 0.0f);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
            if (lane == 0) sc[warp][c] = t + b3;
            tmax = fmaxf(tmax, targets[r0 + c]);
        }
        __syncwarp();
        // normalised targets t_c / sum_c' t_c', formed as (t_c / t_max) / sum_c' (t_c' / t_max): the
        // smooth distance's residuals exp(-alpha r) can be FP32 denormals, whose sum has no finite
        // reciprocal
        float tsum = 0.0f;
        if (tmax > 0.0f)
            for (int c = 0; c < nc; ++c) tsum += targets[r0 + c] / tmax;
        float mx = -3.0e38f;
        for (int c = 0; c < nc; ++c) mx = fmaxf(mx, sc[warp][c]);
        float Z = 0.0f;
        for (int c = 0; c < nc; ++c) Z += __expf(sc[warp][c] - mx);
        const float logZ = __logf(Z);
        const float tnorm = tsum > 0.0f ? 1.0f / tsum : 0.0f;
        // backward, recomputing each row's activations
        for (int c = 0; c < nc; ++c) {
            const float* x = feats + 6 * (r0 + c);
            const float t = tsum > 0.0f ? (targets[r0 + c] / tmax) * tnorm : 1.0f / nc;
            const float lp = sc[warp][c] - mx - logZ;
            if (lane == 0) lsum -= t * lp;
            const float ds = (__expf(lp) - t) * inv_sets;
            float z = b1;
            for (int k = 0; k < kIn; ++k) z = fmaf(w[oW1 + lane * kIn + k], x[k], z);
            const float h1 = fmaxf(z, 0.0f);
            float z2 = b2;
            for (int k = 0; k < kH; ++k) z2 = fmaf(w[oW2 + lane * kH + k], __shfl_sync(0xFFFFFFFFu, h1, k), z2);
            const float h2 = fmaxf(z2, 0.0f);
            gw3 = fmaf(ds, h2, gw3);
            if (lane == 0) gb3 += ds;
            const float dh2 = z2 > 0.0f ? ds * w3 : 0.0f;
            gb2 += dh2;
            float dh1 = 0.0f;
            for (int k = 0; k < kH; ++k) {
                const float h1k = __shfl_sync(0xFFFFFFFFu, h1, k);
                gW2[k] = fmaf(dh2, h1k, gW2[k]);
                // dh1 of unit `lane`: sum_i W2[i][lane] dh2_i
                dh1 = fmaf(w[oW2 + k * kH + lane], __shfl_sync(0xFFFFFFFFu, dh2, k), dh1);
            }
            dh1 = z > 0.0f ? dh1 : 0.0f;
            gb1 += dh1;
            for (int k = 0; k < kIn; ++k) gW1[k] = fmaf(dh1, x[k], gW1[k]);
        }
        __syncwarp();
    }
    float* wp = wpart[warp];
    for (int k = 0; k < kIn; ++k) wp[oW1 + lane * kIn + k] = gW1[k];
    wp[ob1 + lane] = gb1;
    for (int k = 0; k < kH; ++k) wp[oW2 + lane * kH + k] = gW2[k];
    wp[ob2 + lane] = gb2;
    wp[ow3 + lane] = gw3;
    if (lane == 0) {
        wp[ob3] = gb3;
        wp[kMlpParams] = lsum * inv_sets;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPartStride; i += blockDim.x) {
        float t = 0.0f;
        for (int v = 0; v < kTrainWarps; ++v) t += wpart[v][i];
        part[(int64_t)blockIdx.x * kPartStride + i] = t;
    }
}

// grad[i] = sum over blocks b (in order) of part[b][i]; loss likewise from the last column
__global__ void k_sum_blocks(const float* __restrict__ part, int blocks, float* __restrict__ grad,
                             float* __restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPartStride) return;
    float t = 0.0f;
    for (int b = 0; b < blocks; ++b) t += part[(int64_t)b * kPartStride + i];
    if (i < kMlpParams) grad[i] = t;
    else *loss = t;
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __half* __restrict__ wh, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    w[i] = wi;
    wh[i] = __float2half_rn(wi);
}

__global__ void k_to_half(const float* __restrict__ w, __half* __restrict__ wh)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpParams) wh[i] = __float2half_rn(w[i]);
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
cudaError_t mlp_alloc(MlpState& M, cudaStream_t s)
{
    cudaError_t e = dalloc((void**)&M.w, kMlpParams * sizeof(float), s);
    if (e == cudaSuccess) e = dalloc((void**)&M.wh, kMlpParams * sizeof(__half), s);
    if (e == cudaSuccess) e = dalloc((void**)&M.m, kMlpParams * sizeof(float), s);
    if (e == cudaSuccess) e = dalloc((void**)&M.v, kMlpParams * sizeof(float), s);
    if (e == cudaSuccess) e = dalloc((void**)&M.grad, kMlpParams * sizeof(float), s);
    if (e == cudaSuccess) e = dalloc((void**)&M.loss, sizeof(float), s);
    M.part_blocks = 8 * device_sm_count();
    if (e == cudaSuccess) e = dalloc((void**)&M.part, (size_t)M.part_blocks * kPartStride * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.m, 0, kMlpParams * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.v, 0, kMlpParams * sizeof(float), s);
    return e;
}

void mlp_release(MlpState& M, cudaStream_t s)
{
    dfree(M.w, s); dfree(M.wh, s); dfree(M.m, s); dfree(M.v, s); dfree(M.grad, s); dfree(M.loss, s);
    dfree(M.part, s);
    M = MlpState();
}

cudaError_t mlp_sync_half(MlpState& M, cudaStream_t s)
{
    k_to_half<<<(kMlpParams + 255) / 256, 256, 0, s>>>(M.w, M.wh);
    note_launch();
    return cudaGetLastError();
}

cudaError_t mlp_scores(const MlpState& M, const float* feats, int64_t n, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = ((n + 31) / 32 + kScoreWarps - 1) / kScoreWarps;
    const int64_t cap = 8 * (int64_t)device_sm_count();
    if (blocks > cap) blocks = cap;
    k_scores<<<(unsigned)blocks, 32 * kScoreWarps, 0, s>>>(M.wh, feats, n, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t mlp_loss_grad(MlpState& M, const float* feats, const float* targets, const int64_t* off, int64_t n_sets,
                          cudaStream_t s)
{
    if (n_sets <= 0) {
        cudaError_t e = cudaMemsetAsync(M.grad, 0, kMlpParams * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(M.loss, 0, sizeof(float), s);
        return e;
    }
    int64_t blocks = (n_sets + kTrainWarps - 1) / kTrainWarps;
    if (blocks > M.part_blocks) blocks = M.part_blocks;  // the partial sums are then added in a fixed order
    k_loss_grad<<<(unsigned)blocks, 32 * kTrainWarps, 0, s>>>(M.w, feats, targets, off, n_sets, 1.0f / (float)n_sets,
                                                             M.part);
    note_launch();
    k_sum_blocks<<<(kPartStride + 255) / 256, 256, 0, s>>>(M.part, (int)blocks, M.grad, M.loss);
    note_launch();
    return cudaGetLastError();
}

cudaError_t mlp_adam_step(MlpState& M, float lr, cudaStream_t s)
{
    M.step += 1;
    const float c1 = 1.0f / (1.0f - powf(0.9f, (float)M.step));
    const float c2 = 1.0f / (1.0f - powf(0.999f, (float)M.step));
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(M.w, M.grad, M.m, M.v, M.wh, lr, c1, c2);
    note_launch();
    return cudaGetLastError();
}

cudaError_t mlp_visit(const TreeView& T, const float* Q, int nq, int samples, uint64_t seed, float near,
                      int max_per_query, int32_t* count, const int64_t* base, int32_t* set_q, int32_t* set_node,
                      cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned b = (unsigned)((nq + 255) / 256);
    if (base == nullptr) k_visit<0><<<b, 256, 0, s>>>(T, Q, nq, samples, key, near, max_per_query, count, nullptr, nullptr, nullptr);
    else k_visit<1><<<b, 256, 0, s>>>(T, Q, nq, samples, key, near, max_per_query, nullptr, base, set_q, set_node);
    note_launch();
    return cudaGetLastError();
}

cudaError_t mlp_set_rows(const TreeView& T, const int32_t* set_node, int64_t n_sets, int64_t* rows, cudaStream_t s)
{
    if (n_sets <= 0) return cudaSuccess;
    k_set_rows<<<(unsigned)((n_sets + 255) / 256), 256, 0, s>>>(T, set_node, n_sets, rows);
    note_launch();
    return cudaGetLastError();
}

cudaError_t mlp_dataset(const sbh_tree* tree, const float* Q, const int32_t* set_q, const int32_t* set_node,
                        int64_t n_sets, const int64_t* set_off, const KernelParams& kp, float* feats, float* targets,
                        cudaStream_t s)
{
    if (n_sets <= 0) return cudaSuccess;
    const TreeView T = tree->t4.view();
    int64_t blocks = (n_sets * 32 + 255) / 256;
    const int64_t cap = 16 * (int64_t)device_sm_count();
    if (blocks > cap) blocks = cap;
    const unsigned b = (unsigned)blocks;
    switch (kp.kind) {
    case SBH_COULOMB: k_dataset<SBH_COULOMB><<<b, 256, 0, s>>>(T, tree->spw, tree->snrm, Q, set_q, set_node, n_sets, set_off, kp, feats, targets); break;
    case SBH_WINDING: k_dataset<SBH_WINDING><<<b, 256, 0, s>>>(T, tree->spw, tree->snrm, Q, set_q, set_node, n_sets, set_off, kp, feats, targets); break;
    case SBH_SMOOTHDIST: k_dataset<SBH_SMOOTHDIST><<<b, 256, 0, s>>>(T, tree->spw, tree->snrm, Q, set_q, set_node, n_sets, set_off, kp, feats, targets); break;
    case SBH_AFFINE: k_dataset<SBH_AFFINE><<<b, 256, 0, s>>>(T, tree->spw, tree->snrm, Q, set_q, set_node, n_sets, set_off, kp, feats, targets); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace sbh

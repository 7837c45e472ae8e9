// sbh_eval.cu -- the stratified path sample estimator (Madan et al. 2025, Sec. 3.3, Eq. 5-7,
// Algorithm 2) walked one lane per query: the counting variant (sbh_eval_count), the adjoint
// (sbh_eval_grad) and sbh_eval's one-lane-per-query schedule (opts->schedule = 1). The default
// schedule of sbh_eval is the batched one of sbh_eval_batched.cu, which evaluates the same terms
// along the same paths.
//
// For each query q and each subdomain a (a child of the root, Sec. 3.3.1):
//   F += CV_a = m_a f(p_a, q)
//   for each of S paths: starting at T = a, while T is not a source point:
//       draw the child c of T holding the path index (probability m_c / m_T), draw the Russian
//       roulette continue with p = Eq. 5 for (T, c); stop if it fails; otherwise add the
//       contribution swap (Eq. 6) Delta_T = sum_children m f - m_T f(p_T, q), weighted by
//       1 / (p(I in T) p(K >= k)), and step into c.
//   F += (sum of the path terms) / S
// The random stream is Philox4x32-10 keyed by the seed; the decision at depth k uses the block
// counted by (query index, subdomain, sample, k - k mod 2), words 0 and 1 at even k and 2 and 3
// at odd k: the first picks the child, the second plays the roulette. Decisions are taken in FP32
// with correctly rounded operations in a fixed order; kernel values use fast FP32 arithmetic.
//
// The adjoint applies the same estimator to grad_q f: paths and weights are those drawn for the
// value (held fixed), every term m f is replaced by its gradient. The weights are those of a valid
// sampling of the tree's telescoping sums, so the expectation is exactly grad F.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_eval.cuh"
#include "sbh_learned.cuh"

namespace sbh {

namespace {

constexpr int kModeCount = 0;
constexpr int kModeGrad = 1;
constexpr int kModeEval = 2;
constexpr int kModeLearned = 3;  // evaluation with the learned child proposal

// most blocks launched per SM (the rest of the queries are taken in grid-stride order)
#ifndef SBH_LANE_GRID_BLOCKS_PER_SM
#define SBH_LANE_GRID_BLOCKS_PER_SM 256
#endif

// Running sum of weighted terms and of their query gradients. The smooth-distance kernel keeps
// both in units of exp(-alpha ref), ref the smallest distance seen so far.
template <int KIND, bool GRAD>
struct Acc {
    float v = 0.0f;
    float g[3] = {0.0f, 0.0f, 0.0f};
    float ref = 3.0e38f;

    // w * m f(p, q) (+ its gradient) for node `node` with record pm
    __device__ __forceinline__ void add(const TreeView& T, int32_t node, float4 pm, float3 q, const KernelParams& kp,
                                        float w)
    {
        const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
        if constexpr (KIND == SBH_COULOMB) {
            const float e = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kp.eps2)));
            const float ir = rsqrt_ftz(e);
            const float t = w * pm.w * ir;
            v += t;
            if (GRAD) {
                const float c = t * ir * ir;  // w m / e^(3/2)
                g[0] = fmaf(c, dx, g[0]); g[1] = fmaf(c, dy, g[1]); g[2] = fmaf(c, dz, g[2]);
            }
        } else if constexpr (KIND == SBH_WINDING) {
            const float4 N = __ldg(&T.dip[node]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 >= kMinNormal) {
                const float ir = rsqrt_ftz(r2);
                const float ir3 = ir * ir * ir;
                const float dn = fmaf(dx, N.x, fmaf(dy, N.y, dz * N.z));
                const float s = w * kInv4Pi;
                v = fmaf(s * dn, ir3, v);
                if (GRAD) {
                    const float c = 3.0f * s * dn * ir3 * ir * ir;  // 3 (d.N) / r^5
                    const float b = -s * ir3;                       // -1 / r^3
                    g[0] += fmaf(b, N.x, c * dx); g[1] += fmaf(b, N.y, c * dy); g[2] += fmaf(b, N.z, c * dz);
                }
            }
        } else if constexpr (KIND == SBH_SMOOTHDIST) {
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ir = rsqrt_ftz(fmaxf(r2, 1e-37f));
            const float r = r2 * ir;
            if (r < ref) {
                const float f = __expf(-kp.alpha * (ref - r));
                v *= f;
                if (GRAD) { g[0] *= f; g[1] *= f; g[2] *= f; }
                ref = r;
            }
            const float t = w * pm.w * __expf(-kp.alpha * (r - ref));
            v += t;
            if (GRAD && r2 > 0.0f) {
                const float c = kp.alpha * t * ir;  // alpha w m exp(-alpha r) / r
                g[0] = fmaf(c, dx, g[0]); g[1] = fmaf(c, dy, g[1]); g[2] = fmaf(c, dz, g[2]);
            }
        } else {
            const float t = w * pm.w;
            v = fmaf(t, 1.0f + fmaf(kp.g[0], dx, fmaf(kp.g[1], dy, kp.g[2] * dz)), v);
            if (GRAD) { g[0] -= t * kp.g[0]; g[1] -= t * kp.g[1]; g[2] -= t * kp.g[2]; }
        }
    }
};

// work counters of one thread: kernel terms evaluated, node records read by swaps and control
// variates, decisions (one Philox block per two depths), prefix fractions read
struct Counters {
    unsigned long long evals = 0, records = 0, decisions = 0, cdf_reads = 0;
};

template <int KIND, int MODE>
__global__ void __launch_bounds__(256) k_stoch_eval(TreeView T, const float* __restrict__ Q, int64_t nq,
                                                    KernelParams kp, int S, uint2 key, int sampling, int rr,
                                                    int coherent, int raw_sum, float* __restrict__ out,
                                                    float* __restrict__ grad, unsigned long long* __restrict__ counts,
                                                    const __half* __restrict__ mlpw, float near, int64_t qbase)
{
    constexpr bool COUNT = MODE == kModeCount;
    constexpr bool GRAD = MODE == kModeGrad;
    constexpr bool LEARNED = MODE == kModeLearned;
    Counters cnt;
    __shared__ float sdiam[kDiamLevels];
    __shared__ __half sw[LEARNED ? kMlpParams : 1];
    if (threadIdx.x < kDiamLevels) sdiam[threadIdx.x] = T.ctrl->diam[threadIdx.x];
    if (LEARNED)
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = mlpw[i];
    __syncthreads();
    const int32_t first_sub = T.ctrl->first_sub;
    const int n_sub = T.ctrl->n_sub;
    const float invS = 1.0f / (float)S;

    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nq; j += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]);
        Acc<KIND, GRAD> acc;
        for (int ai = 0; ai < n_sub; ++ai) {
            const int32_t a = first_sub + ai;
            const float4 pa = __ldg(&T.pm[a]);
            const uint32_t ma = __ldg(&T.meta[a]);
            if (COUNT) { cnt.evals += 1; cnt.records += 1; }
            else acc.add(T, a, pa, q, kp, 1.0f);  // control variate CV_a
            if (meta_kind(ma) == kPoint) continue;
            // a's weight for p(I in T): aggregate mass or point count
            const float wa = sampling ? (float)(__ldg(&T.ne[a]) - __ldg(&T.nb[a])) : pa.w;
            const float da = dist_rn(pa.x, pa.y, pa.z, q);
            for (int s = 0; s < S; ++s) {
                int32_t node = a;
                float4 pT = pa;
                uint32_t mT = ma;
                float dT = da;
                float prr = 1.0f;
                float wT = wa;
                float ppath = 1.0f;  // learned proposal: probability of the picks so far
                uint4 blk = make_uint4(0u, 0u, 0u, 0u);
                for (uint32_t depth = 0; meta_kind(mT) != kPoint && depth < (uint32_t)kMaxDepth; ++depth) {
                    // one Philox block serves depths 2i (words 0, 1) and 2i + 1 (words 2, 3)
                    if ((depth & 1u) == 0u)
                        blk = philox4x32_10(
                            make_uint4(coherent ? 0u : (uint32_t)(j + qbase), (uint32_t)ai, (uint32_t)s, depth), key);
                    const uint2 x = (depth & 1u) ? make_uint2(blk.z, blk.w) : make_uint2(blk.x, blk.y);
                    const int32_t f = __ldg(&T.fc[node]);
                    const int nc = (int)meta_nchild(mT);
                    int pick = 0;
                    float pick_prob = 1.0f;
                    if (LEARNED) {
                        pick = learned_pick(T, sw, sdiam, node, mT, pT, dT, near, q, KIND == SBH_WINDING, x.x,
                                            &pick_prob);
                    } else if (sampling == 0) {
                        const float u = unit24(x.x);
                        for (int k = 0; k < nc - 1; ++k) pick += (__ldg(&T.cdf[f + k]) <= u) ? 1 : 0;
                    } else {
                        const int32_t b = __ldg(&T.nb[node]);
                        const int32_t cnt_pts = __ldg(&T.ne[node]) - b;
                        const int32_t target = b + (int32_t)(((uint64_t)(x.x >> 8) * (uint64_t)cnt_pts) >> 24);
                        for (int k = 1; k < nc; ++k) pick += (__ldg(&T.nb[f + k]) <= target) ? 1 : 0;
                    }
                    if (COUNT) { cnt.decisions += 1; cnt.cdf_reads += (uint64_t)(nc - 1); }
                    const int32_t c = f + pick;
                    const float4 pc = __ldg(&T.pm[c]);
                    const uint32_t mc = __ldg(&T.meta[c]);
                    const float dc = dist_rn(pc.x, pc.y, pc.z, q);
                    float p = 1.0f;
                    if (!rr_continue(rr, unit24(x.y), dT, sdiam[meta_level(mT)], meta_level(mT), dc, meta_level(mc), p))
                        break;
                    prr *= p;
                    const float pagg = LEARNED ? ppath : wT / wa;
                    const float w = 1.0f / (pagg * prr) * invS;
                    ppath *= pick_prob;
                    if (COUNT) {
                        cnt.evals += (uint64_t)nc + 1;
                        cnt.records += (uint64_t)nc;
                    } else {
                        for (int k = 0; k < nc; ++k) acc.add(T, f + k, __ldg(&T.pm[f + k]), q, kp, w);
                        acc.add(T, node, pT, q, kp, -w);
                    }
                    node = c;
                    pT = pc;
                    mT = mc;
                    dT = dc;
                    wT = sampling ? (float)(__ldg(&T.ne[c]) - __ldg(&T.nb[c])) : pc.w;
                }
            }
        }
        if (COUNT) continue;
        if constexpr (KIND == SBH_SMOOTHDIST) {
            // d = ref - log(acc) / alpha; grad d = -grad F / (alpha F): the exp(-alpha ref) units cancel
            if (raw_sum) {
                const float sc = __expf(-kp.alpha * acc.ref);
                out[j] = acc.v * sc;
                if (GRAD) { grad[3 * j] = acc.g[0] * sc; grad[3 * j + 1] = acc.g[1] * sc; grad[3 * j + 2] = acc.g[2] * sc; }
            } else {
                const bool pos = acc.v > 0.0f;
                out[j] = pos ? acc.ref - __logf(acc.v) / kp.alpha : __int_as_float(0x7F800000);
                if (GRAD) {
                    const float c = pos ? -1.0f / (kp.alpha * acc.v) : __int_as_float(0x7FC00000);
                    grad[3 * j] = c * acc.g[0]; grad[3 * j + 1] = c * acc.g[1]; grad[3 * j + 2] = c * acc.g[2];
                }
            }
        } else {
            out[j] = acc.v;
            if (GRAD) { grad[3 * j] = acc.g[0]; grad[3 * j + 1] = acc.g[1]; grad[3 * j + 2] = acc.g[2]; }
        }
    }
    if (COUNT) {
        unsigned long long v[4] = {cnt.evals, cnt.records, cnt.decisions, cnt.cdf_reads};
        for (int k = 0; k < 4; ++k) {
            unsigned long long x = v[k];
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, off);
            if ((threadIdx.x & 31) == 0) atomicAdd(&counts[k], x);
        }
    }
}

template <int MODE>
cudaError_t launch_lane_impl(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                             uint64_t seed, const sbh_eval_opts& o, float* out, float* grad,
                             unsigned long long* counts, cudaStream_t s, const __half* mlpw = nullptr,
                             float near = 0.0f, int64_t qbase = 0)
{
    if (nq <= 0) return cudaSuccess;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int threads = 256;
    int64_t blocks = (nq + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * SBH_LANE_GRID_BLOCKS_PER_SM;
    if (blocks > cap) blocks = cap;
    const unsigned b = (unsigned)blocks;
    switch (kp.kind) {
    case SBH_COULOMB:
        k_stoch_eval<SBH_COULOMB, MODE><<<b, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, grad, counts, mlpw, near, qbase);
        break;
    case SBH_WINDING:
        k_stoch_eval<SBH_WINDING, MODE><<<b, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, grad, counts, mlpw, near, qbase);
        break;
    case SBH_SMOOTHDIST:
        k_stoch_eval<SBH_SMOOTHDIST, MODE><<<b, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, grad, counts, mlpw, near, qbase);
        break;
    case SBH_AFFINE:
        k_stoch_eval<SBH_AFFINE, MODE><<<b, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, grad, counts, mlpw, near, qbase);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stoch_eval(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                              const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                              cudaStream_t s, int64_t qbase)
{
    if (o.schedule == 1)
        return launch_lane_impl<kModeEval>(T, Q, nq, kp, S, seed, o, out, nullptr, nullptr, s, nullptr, 0.0f, qbase);
    return launch_stoch_batched(T, host_ctrl, Q, nq, kp, S, seed, o, out, s, qbase);
}

cudaError_t launch_stoch_lane(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                              uint64_t seed, const sbh_eval_opts& o, float* out, cudaStream_t s)
{
    return launch_lane_impl<kModeEval>(T, Q, nq, kp, S, seed, o, out, nullptr, nullptr, s);
}

cudaError_t launch_stoch_learned(const TreeView& T, const TreeCtrl& host_ctrl, const void* mlp_half, float near,
                                 const float* Q, int64_t nq, const KernelParams& kp, int S, uint64_t seed,
                                 const sbh_eval_opts& o, float* out, cudaStream_t s)
{
    if (o.schedule == 1)
        return launch_lane_impl<kModeLearned>(T, Q, nq, kp, S, seed, o, out, nullptr, nullptr, s,
                                              (const __half*)mlp_half, near);
    return launch_stoch_batched_learned(T, host_ctrl, mlp_half, near, Q, nq, kp, S, seed, o, out, s);
}

cudaError_t launch_stoch_count(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                               uint64_t seed, const sbh_eval_opts& o, unsigned long long* counts, cudaStream_t s)
{
    return launch_lane_impl<kModeCount>(T, Q, nq, kp, S, seed, o, nullptr, nullptr, counts, s);
}

cudaError_t launch_stoch_grad(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                              const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                              float* grad, cudaStream_t s)
{
    if (o.schedule == 1) return launch_lane_impl<kModeGrad>(T, Q, nq, kp, S, seed, o, out, grad, nullptr, s);
    return launch_stoch_batched_grad(T, host_ctrl, Q, nq, kp, S, seed, o, out, grad, s);
}

}  // namespace sbh

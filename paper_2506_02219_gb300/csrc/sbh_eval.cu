// sbh_eval.cu -- the stratified path sample estimator (Madan et al. 2025, Sec. 3.3, Eq. 5-7,
// Algorithm 2) on the 64-ary tree.
//
// For each query q and each subdomain a (a child of the root, Sec. 3.3.1):
//   F += CV_a = m_a f(p_a, q)
//   for each of S paths: starting at T = a, while T is not a source point:
//       draw the child c of T holding the path index (probability m_c / m_T), draw the Russian
//       roulette continue with p = Eq. 5 for (T, c); stop if it fails; otherwise add the
//       contribution swap (Eq. 6) Delta_T = sum_children m f - m_T f(p_T, q), weighted by
//       1 / (p(I in T) p(K >= k)), and step into c.
//   F += (sum of the path terms) / S
// The random stream is Philox4x32-10 keyed by the seed and counted by (query index, subdomain,
// sample, depth): word 0 picks the child, word 1 plays the roulette.
//
// Decisions (child pick, roulette) are taken in FP32 with correctly rounded operations in a fixed
// order; kernel values use fast FP32 arithmetic.
//
// This file's kernel walks each query's paths one lane per query; it is the counting variant
// behind sbh_eval_count (same paths, same decisions). sbh_eval itself runs the batched schedule of
// sbh_eval_batched.cu, which evaluates the same terms.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_eval.cuh"

namespace sbh {

template <int KIND>
struct Terms {
    // m f(p, q) for node record pm (and its dipole for the winding kernel)
    static __device__ __forceinline__ float value(const TreeView& T, int32_t v, float4 pm, float3 q,
                                                  const KernelParams& kp)
    {
        if constexpr (KIND == SBH_COULOMB) {
            return term_coulomb(pm, q, kp.eps2);
        } else if constexpr (KIND == SBH_WINDING) {
            return term_winding(pm, __ldg(&T.dip[v]), q);
        } else if constexpr (KIND == SBH_AFFINE) {
            return term_affine(pm, q, kp.g);
        } else {
            return 0.0f;  // smooth distance goes through the exp accumulator
        }
    }
};

// sum_c m_c f(p_c, q) over the children [f, f + nc) of a node, minus m_T f(p_T, q), times w,
// added to the running accumulator
// work counters of one thread (compiled out unless COUNT): kernel terms evaluated, node records
// read by swaps and control variates, decisions (one Philox block each), prefix fractions read
struct Counters {
    unsigned long long evals = 0, records = 0, decisions = 0, cdf_reads = 0;
};

template <int KIND>
__device__ __forceinline__ void add_swap(const TreeView& T, int32_t node, int32_t f, int nc, float4 pT, float dT_fast,
                                         float3 q, const KernelParams& kp, float w, float& acc, ExpAcc& ex)
{
    if constexpr (KIND == SBH_SMOOTHDIST) {
        for (int k = 0; k < nc; ++k) {
            const float4 pc = __ldg(&T.pm[f + k]);
            const float d = dist_fast(pc, q);
            ex.lower(d, kp.alpha);
            ex.acc = fmaf(w * pc.w, ex.scale(d, kp.alpha), ex.acc);
        }
        ex.lower(dT_fast, kp.alpha);
        ex.acc = fmaf(-w * pT.w, ex.scale(dT_fast, kp.alpha), ex.acc);
    } else {
        float s = 0.0f;
        for (int k = 0; k < nc; ++k) {
            const float4 pc = __ldg(&T.pm[f + k]);
            s += Terms<KIND>::value(T, f + k, pc, q, kp);
        }
        acc = fmaf(w, s - Terms<KIND>::value(T, node, pT, q, kp), acc);
    }
}

template <int KIND, bool COUNT>
__global__ void __launch_bounds__(256) k_stoch_eval(TreeView T, const float* __restrict__ Q, int64_t nq,
                                                    KernelParams kp, int S, uint2 key, int sampling, int rr,
                                                    int coherent, int raw_sum, float* __restrict__ out,
                                                    unsigned long long* __restrict__ counts)
{
    Counters cnt;
    __shared__ float sdiam[kDiamLevels];
    if (threadIdx.x < kDiamLevels) sdiam[threadIdx.x] = T.ctrl->diam[threadIdx.x];
    __syncthreads();
    const int32_t first_sub = T.ctrl->first_sub;
    const int n_sub = T.ctrl->n_sub;
    const float invS = 1.0f / (float)S;

    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nq; j += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(Q[3 * j], Q[3 * j + 1], Q[3 * j + 2]);
        float acc = 0.0f;
        ExpAcc ex;
        ex.init(3.0e38f);
        for (int ai = 0; ai < n_sub; ++ai) {
            const int32_t a = first_sub + ai;
            const float4 pa = __ldg(&T.pm[a]);
            const uint32_t ma = __ldg(&T.meta[a]);
            // control variate CV_a
            float ta_fast = 0.0f;
            if constexpr (KIND == SBH_SMOOTHDIST) {
                ta_fast = dist_fast(pa, q);
                ex.lower(ta_fast, kp.alpha);
                ex.acc = fmaf(pa.w, ex.scale(ta_fast, kp.alpha), ex.acc);
            } else {
                acc += Terms<KIND>::value(T, a, pa, q, kp);
            }
            if (COUNT) { cnt.evals += 1; cnt.records += 1; }
            if (meta_kind(ma) == kPoint) continue;
            // a's weight for p(I in T): aggregate mass or point count
            const float wa = sampling ? (float)(__ldg(&T.ne[a]) - __ldg(&T.nb[a])) : pa.w;
            const float da = dist_rn(pa.x, pa.y, pa.z, q);
            for (int s = 0; s < S; ++s) {
                int32_t node = a;
                float4 pT = pa;
                uint32_t mT = ma;
                float dT = da, dT_fast = ta_fast;
                float prr = 1.0f;
                float wT = wa;
                for (uint32_t depth = 0; meta_kind(mT) != kPoint && depth < (uint32_t)kMaxDepth; ++depth) {
                    const uint4 x = philox4x32_10(
                        make_uint4(coherent ? 0u : (uint32_t)j, (uint32_t)ai, (uint32_t)s, depth), key);
                    const int32_t f = __ldg(&T.fc[node]);
                    const int nc = (int)meta_nchild(mT);
                    int pick = 0;
                    if (sampling == 0) {
                        const float u = unit24(x.x);
                        for (int k = 0; k < nc - 1; ++k) pick += (__ldg(&T.cdf[f + k]) <= u) ? 1 : 0;
                    } else {
                        const int32_t b = __ldg(&T.nb[node]);
                        const int32_t cnt = __ldg(&T.ne[node]) - b;
                        const int32_t target = b + (int32_t)(((uint64_t)(x.x >> 8) * (uint64_t)cnt) >> 24);
                        for (int k = 1; k < nc; ++k) pick += (__ldg(&T.nb[f + k]) <= target) ? 1 : 0;
                    }
                    if (COUNT) { cnt.decisions += 1; cnt.cdf_reads += (uint64_t)(nc - 1); }
                    const int32_t c = f + pick;
                    const float4 pc = __ldg(&T.pm[c]);
                    const uint32_t mc = __ldg(&T.meta[c]);
                    const float dc = dist_rn(pc.x, pc.y, pc.z, q);
                    float p;
                    if (rr == 0) p = rr_prob_rn(dT, sdiam[meta_level(mT)], dc, sdiam[meta_level(mc)]);
                    else p = (rr == 1) ? 1.0f : 0.5f;
                    if (unit24(x.y) >= p) break;
                    prr *= p;
                    const float pagg = wT / wa;
                    const float w = 1.0f / (pagg * prr) * invS;
                    add_swap<KIND>(T, node, f, nc, pT, dT_fast, q, kp, w, acc, ex);
                    if (COUNT) { cnt.evals += (uint64_t)nc + 1; cnt.records += (uint64_t)nc; }
                    node = c;
                    pT = pc;
                    mT = mc;
                    dT = dc;
                    if constexpr (KIND == SBH_SMOOTHDIST) dT_fast = dist_fast(pc, q);
                    wT = sampling ? (float)(__ldg(&T.ne[c]) - __ldg(&T.nb[c])) : pc.w;
                }
            }
        }
        if (COUNT) continue;
        if constexpr (KIND == SBH_SMOOTHDIST) {
            if (raw_sum) out[j] = ex.acc * __expf(-kp.alpha * ex.ref);
            else out[j] = ex.acc > 0.0f ? ex.ref - __logf(ex.acc) / kp.alpha : __int_as_float(0x7F800000);
        } else {
            out[j] = acc;
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

template <bool COUNT>
static cudaError_t launch_stoch_impl(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                                     uint64_t seed, const sbh_eval_opts& o, float* out,
                                     unsigned long long* counts, cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int threads = 256;
    int64_t blocks = (nq + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    switch (kp.kind) {
    case SBH_COULOMB:
        k_stoch_eval<SBH_COULOMB, COUNT><<<(unsigned)blocks, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, counts);
        break;
    case SBH_WINDING:
        k_stoch_eval<SBH_WINDING, COUNT><<<(unsigned)blocks, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, counts);
        break;
    case SBH_SMOOTHDIST:
        k_stoch_eval<SBH_SMOOTHDIST, COUNT><<<(unsigned)blocks, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, counts);
        break;
    case SBH_AFFINE:
        k_stoch_eval<SBH_AFFINE, COUNT><<<(unsigned)blocks, threads, 0, s>>>(T, Q, nq, kp, S, key, o.sampling, o.rr, o.seed_mode, o.raw_sum, out, counts);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stoch_eval(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                              const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                              cudaStream_t s)
{
    return launch_stoch_batched(T, host_ctrl, Q, nq, kp, S, seed, o, out, s);
}

cudaError_t launch_stoch_count(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                               uint64_t seed, const sbh_eval_opts& o, unsigned long long* counts, cudaStream_t s)
{
    return launch_stoch_impl<true>(T, Q, nq, kp, S, seed, o, nullptr, counts, s);
}

}  // namespace sbh

// sbh_eval_batched.cu -- the stratified path estimator (Madan et al. 2025, Sec. 3.3, Eq. 5-7,
// Algorithm 2) organised for full SIMT lanes.
//
// The arithmetic and the random stream are those of Algorithm 2 (see sbh_eval.cu for the
// statement); what differs is how a warp schedules the work of its 32 queries. Per subdomain a
// every lane takes the depth-0 decision of its own query (same node, so the child records and
// prefix fractions it reads are the same addresses for all lanes). Everything after that is a task:
//   decision task  (query, node T, depth k, ...): draw the child, play the roulette (Eq. 5);
//   swap task      (query, node T, weight w):     add w * Delta_T (Eq. 6) to the query's sum.
// A continuing decision emits one swap task and one decision task for the chosen child. Tasks
// wait in two per-warp rings in shared memory and are run 32 at a time, one per lane, so the
// lanes stay busy however the paths of the 32 queries diverge. Swap results reach a query's sum
// through a lane-ordered reduction among the tasks of that query, so results are deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_eval.cuh"

namespace sbh {

namespace {

constexpr int kWarpsPerBlock = 8;
constexpr int kRing = 64;  // ring capacity per warp; at most 63 tasks wait at any time
constexpr uint32_t kRingMask = kRing - 1;

// per-warp shared state, structure of arrays
struct WarpState {
    // decision tasks
    int32_t d_node[kRing];
    uint32_t d_tag[kRing];   // slot | depth << 5 | sample << 13
    int32_t d_ai[kRing];
    float d_prr[kRing];
    float d_dT[kRing];       // correctly rounded distance from the query to the node's centre
    float d_wT[kRing];       // the node's mass (or point count)
    float d_wa[kRing];       // the subdomain's mass (or point count)
    // swap tasks
    int32_t s_node[kRing];
    uint32_t s_slot[kRing];
    float s_w[kRing];
    // the warp's 32 queries
    float qx[32], qy[32], qz[32];
    uint32_t qctr[32];       // counter word 0 of each query's random stream
    float acc[32];           // sum of the swap terms (smooth distance: in units of exp(-alpha ref))
    float ref[32];
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

// The subdomains and their children (node generations 1 and 2) are read by every query: each
// block copies them (up to kStageMax nodes) into shared memory at start and reads them there.
constexpr int kStageMax = 2048;

struct Stage {
    int32_t lo;       // first staged node id
    uint32_t n;       // number of staged nodes
    float4* pm;
    float4* dip;      // winding kernel only
    float* cdf;
    uint32_t* meta;
    int32_t* fc;
};

__device__ __forceinline__ float4 ld_pm(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? S.pm[i] : __ldg(&T.pm[v]);
}
__device__ __forceinline__ float4 ld_dip(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? S.dip[i] : __ldg(&T.dip[v]);
}
__device__ __forceinline__ float ld_cdf(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? S.cdf[i] : __ldg(&T.cdf[v]);
}
__device__ __forceinline__ uint32_t ld_meta(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? S.meta[i] : __ldg(&T.meta[v]);
}
__device__ __forceinline__ int32_t ld_fc(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? S.fc[i] : __ldg(&T.fc[v]);
}

// m f(p, q) of a node record (not used for the smooth distance, which works in exp frames)
template <int KIND>
__device__ __forceinline__ float node_value(const TreeView& T, const Stage& S, int32_t v, float4 pm, float3 q,
                                            const KernelParams& kp)
{
    if constexpr (KIND == SBH_COULOMB) return term_coulomb(pm, q, kp.eps2);
    else if constexpr (KIND == SBH_WINDING) return term_winding(pm, ld_dip(T, S, v), q);
    else return term_affine(pm, q, kp.g);
}

// child index (0-based) picked by the 24-bit draw x: mass -> the number of prefix fractions <= u
// among all but the last child; count -> the child holding point floor(u * |T|) of the node's
// range. Both are found by binary search (prefix fractions and child ranges are nondecreasing),
// which gives the same index as counting.
__device__ __forceinline__ int pick_child(const TreeView& T, const Stage& S, int32_t node, int32_t f, int nc, uint32_t x,
                                          int sampling)
{
    if (sampling == 0) {
        const float u = unit24(x);
        int lo = 0, hi = nc - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ld_cdf(T, S, f + mid) <= u) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    }
    const int32_t b = __ldg(&T.nb[node]);
    const int32_t cnt = __ldg(&T.ne[node]) - b;
    const int32_t target = b + (int32_t)(((uint64_t)(x >> 8) * (uint64_t)cnt) >> 24);
    int lo = 1, hi = nc;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&T.nb[f + mid]) <= target) lo = mid + 1;
        else hi = mid;
    }
    return lo - 1;
}

struct Params {
    TreeView T;
    const float* Q;
    int64_t nq;
    KernelParams kp;
    int S;
    uint2 key;
    int sampling, rr, coherent, raw_sum;
    float* out;
};

// One decision per lane (Algorithm 2's loop body up to the break test). On a continue the lane
// appends a swap task for its node and a decision task for the chosen child.
template <int KIND>
__device__ __forceinline__ void decide(const Params& P, const Stage& S, WarpState& W, const float* sdiam, bool valid,
                                       int32_t node,
                                       uint32_t tag, int32_t ai, float prr, float dT, float wT, float wa,
                                       uint32_t& d_tail, uint32_t& s_tail)
{
    const TreeView& T = P.T;
    bool cont = false;
    int32_t child = 0;
    float dc = 0.0f, wc = 0.0f, w = 0.0f, prr2 = 0.0f;
    const uint32_t slot = tag & 31u;
    if (valid) {
        const uint32_t depth = (tag >> 5) & 0xFFu, s = tag >> 13;
        const float3 q = make_float3(W.qx[slot], W.qy[slot], W.qz[slot]);
        const uint4 x = philox4x32_10(make_uint4(W.qctr[slot], (uint32_t)ai, s, depth), P.key);
        const uint32_t mT = ld_meta(T, S, node);
        const int32_t f = ld_fc(T, S, node);
        const int nc = (int)meta_nchild(mT);
        child = f + pick_child(T, S, node, f, nc, x.x, P.sampling);
        const float4 pc = ld_pm(T, S, child);
        const uint32_t mc = ld_meta(T, S, child);
        dc = dist_rn(pc.x, pc.y, pc.z, q);
        float p;
        if (P.rr == 0) p = rr_prob_rn(dT, sdiam[meta_level(mT)], dc, sdiam[meta_level(mc)]);
        else p = (P.rr == 1) ? 1.0f : 0.5f;
        cont = unit24(x.y) < p;
        if (cont) {
            prr2 = prr * p;
            const float pagg = wT / wa;
            w = 1.0f / (pagg * prr2) / (float)P.S;
            wc = P.sampling ? (float)(__ldg(&T.ne[child]) - __ldg(&T.nb[child])) : pc.w;
            // a path that reaches a source point stops there: no decision task for it (levels
            // strictly increase, so depth < kMaxDepth always holds; the test only guards a damaged tree)
            if (meta_kind(mc) == kPoint || depth + 1 >= (uint32_t)kMaxDepth) wc = -1.0f;
        }
    }
    const unsigned push_s = __ballot_sync(0xFFFFFFFFu, cont);
    const unsigned push_d = __ballot_sync(0xFFFFFFFFu, cont && wc >= 0.0f);
    if (cont) {
        const uint32_t i = (s_tail + __popc(push_s & lanemask_lt())) & kRingMask;
        W.s_node[i] = node;
        W.s_slot[i] = slot;
        W.s_w[i] = w;
        if (wc >= 0.0f) {
            const uint32_t k = (d_tail + __popc(push_d & lanemask_lt())) & kRingMask;
            W.d_node[k] = child;
            W.d_tag[k] = tag + (1u << 5);  // depth + 1
            W.d_ai[k] = ai;
            W.d_prr[k] = prr2;
            W.d_dT[k] = dc;
            W.d_wT[k] = wc;
            W.d_wa[k] = wa;
        }
    }
    s_tail += __popc(push_s);
    d_tail += __popc(push_d);
    __syncwarp();
}

// Run up to 32 decision tasks from the front of the ring.
template <int KIND>
__device__ __forceinline__ void decision_batch(const Params& P, const Stage& S, WarpState& W, const float* sdiam,
                                               uint32_t& d_head,
                                               uint32_t& d_tail, uint32_t& s_tail)
{
    const uint32_t avail = d_tail - d_head;
    const uint32_t take = avail < 32u ? avail : 32u;
    const bool valid = lane_id() < take;
    int32_t node = 0, ai = 0;
    uint32_t tag = 0;
    float prr = 0.f, dT = 0.f, wT = 0.f, wa = 1.f;
    if (valid) {
        const uint32_t i = (d_head + lane_id()) & kRingMask;
        node = W.d_node[i]; tag = W.d_tag[i]; ai = W.d_ai[i]; prr = W.d_prr[i]; dT = W.d_dT[i];
        wT = W.d_wT[i]; wa = W.d_wa[i];
    }
    __syncwarp();  // every task is read before new ones may reuse its slot
    d_head += take;
    decide<KIND>(P, S, W, sdiam, valid, node, tag, ai, prr, dT, wT, wa, d_tail, s_tail);
}

// Run up to 32 swap tasks: w * (sum_children m_c f(p_c, q) - m_T f(p_T, q)), added to the
// query's sum in lane order.
template <int KIND>
__device__ __forceinline__ void swap_batch(const Params& P, const Stage& S, WarpState& W, uint32_t& s_head,
                                           uint32_t s_tail)
{
    const TreeView& T = P.T;
    const uint32_t avail = s_tail - s_head;
    const uint32_t take = avail < 32u ? avail : 32u;
    const bool valid = lane_id() < take;
    int32_t node = 0;
    uint32_t slot = 32u + lane_id();  // unique key for idle lanes
    float w = 0.0f;
    if (valid) {
        const uint32_t i = (s_head + lane_id()) & kRingMask;
        node = W.s_node[i];
        slot = W.s_slot[i];
        w = W.s_w[i];
    }
    __syncwarp();
    s_head += take;
    float v = 0.0f, r = 3.0e38f;
    if (valid) {
        const float3 q = make_float3(W.qx[slot], W.qy[slot], W.qz[slot]);
        const uint32_t m = ld_meta(T, S, node);
        const int32_t f = ld_fc(T, S, node);
        const int nc = (int)meta_nchild(m);
        const float4 pT = ld_pm(T, S, node);
        if constexpr (KIND == SBH_SMOOTHDIST) {
            const float a = P.kp.alpha;
            r = dist_fast(pT, q);
            v = -w * pT.w;
            for (int k = 0; k < nc; ++k) {
                const float4 pc = ld_pm(T, S, f + k);
                const float d = dist_fast(pc, q);
                if (d < r) { v *= __expf(-a * (r - d)); r = d; }
                v = fmaf(w * pc.w, __expf(-a * (d - r)), v);
            }
        } else {
            // two independent partial sums: two child records in flight per iteration
            float s0 = 0.0f, s1 = 0.0f;
            int k = 0;
            for (; k + 1 < nc; k += 2) {
                const float4 p0 = ld_pm(T, S, f + k), p1 = ld_pm(T, S, f + k + 1);
                s0 += node_value<KIND>(T, S, f + k, p0, q, P.kp);
                s1 += node_value<KIND>(T, S, f + k + 1, p1, q, P.kp);
            }
            if (k < nc) s0 += node_value<KIND>(T, S, f + k, ld_pm(T, S, f + k), q, P.kp);
            v = w * ((s0 + s1) - node_value<KIND>(T, S, node, pT, q, P.kp));
        }
    }
    // lane-ordered sum over the tasks of each query
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, slot);
    float tot = 0.0f, tr = 3.0e38f;
    for (unsigned rest = peers; rest; rest &= rest - 1u) {
        const int src = __ffs(rest) - 1;
        const float vs = __shfl_sync(peers, v, src);
        if constexpr (KIND == SBH_SMOOTHDIST) {
            const float rs = __shfl_sync(peers, r, src);
            const float a = P.kp.alpha;
            if (rs < tr) { tot = tot * __expf(-a * (tr - rs)) + vs; tr = rs; }
            else tot = fmaf(vs, __expf(-a * (rs - tr)), tot);
        } else {
            tot += vs;
        }
    }
    if (valid && lane_id() == (uint32_t)(__ffs(peers) - 1)) {
        if constexpr (KIND == SBH_SMOOTHDIST) {
            const float a = P.kp.alpha;
            float qr = W.ref[slot], qa = W.acc[slot];
            if (tr < qr) { qa = qa * __expf(-a * (qr - tr)) + tot; qr = tr; }
            else qa = fmaf(tot, __expf(-a * (tr - qr)), qa);
            W.ref[slot] = qr;
            W.acc[slot] = qa;
        } else {
            W.acc[slot] += tot;
        }
    }
    __syncwarp();
}

// One tile of 32 queries (query index tile * 32 + lane within the set described by P), run by
// one warp: control variates and depth-0 decisions lane-parallel, everything else as tasks.
template <int KIND>
__device__ __forceinline__ void run_tile(const Params& P, const Stage& S, WarpState& W, const float* sdiam,
                                         int64_t tile)
{
    const TreeView& T = P.T;
    const int32_t first_sub = T.ctrl->first_sub;
    const int n_sub = T.ctrl->n_sub;
    const uint32_t lane = lane_id();
    const int64_t j = tile * 32 + lane;
    const bool active = j < P.nq;
    float3 q = make_float3(0.f, 0.f, 0.f);
    if (active) q = make_float3(P.Q[3 * j], P.Q[3 * j + 1], P.Q[3 * j + 2]);
    W.qx[lane] = q.x; W.qy[lane] = q.y; W.qz[lane] = q.z;
    W.qctr[lane] = P.coherent ? 0u : (uint32_t)j;
    W.acc[lane] = 0.0f;
    W.ref[lane] = 3.0e38f;
    __syncwarp();
    float cv = 0.0f;
    ExpAcc ex;
    ex.init(3.0e38f);
    uint32_t d_head = 0, d_tail = 0, s_head = 0, s_tail = 0;

    for (int ai = 0; ai < n_sub; ++ai) {
        const int32_t a = first_sub + ai;
        const float4 pa = ld_pm(T, S, a);
        const uint32_t ma = ld_meta(T, S, a);
        if (active) {  // control variate CV_a
            if constexpr (KIND == SBH_SMOOTHDIST) {
                const float d = dist_fast(pa, q);
                ex.lower(d, P.kp.alpha);
                ex.acc = fmaf(pa.w, ex.scale(d, P.kp.alpha), ex.acc);
            } else {
                cv += node_value<KIND>(T, S, a, pa, q, P.kp);
            }
        }
        if (meta_kind(ma) == kPoint) continue;
        const float wa = P.sampling ? (float)(__ldg(&T.ne[a]) - __ldg(&T.nb[a])) : pa.w;
        const float da = dist_rn(pa.x, pa.y, pa.z, q);
        for (int s = 0; s < P.S; ++s) {
            decide<KIND>(P, S, W, sdiam, active, a, lane | ((uint32_t)s << 13), ai, 1.0f, da, wa, wa, d_tail, s_tail);
            while (s_tail - s_head >= 32u) swap_batch<KIND>(P, S, W, s_head, s_tail);
            while (d_tail - d_head >= 32u) {
                decision_batch<KIND>(P, S, W, sdiam, d_head, d_tail, s_tail);
                while (s_tail - s_head >= 32u) swap_batch<KIND>(P, S, W, s_head, s_tail);
            }
        }
    }
    // drain the partial batches
    while (d_tail != d_head || s_tail != s_head) {
        if (s_tail != s_head) swap_batch<KIND>(P, S, W, s_head, s_tail);
        if (d_tail != d_head) decision_batch<KIND>(P, S, W, sdiam, d_head, d_tail, s_tail);
    }
    __syncwarp();
    if (active) {
        if constexpr (KIND == SBH_SMOOTHDIST) {
            const float a = P.kp.alpha;
            float r = W.ref[lane], v = W.acc[lane];
            // merge the swap sum into the control-variate sum
            if (r < ex.ref) { ex.acc = ex.acc * __expf(-a * (ex.ref - r)) + v; ex.ref = r; }
            else ex.acc = fmaf(v, __expf(-a * (r - ex.ref)), ex.acc);
            if (P.raw_sum) P.out[j] = ex.acc * __expf(-a * ex.ref);
            else P.out[j] = ex.acc > 0.0f ? ex.ref - __logf(ex.acc) / a : __int_as_float(0x7F800000);
        } else {
            P.out[j] = cv + W.acc[lane];
        }
    }
    __syncwarp();
}

template <int KIND>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 3) k_stoch_batched(Params P, int32_t stage_lo, uint32_t stage_n)
{
    __shared__ WarpState s_state[kWarpsPerBlock];
    __shared__ float sdiam[kDiamLevels];
    extern __shared__ float4 s_stage[];
    Stage S;
    S.lo = stage_lo;
    S.n = stage_n;
    S.pm = s_stage;
    S.dip = s_stage + stage_n;
    S.cdf = (float*)(S.dip + (KIND == SBH_WINDING ? stage_n : 0));
    S.meta = (uint32_t*)(S.cdf + stage_n);
    S.fc = (int32_t*)(S.meta + stage_n);
    for (uint32_t i = threadIdx.x; i < stage_n; i += blockDim.x) {
        const int32_t v = stage_lo + (int32_t)i;
        S.pm[i] = __ldg(&P.T.pm[v]);
        if (KIND == SBH_WINDING) S.dip[i] = __ldg(&P.T.dip[v]);
        S.cdf[i] = __ldg(&P.T.cdf[v]);
        S.meta[i] = __ldg(&P.T.meta[v]);
        S.fc[i] = __ldg(&P.T.fc[v]);
    }
    if (threadIdx.x < kDiamLevels) sdiam[threadIdx.x] = P.T.ctrl->diam[threadIdx.x];
    __syncthreads();
    WarpState& W = s_state[threadIdx.x >> 5];
    const int64_t n_tiles = (P.nq + 31) / 32;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t warp_stride = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t tile = warp_global; tile < n_tiles; tile += warp_stride) run_tile<KIND>(P, S, W, sdiam, tile);
}

// ------------------------------------------------------------------------------------------------
// Many independent problems in one persistent launch: every warp takes the next 32-query tile
// from a global counter (dynamic balance over sets of very different sizes, no waiting) and runs it
// against its set's tree. Query indices are local to each set, so every set's output equals what
// sbh_eval returns for that set alone.
// ------------------------------------------------------------------------------------------------
struct SetDesc {
    TreeView T;
    const float* Q;
    float* out;
    int64_t nq;
    int64_t tile_begin;  // first global tile of this set
};

struct MultiParams {
    const SetDesc* sets;
    int n_sets;
    int64_t total_tiles;
    unsigned long long* counter;
    Params base;  // kernel, samples, key and options shared by all sets
};

template <int KIND>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 3) k_stoch_multi(MultiParams M)
{
    __shared__ WarpState s_state[kWarpsPerBlock];
    __shared__ float s_diam[kWarpsPerBlock][kDiamLevels];
    const int warp = threadIdx.x >> 5;
    WarpState& W = s_state[warp];
    float* sdiam = s_diam[warp];
    Stage S;
    S.lo = 0; S.n = 0; S.pm = nullptr; S.dip = nullptr; S.cdf = nullptr; S.meta = nullptr; S.fc = nullptr;
    Params P = M.base;
    int cur = -1;
    const uint32_t lane = lane_id();
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(M.counter, 1ull);
        const int64_t tile = (int64_t)__shfl_sync(0xFFFFFFFFu, t, 0);
        if (tile >= M.total_tiles) break;
        // the last set whose first tile is <= tile (empty sets are skipped by taking the last)
        int lo = 0, hi = M.n_sets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (M.sets[mid].tile_begin <= tile) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {
            cur = lo;
            const SetDesc& D = M.sets[lo];
            P.T = D.T; P.Q = D.Q; P.out = D.out; P.nq = D.nq;
            if (lane < (uint32_t)kDiamLevels) sdiam[lane] = D.T.ctrl->diam[lane];
            __syncwarp();
        }
        run_tile<KIND>(P, S, W, sdiam, tile - M.sets[lo].tile_begin);
    }
}

template <int KIND>
static cudaError_t launch_kind(const Params& P, unsigned blocks, int32_t lo, uint32_t n, cudaStream_t s)
{
    const size_t bytes = (size_t)n * (sizeof(float4) * (KIND == SBH_WINDING ? 2 : 1) + 3 * sizeof(uint32_t));
    cudaError_t e = cudaFuncSetAttribute(k_stoch_batched<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_stoch_batched<KIND><<<blocks, 32 * kWarpsPerBlock, bytes, s>>>(P, lo, n);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_stoch_batched(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                                 const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                                 cudaStream_t s)
{
    if (nq <= 0) return cudaSuccess;
    Params P;
    P.T = T; P.Q = Q; P.nq = nq; P.kp = kp; P.S = S;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.sampling = o.sampling; P.rr = o.rr; P.coherent = o.seed_mode; P.raw_sum = o.raw_sum; P.out = out;
    const int64_t tiles = (nq + 31) / 32;
    int64_t blocks = (tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (blocks > 152 * 16) blocks = 152 * 16;
    // stage generations 1 and 2 (the subdomains and their children), at most kStageMax nodes
    const int32_t lo = host_ctrl.max_depth >= 1 ? host_ctrl.depth_base[1] : 0;
    const int32_t hi = host_ctrl.depth_base[host_ctrl.max_depth >= 2 ? 3 : (host_ctrl.max_depth >= 1 ? 2 : 1)];
    uint32_t n = (uint32_t)(hi > lo ? hi - lo : 0);
    if (n > (uint32_t)kStageMax) n = kStageMax;
    cudaError_t e;
    switch (kp.kind) {
    case SBH_COULOMB: e = launch_kind<SBH_COULOMB>(P, (unsigned)blocks, lo, n, s); break;
    case SBH_WINDING: e = launch_kind<SBH_WINDING>(P, (unsigned)blocks, lo, n, s); break;
    case SBH_SMOOTHDIST: e = launch_kind<SBH_SMOOTHDIST>(P, (unsigned)blocks, lo, n, s); break;
    case SBH_AFFINE: e = launch_kind<SBH_AFFINE>(P, (unsigned)blocks, lo, n, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_stoch_multi(const void* set_descs, int n_sets, int64_t total_tiles, unsigned long long* counter,
                               const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, cudaStream_t s)
{
    if (total_tiles <= 0) return cudaSuccess;
    MultiParams M;
    M.sets = (const SetDesc*)set_descs;
    M.n_sets = n_sets;
    M.total_tiles = total_tiles;
    M.counter = counter;
    Params& P = M.base;
    P.T = TreeView{}; P.Q = nullptr; P.nq = 0; P.kp = kp; P.S = S; P.out = nullptr;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.sampling = o.sampling; P.rr = o.rr; P.coherent = o.seed_mode; P.raw_sum = o.raw_sum;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    // persistent: three blocks per SM
    const unsigned blocks = 152 * 3;
    switch (kp.kind) {
    case SBH_COULOMB: k_stoch_multi<SBH_COULOMB><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(M); break;
    case SBH_WINDING: k_stoch_multi<SBH_WINDING><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(M); break;
    case SBH_SMOOTHDIST: k_stoch_multi<SBH_SMOOTHDIST><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(M); break;
    case SBH_AFFINE: k_stoch_multi<SBH_AFFINE><<<blocks, 32 * kWarpsPerBlock, 0, s>>>(M); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

size_t multi_set_desc_bytes() { return sizeof(SetDesc); }

void multi_fill_desc(void* dst, const TreeView& T, const float* Q, float* out, int64_t nq, int64_t tile_begin)
{
    SetDesc* d = (SetDesc*)dst;
    d->T = T;
    d->Q = Q;
    d->out = out;
    d->nq = nq;
    d->tile_begin = tile_begin;
}

}  // namespace sbh

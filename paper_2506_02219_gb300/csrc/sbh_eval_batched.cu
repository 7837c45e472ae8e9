// sbh_eval_batched.cu -- the stratified path estimator (Madan et al. 2025, Sec. 3.3, Eq. 5-7,
// Algorithm 2) organised for full SIMT lanes.
//
// The arithmetic and the random stream are those of Algorithm 2 (see sbh_eval.cu for the
// statement); what differs is how a warp schedules the work of its 32 queries. Every decision is
// a task:
//   decision task  (query, node T, depth k, ...): draw the child, play the roulette (Eq. 5);
//   swap task      (query, node T, weight w):     add w * Delta_T (Eq. 6) to the query's sum.
// A continuing decision emits one swap task and, unless the child is a source point, one
// decision task for the chosen child. The random words of a decision are drawn when its task is
// made (at depth 0 per subdomain, every lane for its own query): a draw whose roulette stops the
// path whichever child is picked (certain_stop) makes no task at all, so the pick, the child's
// record and the roulette test run only for paths that may continue. One Philox block serves two
// consecutive depths (words 0, 1 at the even depth, 2, 3 at the odd one), so a depth-0 draw also
// gives the words of the depth-1 decision that follows it. Tasks wait in two per-warp
// rings in shared memory and are run 32 at a time, one per lane, so the
// lanes stay busy however the paths of the 32 queries diverge. Swap results reach a query's sum
// through a lane-ordered reduction among the tasks of that query, so results are deterministic.
//
// Three instances share this schedule: the estimator; its adjoint (GRAD: every term also adds its
// query gradient, with the same weights); and the learned child proposal (LEARNED: the children of
// a batch's gated decisions are scored together on the tensor cores, see learned_picks). One more
// kernel, k_stoch_multi, runs many independent problems in one persistent launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_eval.cuh"
#include "sbh_learned.cuh"

namespace sbh {

namespace {

// resident blocks per SM the register budget is set for, and the most nodes staged per block
// (5 and 128 measured best: more warps in flight beat a deeper stage, which L1 mostly covers; at
// 5 blocks, 48 registers, the winding instance spills 16 bytes and still runs 2% faster than 4)
#ifndef SBH_BATCHED_MIN_BLOCKS
#define SBH_BATCHED_MIN_BLOCKS 5
#endif
// the smooth-distance instance fits 5 blocks per SM in 48 registers without spills (2% faster)
#ifndef SBH_SMOOTH_MIN_BLOCKS
#define SBH_SMOOTH_MIN_BLOCKS 5
#endif
// resident blocks per SM the estimator is built for, per kernel kind
template <int KIND>
constexpr int value_min_blocks() { return KIND == SBH_SMOOTHDIST ? SBH_SMOOTH_MIN_BLOCKS : SBH_BATCHED_MIN_BLOCKS; }
// the multi-set kernel holds its set's parameters too: 4 blocks (5 would spill) but for the smooth
// distance (5)
#ifndef SBH_MULTI_MIN_BLOCKS
#define SBH_MULTI_MIN_BLOCKS 4
#endif
template <int KIND>
constexpr int multi_min_blocks() { return KIND == SBH_SMOOTHDIST ? SBH_SMOOTH_MIN_BLOCKS : SBH_MULTI_MIN_BLOCKS; }
#ifndef SBH_STAGE_MAX
#define SBH_STAGE_MAX 128
#endif
// A subdomain's depth-0 decisions are taken in place by the warp (every lane at the same node)
// when more than this many of its lanes may continue, else queued as decision tasks. Measured on
// the estimator: 20 (16 to 24 within 1%). The smooth-distance, adjoint and learned instances
// always queue them (32): their larger code ran slower with the decision inlined twice (smooth
// distance 2.55 against 2.29 ms, adjoint 32.7 against 31.3), and queueing let the learned one keep
// its state in registers.
#ifndef SBH_DEPTH0_QUEUE_MAX
#define SBH_DEPTH0_QUEUE_MAX 20
#endif
// resident blocks per SM of the adjoint instance: 4 (64 registers) measured 0.6-0.9% faster than 3
#ifndef SBH_GRAD_MIN_BLOCKS
#define SBH_GRAD_MIN_BLOCKS 4
#endif
#ifndef SBH_DEPTH0_QUEUE_MAX_SMOOTH
#define SBH_DEPTH0_QUEUE_MAX_SMOOTH 32
#endif
template <int KIND, bool LEARNED, bool GRAD>
constexpr int depth0_queue_max()
{
    return (LEARNED || GRAD) ? 32 : (KIND == SBH_SMOOTHDIST ? SBH_DEPTH0_QUEUE_MAX_SMOOTH : SBH_DEPTH0_QUEUE_MAX);
}
// resident blocks per SM of the learned-proposal instance: four (64 registers) fit its shared
// memory without a stage and with 64-row scoring groups; 8-16% faster than three blocks of 80
// registers with the stage and 128-row groups
#ifndef SBH_LEARNED_MIN_BLOCKS
#define SBH_LEARNED_MIN_BLOCKS 4
#endif
// most blocks launched per SM (the rest of the tiles are taken in grid-stride order)
#ifndef SBH_GRID_BLOCKS_PER_SM
#define SBH_GRID_BLOCKS_PER_SM 96
#endif

constexpr int kWarpsPerBlock = 8;
constexpr int kRing = 64;  // ring capacity per warp; at most 63 tasks wait at any time
constexpr uint32_t kRingMask = kRing - 1;
// a decision task's tag: the query's slot in the warp (5 bits), the depth (5 bits: at most
// kMaxDepth generations), the subdomain index (6 bits: a root has at most 64 children, and a
// multi-point root leaf at most 64 points) and the sample index (16 bits)
__device__ __forceinline__ uint32_t make_tag(uint32_t slot, uint32_t depth, uint32_t ai, uint32_t sample)
{
    return slot | depth << 5 | ai << 10 | sample << 16;
}
__device__ __forceinline__ uint32_t tag_slot(uint32_t t) { return t & 31u; }
__device__ __forceinline__ uint32_t tag_depth(uint32_t t) { return (t >> 5) & 31u; }
__device__ __forceinline__ uint32_t tag_sub(uint32_t t) { return (t >> 10) & 63u; }
__device__ __forceinline__ uint32_t tag_sample(uint32_t t) { return t >> 16; }
static_assert(kMaxDepth < 32 && SBH_MAX_SAMPLES_PER_SUBDOMAIN <= 65536 && kMaxLeafSize <= 64, "tag fields");
// unroll factor of a swap's loop over pairs of children, measured per kernel: 2 for the terms of
// one 16-byte record (Coulomb, affine), 1 for the winding term and its 32-byte record. Left to the
// compiler, the Coulomb instance unrolled further and spilled registers.
#ifndef SBH_SWAP_UNROLL_WINDING
#define SBH_SWAP_UNROLL_WINDING 1
#endif
template <int KIND>
constexpr int swap_unroll() { return KIND == SBH_WINDING ? SBH_SWAP_UNROLL_WINDING : 2; }

// per-warp shared state, structure of arrays
template <int KIND>
struct WarpState {
    // decision tasks
    int32_t d_node[kRing];
    uint32_t d_x0[kRing];    // the decision's random words: child pick
    uint32_t d_x1[kRing];    //                              roulette
    uint32_t d_tag[kRing];   // slot | depth << 5 | subdomain << 10 | sample << 16
    // depth >= 1: the bits of p_rr and of the node's mass (or point count, or with the learned
    // proposal the probability of reaching the node); depth 0, where those are 1 and the
    // subdomain's weight: words 2 and 3 of the decision's Philox block (the depth-1 draws)
    uint32_t d_w2[kRing];
    uint32_t d_w3[kRing];
    float d_dT[kRing];       // correctly rounded distance from the query to the node's centre
    // swap tasks
    int32_t s_node[kRing];
    uint32_t s_slot[kRing];
    float s_w[kRing];
    // the warp's 32 queries
    float qx[32], qy[32], qz[32];
    uint32_t qctr[32];       // counter word 0 of each query's random stream
    float acc[32];           // sum of the swap terms (smooth distance: in units of exp(-alpha ref))
    float ref[KIND == SBH_SMOOTHDIST ? 32 : 1];  // smooth distance: the frame of acc (unused otherwise)
    float slack;             // certain_stop's slack for the current tree
    int32_t first_sub;       // the current tree's first subdomain
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

// The subdomains (node generation 1) are read by every query: each block copies the first
// kStageMax nodes of generations 1 and 2 (the subdomains, then the first of their children) into
// shared memory at start and reads them there; everything else is read through L1.
constexpr int kStageMax = SBH_STAGE_MAX;

// The stage sits at the start of the dynamic shared memory in a fixed layout of kStageMax entries
// per array, so that its arrays are constant shared-memory addresses (no pointers held in
// registers): pm [kStageMax] float4, cdf, meta and fc [kStageMax] 4-byte words, gd [kStageMax]
// bytes, then for the winding kernel dip [kStageMax] float4. What else a block keeps in dynamic
// shared memory follows.
extern __shared__ float4 s_dyn[];
constexpr size_t kStageBaseBytes = (size_t)kStageMax * (sizeof(float4) + 3 * sizeof(uint32_t) + sizeof(uint8_t));
static_assert(kStageBaseBytes % 16 == 0, "dip and what follows the stage stay 16-byte aligned");
template <int KIND>
constexpr size_t stage_bytes() { return kStageBaseBytes + (KIND == SBH_WINDING ? kStageMax * sizeof(float4) : 0); }

struct Stage {
    int32_t lo;       // first staged node id
    uint32_t n;       // number of staged nodes (0: nothing staged)
    __device__ __forceinline__ static float4* pm() { return s_dyn; }
    __device__ __forceinline__ static float* cdf() { return reinterpret_cast<float*>(s_dyn + kStageMax); }
    __device__ __forceinline__ static uint32_t* meta() { return reinterpret_cast<uint32_t*>(cdf() + kStageMax); }
    __device__ __forceinline__ static int32_t* fc() { return reinterpret_cast<int32_t*>(meta() + kStageMax); }
    __device__ __forceinline__ static uint8_t* gd() { return reinterpret_cast<uint8_t*>(fc() + kStageMax); }
    __device__ __forceinline__ static float4* dip()  // winding kernel only
    {
        return reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(s_dyn) + kStageBaseBytes);
    }
    template <int KIND>
    __device__ __forceinline__ static unsigned char* after()
    {
        return reinterpret_cast<unsigned char*>(s_dyn) + stage_bytes<KIND>();
    }
};

__device__ __forceinline__ float4 ld_pm(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? Stage::pm()[i] : __ldg(&T.pm[v]);
}
__device__ __forceinline__ float4 ld_dip(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? Stage::dip()[i] : __ldg(&T.dip[v]);
}
__device__ __forceinline__ uint32_t ld_meta(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? Stage::meta()[i] : __ldg(&T.meta[v]);
}
__device__ __forceinline__ int32_t ld_fc(const TreeView& T, const Stage& S, int32_t v)
{
    const uint32_t i = (uint32_t)(v - S.lo);
    return i < S.n ? Stage::fc()[i] : __ldg(&T.fc[v]);
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
// range. Mass: the scan starts at the guide entry of u's slot floor(u nc) (k_guide), a lower bound
// of that number, and steps up while the prefix fractions (nondecreasing) are <= u: the same
// index as counting, in one or two reads on average. Count: binary search over the child ranges.
__device__ __forceinline__ int pick_child(const TreeView& T, const Stage& S, int32_t node, int32_t f, int nc, uint32_t x,
                                          int sampling)
{
    if (sampling == 0) {
        const float u = unit24(x);
        const bool st = f >= S.lo && (uint32_t)(f + nc - S.lo) <= S.n;
        const float* cdf = st ? Stage::cdf() + (f - S.lo) : T.cdf + f;
        const uint8_t* gd = st ? Stage::gd() + (f - S.lo) : T.gd + f;
        int i = gd[((x >> 8) * (uint32_t)nc) >> 24];  // (x >> 8) nc < 2^30
        while (i < nc - 1 && cdf[i] <= u) ++i;
        return i;
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

// per-warp scratch of the learned pick: one chunk of FP16 feature rows, the rows of one group of
// decisions (exp of the clamped score, child mass), and the gated decisions of the batch
// (rows per group of decisions: 64, one decision's widest child set, keeps four blocks' shared
// memory within an SM's)
#ifndef SBH_LEARN_ROWS
#define SBH_LEARN_ROWS 64
#endif
constexpr int kLearnRows = SBH_LEARN_ROWS;
static_assert(kLearnRows >= 64 && kLearnRows <= 256, "a group holds at least one decision's 64 children; rk is 8-bit");
struct __align__(16) LearnScratch {
    uint32_t A[32 * kChunkWords];
    float sc[32];
    float pe[kLearnRows];   // within each decision: prefix sums of exp(clamped score)
    float pm[kLearnRows];   //                       prefix sums of the child masses
    uint8_t rk[kLearnRows]; // decision (compact index) of each row
    float qx[32], qy[32], qz[32];
    float lnBT[32], lnmT[32], lndT[32];  // logs of the node's cell diagonal, mass, guarded distance
    float u[32];            // the decision's uniform draw
    float prob[32];         // out: probability of the child picked
    int32_t f[32];
    int32_t off[32];
    int32_t nc[32];
    int32_t pick[32];       // out: child picked (0-based)
};

struct Params {
    TreeView T;
    const float* Q;
    int64_t nq;
    KernelParams kp;
    int S;
    uint2 key;
    int sampling, rr, coherent, raw_sum;
    float* out;
    int64_t qbase;           // index of the first query in the caller's whole query set (chunked runs)
    float* grad;             // adjoint only: d out / d q, [nq][3]
    // learned proposal only
    const __half* mlpw;
    float near;
};

// whether the learned-proposal instance stages nodes (1) or reads every record through L1 (0),
// leaving its shared memory to the scoring scratch (0: a fourth block fits)
#ifndef SBH_LEARNED_STAGE
#define SBH_LEARNED_STAGE 0
#endif
// bytes of dynamic shared memory the stage takes in an instance
template <int KIND, bool LEARNED>
constexpr size_t stage_bytes_of() { return (LEARNED && !SBH_LEARNED_STAGE) ? 0 : stage_bytes<KIND>(); }

// What follows the stage in dynamic shared memory, at fixed offsets: the learned proposal's weight
// fragments and one scoring scratch per warp, or the adjoint's per-warp [32][3] gradient sums
template <int KIND>
__device__ __forceinline__ MlpFrag* mlp_frag()
{
    return reinterpret_cast<MlpFrag*>(reinterpret_cast<unsigned char*>(s_dyn) + stage_bytes_of<KIND, true>());
}
template <int KIND>
__device__ __forceinline__ LearnScratch* learn_scratch()
{
    return reinterpret_cast<LearnScratch*>(reinterpret_cast<unsigned char*>(mlp_frag<KIND>()) + sizeof(MlpFrag));
}
template <int KIND>
__device__ __forceinline__ float* grad_sums() { return reinterpret_cast<float*>(Stage::after<KIND>()); }

// The learned picks of the gated lanes of a decision batch (every lane of the warp takes part).
// Rows = the children of the gated decisions in lane order, processed in groups of whole
// decisions of at most kLearnRows rows, 32 rows (one per lane) at a time: features, tensor-core
// scores, and segmented prefix sums (restarting at each decision's first row) of exp(score) and
// of the child masses. Then each row tests whether its decision's draw u falls in its interval
// [cum_{r-1}, cum_r) of the mixed proposal's cumulative distribution
//   cum_r = (1 - eps) Pe_r / Z + eps Pm_r / M   (Z, M: the decision's totals),
// the last row taking [cum_{r-1}, 1): exactly one row of each decision is picked, and its
// probability is the width of its interval.
template <int KIND>
__device__ __forceinline__ void learned_picks(const Params& P, const Stage& S, const float* sdiam, unsigned gm,
                                           bool gated, float3 q, float4 pT, float BT, int32_t f, int nc, float u,
                                           int32_t& child, float& prob)
{
    const float* slnB = sdiam + kDiamLevels;  // ln |B| per level, stored after the diagonals
    const TreeView& T = P.T;
    LearnScratch& L = learn_scratch<KIND>()[threadIdx.x >> 5];
    const uint32_t lane = lane_id();
    const int k = __popc(gm & lanemask_lt());
    const int v = gated ? nc : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    const int off = incl - v;
    if (gated) {
        const float tx = pT.x - q.x, ty = pT.y - q.y, tz = pT.z - q.z;
        const float t2 = tx * tx + ty * ty + tz * tz;
        L.qx[k] = q.x; L.qy[k] = q.y; L.qz[k] = q.z;
        L.f[k] = f; L.off[k] = off; L.nc[k] = nc; L.u[k] = u;
        L.lnBT[k] = __logf(BT);
        L.lnmT[k] = __logf(pT.w);
        L.lndT[k] = __logf((t2 > 0.0f ? t2 * rsqrtf(t2) : 0.0f) + 1e-6f * BT);
    }
    const int G = __popc(gm);
    __syncwarp();
    for (int base_k = 0; base_k < G;) {
        const int off_base = L.off[base_k];
        const bool member = gated && k >= base_k && off + nc - off_base <= kLearnRows;
        const int end_k = base_k + __popc(__ballot_sync(0xFFFFFFFFu, member));
        const int R = L.off[end_k - 1] + L.nc[end_k - 1] - off_base;
        float carry_e = 0.0f, carry_m = 0.0f;  // the open segment's sums at the end of the last chunk
        for (int r0 = 0; r0 < R; r0 += 32) {
            const int r = r0 + (int)lane;
            const bool live = r < R;
            float x[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            float mc = 0.0f;
            bool head = false;
            if (live) {
                int lo = base_k, hi = end_k - 1;  // the decision that owns row r
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (L.off[mid] - off_base <= r) lo = mid;
                    else hi = mid - 1;
                }
                L.rk[r] = (uint8_t)lo;
                const int c = off_base + r - L.off[lo];
                head = c == 0;
                const int32_t ch = L.f[lo] + c;
                const float4 pc = ld_pm(T, S, ch);
                const uint32_t lc = meta_level(ld_meta(T, S, ch));
                // the features of features_of, with fast logarithms and the node's logs shared
                const float vx = pc.x - L.qx[lo], vy = pc.y - L.qy[lo], vz = pc.z - L.qz[lo];
                const float v2 = vx * vx + vy * vy + vz * vz;
                const float Bc = sdiam[lc], lnBc = slnB[lc];
                const float dc = (v2 > 0.0f ? v2 * rsqrtf(v2) : 0.0f) + 1e-6f * Bc;
                const float lndc = __logf(dc);
                x[0] = lndc - lnBc;
                x[1] = __logf(pc.w) - L.lnmT[lo];
                x[2] = lnBc - L.lnBT[lo];
                x[3] = lndc - L.lndT[lo];
                if constexpr (KIND == SBH_WINDING) {
                    const float4 N = ld_dip(T, S, ch);
                    const float n2 = N.x * N.x + N.y * N.y + N.z * N.z;
                    const float inv_n = n2 > 0.0f ? rsqrtf(n2) : 0.0f;
                    x[4] = __fdividef(n2 * inv_n, pc.w);
                    x[5] = __fdividef((vx * N.x + vy * N.y + vz * N.z) * inv_n, dc);
                }
                mc = pc.w;
            }
            store_feature_row(&L.A[lane * kChunkWords], x, live);
            __syncwarp();
            const float sco = score_chunk_shared(*mlp_frag<KIND>(), L.A, L.sc);
            // segmented inclusive prefix sums over the lanes, restarting at each decision's head
            float pe = live ? __expf(clamp_score(sco)) : 0.0f, pm = mc;
            const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
            const unsigned at_or_below = heads & (0xFFFFFFFFu >> (31u - lane));
            const int start = at_or_below ? 31 - __clz(at_or_below) : -1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float ye = __shfl_up_sync(0xFFFFFFFFu, pe, o);
                const float ym = __shfl_up_sync(0xFFFFFFFFu, pm, o);
                if ((int)lane - o >= start && (int)lane >= o) { pe += ye; pm += ym; }
            }
            if (start < 0) { pe += carry_e; pm += carry_m; }  // the segment began in an earlier chunk
            if (live) { L.pe[r] = pe; L.pm[r] = pm; }
            carry_e = __shfl_sync(0xFFFFFFFFu, pe, 31);
            carry_m = __shfl_sync(0xFFFFFFFFu, pm, 31);
        }
        __syncwarp();
        for (int r0 = 0; r0 < R; r0 += 32) {
            const int r = r0 + (int)lane;
            if (r < R) {
                const int kd = L.rk[r];
                const int first = L.off[kd] - off_base, last = first + L.nc[kd] - 1;
                const float a = (1.0f - kMixEps) / L.pe[last], b = kMixEps / L.pm[last];
                const float hi = fmaf(L.pe[r], a, L.pm[r] * b);
                const float lo = r == first ? 0.0f : fmaf(L.pe[r - 1], a, L.pm[r - 1] * b);
                const float ud = L.u[kd];
                if (ud >= lo && (ud < hi || r == last)) {
                    L.pick[kd] = r - first;
                    L.prob[kd] = r == last ? 1.0f - lo : hi - lo;
                }
            }
        }
        __syncwarp();
        if (member) {
            child = f + L.pick[k];
            prob = L.prob[k];
        }
        __syncwarp();
        base_k = end_k;
    }
}

// The Philox block of the path in tag (query slot, subdomain, sample) at the tag's depth k: it
// serves the decisions at depths k - k mod 2 (words 0, 1) and k - k mod 2 + 1 (words 2, 3).
template <int KIND>
__device__ __forceinline__ uint4 draw_block(const PhiloxRoundKeys& K, const WarpState<KIND>& W, uint32_t tag)
{
    return philox4x32_10(make_uint4(W.qctr[tag_slot(tag)], tag_sub(tag), tag_sample(tag), tag_depth(tag) & ~1u), K);
}

// One decision per lane (Algorithm 2's loop body up to the break test), its random words x0, x1
// drawn when the task was made; at depth 0, x2, x3 are the rest of its Philox block, the words of
// the depth-1 decision (D0: every lane's task is at depth 0). On a continue the lane appends a
// swap task for its node and, if the chosen child's own decision may continue, a decision task for
// the child.
// With the learned proposal, wT carries p(path reaches node) (the product of the picks'
// probabilities) and wa = 1, so that p_agg = wT / wa in both cases; its decisions are always queued
// tasks, and ring_i is the task's slot in the ring.
template <int KIND, bool LEARNED, bool D0>
__device__ __forceinline__ void decide(const Params& P, const PhiloxRoundKeys& K, const Stage& S, WarpState<KIND>& W,
                                       const float* sdiam, bool valid, int32_t node, uint32_t x0, uint32_t x1,
                                       uint32_t x2, uint32_t x3, uint32_t tag, float prr, float dT, float wT, float wa,
                                       uint32_t& d_tail, uint32_t& s_tail, uint32_t ring_i = 0)
{
    const TreeView& T = P.T;
    bool cont = false;
    int32_t child = 0;
    float dc = 0.0f, wc = 0.0f, w = 0.0f, prr2 = 0.0f;
    uint32_t slot = tag_slot(tag);
    float3 q = make_float3(0.0f, 0.0f, 0.0f);
    uint32_t mT = 0;
    int32_t f = 0;
    int nc = 0;
    uint32_t y0 = 0, y1 = 0;  // the child's decision, drawn on a continue
    if (valid) {
        q = make_float3(W.qx[slot], W.qy[slot], W.qz[slot]);
        mT = ld_meta(T, S, node);
        f = ld_fc(T, S, node);
        nc = (int)meta_nchild(mT);
    }
    float pick_prob = 1.0f;
    if constexpr (LEARNED) {
        const float4 pT = valid ? ld_pm(T, S, node) : make_float4(0.0f, 0.0f, 0.0f, 1.0f);
        const float BT = sdiam[meta_level(mT)];
        const bool gated = valid && learned_gate(nc, dT, P.near, BT);
        const unsigned gm = __ballot_sync(0xFFFFFFFFu, gated);
        if (valid && !gated) {
            child = f + pick_child(T, S, node, f, nc, x0, 0);
            pick_prob = -pT.w;  // a mass pick: its probability m_c / m_T is formed on a continue
        }
        if (gm) learned_picks<KIND>(P, S, sdiam, gm, gated, q, pT, BT, f, nc, unit24(x0), child, pick_prob);
        // read the task and its query again rather than hold them through the scoring loop
        // (registers): its ring slot is not reused before this decision's pushes below
        if (valid) {
            node = W.d_node[ring_i]; x1 = W.d_x1[ring_i]; tag = W.d_tag[ring_i]; dT = W.d_dT[ring_i];
            x2 = W.d_w2[ring_i]; x3 = W.d_w3[ring_i];
            const bool d0 = tag_depth(tag) == 0u;
            prr = d0 ? 1.0f : __uint_as_float(x2);
            wT = d0 ? wa : __uint_as_float(x3);
            mT = ld_meta(T, S, node);
            slot = tag_slot(tag);
            q = make_float3(W.qx[slot], W.qy[slot], W.qz[slot]);
        }
    } else {
        if (valid) child = f + pick_child(T, S, node, f, nc, x0, P.sampling);
    }
    if (valid) {
        const float4 pc = ld_pm(T, S, child);
        const uint32_t mc = ld_meta(T, S, child);
        dc = dist_rn(pc.x, pc.y, pc.z, q);
        float p = 1.0f;
        const uint32_t lT = meta_level(mT);
        cont = rr_continue(P.rr, unit24(x1), dT, sdiam[lT], lT, dc, meta_level(mc), p);
        if (cont) {
            prr2 = prr * p;
            // 1 / (p_agg p_rr S), p_agg = wT / wa: a weight, never a decision, so the fast quotient
            // (within 2 ulp), exact-rounded only where the divisor passes 2^126 and it does not hold
            const float den = wT * prr2 * (float)P.S;
            w = den < 8.5e37f ? __fdividef(wa, den) : __fdiv_rn(wa, den);
            if constexpr (LEARNED) wc = wT * (pick_prob < 0.0f ? pc.w / -pick_prob : pick_prob);
            else wc = P.sampling ? (float)(__ldg(&T.ne[child]) - __ldg(&T.nb[child])) : pc.w;
            // a path that reaches a source point stops there: no decision task for it (levels
            // strictly increase, so depth < kMaxDepth always holds; the test only guards a damaged
            // tree); nor does one whose next roulette stops it whichever child it draws. The
            // child's words: at depth 0 the rest of this block; deeper, from the child's block.
            const uint32_t kc = tag_depth(tag) + 1u;
            if (meta_kind(mc) == kPoint || kc >= (uint32_t)kMaxDepth) {
                wc = -1.0f;
            } else {
                if (!D0 && kc != 1u) {
                    const uint4 b = draw_block(K, W, tag + (1u << 5));
                    x2 = (kc & 1u) ? b.z : b.x;
                    x3 = (kc & 1u) ? b.w : b.y;
                }
                y0 = x2;
                y1 = x3;
                if (certain_stop(P.rr, unit24(y1), dc, sdiam[meta_level(mc)], W.slack)) wc = -1.0f;
            }
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
            W.d_x0[k] = y0;
            W.d_x1[k] = y1;
            W.d_tag[k] = tag + (1u << 5);  // depth + 1
            W.d_w2[k] = __float_as_uint(prr2);
            W.d_w3[k] = __float_as_uint(wc);
            W.d_dT[k] = dc;
        }
    }
    s_tail += __popc(push_s);
    d_tail += __popc(push_d);
    __syncwarp();
}

// The weight of a path's subdomain a in p_agg: its mass (or point count); 1 with the learned
// proposal, whose wT is already the probability of reaching the node
template <bool LEARNED>
__device__ __forceinline__ float subdomain_weight(const Params& P, const Stage& S, int32_t a)
{
    if constexpr (LEARNED) return 1.0f;
    const TreeView& T = P.T;
    return P.sampling ? (float)(__ldg(&T.ne[a]) - __ldg(&T.nb[a])) : ld_pm(T, S, a).w;
}

// Run up to 32 decision tasks from the front of the ring.
template <int KIND, bool LEARNED>
__device__ __forceinline__ void decision_batch(const Params& P, const PhiloxRoundKeys& K, const Stage& S,
                                               WarpState<KIND>& W, const float* sdiam, uint32_t& d_head,
                                               uint32_t& d_tail, uint32_t& s_tail)
{
    const uint32_t avail = d_tail - d_head;
    const uint32_t take = avail < 32u ? avail : 32u;
    const bool valid = lane_id() < take;
    int32_t node = 0;
    uint32_t tag = 0, x0 = 0, x1 = 0, x2 = 0, x3 = 0;
    float prr = 0.f, dT = 0.f, wT = 0.f, wa = 1.f;
    const uint32_t i = (d_head + lane_id()) & kRingMask;
    if (valid) {
        node = W.d_node[i]; tag = W.d_tag[i]; dT = W.d_dT[i];
        x0 = W.d_x0[i]; x1 = W.d_x1[i]; x2 = W.d_w2[i]; x3 = W.d_w3[i];
    }
    __syncwarp();  // every task is read before new ones may reuse its slot
    d_head += take;
    if (valid) {
        wa = subdomain_weight<LEARNED>(P, S, W.first_sub + (int32_t)tag_sub(tag));
        const bool d0 = tag_depth(tag) == 0u;  // p_rr = 1 and wT = wa at a subdomain
        prr = d0 ? 1.0f : __uint_as_float(x2);
        wT = d0 ? wa : __uint_as_float(x3);
    }
    decide<KIND, LEARNED, false>(P, K, S, W, sdiam, valid, node, x0, x1, x2, x3, tag, prr, dT, wT, wa, d_tail, s_tail,
                                 i);
}

// m f(p, q) and its gradient in q (added to g), for the adjoint: the kernel ∇_q f applied to the
// same terms (dp: the node's dipole sum, winding kernel only)
template <int KIND>
__device__ __forceinline__ float term_vg(float4 pm, float4 dp, float3 q, const KernelParams& kp, float g[3])
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    if constexpr (KIND == SBH_COULOMB) {
        const float e = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, kp.eps2)));
        const float ir = rsqrt_ftz(e);
        const float t = pm.w * ir;
        const float c = t * ir * ir;  // m / e^(3/2)
        g[0] = fmaf(c, dx, g[0]); g[1] = fmaf(c, dy, g[1]); g[2] = fmaf(c, dz, g[2]);
        return t;
    } else if constexpr (KIND == SBH_WINDING) {
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(r2 >= kMinNormal)) return 0.0f;
        const float ir = rsqrt_ftz(r2);
        const float ir3 = ir * ir * ir;
        const float dn = fmaf(dx, dp.x, fmaf(dy, dp.y, dz * dp.z));
        const float c = 3.0f * kInv4Pi * dn * ir3 * ir * ir;  // 3 (d.N) / (4 pi r^5)
        const float b = -kInv4Pi * ir3;                       // -1 / (4 pi r^3)
        g[0] += fmaf(b, dp.x, c * dx); g[1] += fmaf(b, dp.y, c * dy); g[2] += fmaf(b, dp.z, c * dz);
        return kInv4Pi * dn * ir3;
    } else {
        g[0] -= pm.w * kp.g[0]; g[1] -= pm.w * kp.g[1]; g[2] -= pm.w * kp.g[2];
        return pm.w * (1.0f + fmaf(kp.g[0], dx, fmaf(kp.g[1], dy, kp.g[2] * dz)));
    }
}

// The winding term and its query gradient times 4 pi (sums of them are scaled by 1 / (4 pi) once):
// value (d.N) / r^3, gradient -N / r^3 + 3 (d.N) d / r^5 (added to g); 0 at r = 0
__device__ __forceinline__ float winding_vg_4pi(float4 pm, float4 dp, float3 q, float g[3])
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (!(r2 >= kMinNormal)) return 0.0f;
    const float ir = rsqrt_ftz(r2);
    const float ir2 = ir * ir;
    const float ir3 = ir2 * ir;
    const float t = fmaf(dx, dp.x, fmaf(dy, dp.y, dz * dp.z)) * ir3;  // (d.N) / r^3
    const float c = 3.0f * t * ir2;                                   // 3 (d.N) / r^5
    g[0] = fmaf(c, dx, fmaf(-ir3, dp.x, g[0]));
    g[1] = fmaf(c, dy, fmaf(-ir3, dp.y, g[1]));
    g[2] = fmaf(c, dz, fmaf(-ir3, dp.z, g[2]));
    return t;
}

// smooth distance: add m exp(-alpha (d - ref)) and its gradient to (v, g) in the frame exp(-alpha ref),
// lowering ref to d first when d is smaller (v and g scale together)
__device__ __forceinline__ void smooth_vg(float4 pm, float3 q, float alpha, float wm, float& ref, float& v, float g[3])
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ir = rsqrt_ftz(fmaxf(r2, 1e-37f));
    const float d = r2 * ir;
    if (d < ref) {
        const float f = __expf(-alpha * (ref - d));
        v *= f; g[0] *= f; g[1] *= f; g[2] *= f;
        ref = d;
    }
    const float t = wm * __expf(-alpha * (d - ref));
    v += t;
    if (r2 > 0.0f) {
        const float c = alpha * t * ir;  // alpha m exp(-alpha d) / d
        g[0] = fmaf(c, dx, g[0]); g[1] = fmaf(c, dy, g[1]); g[2] = fmaf(c, dz, g[2]);
    }
}

// One swap: w * (sum_children m_c f(p_c, q) - m_T f(p_T, q)) at node `node` for the query at q.
// v gets the value (smooth distance: in the frame exp(-alpha r), r the smallest distance met);
// GRAD: g gets the same for the terms' query gradients.
template <int KIND, bool GRAD>
__device__ __forceinline__ void swap_terms(const Params& P, const Stage& S, int32_t node, float3 q, float w, float& v,
                                           float& r, float g[3])
{
    const TreeView& T = P.T;
    const uint32_t m = ld_meta(T, S, node);
    const int32_t f = ld_fc(T, S, node);
    const int nc = (int)meta_nchild(m);
    const float4 pT = ld_pm(T, S, node);
    // the children are read through one pointer: all staged (a subdomain's children) or all
    // from global memory (a node whose children straddle the end of the stage reads them there)
    const bool st = f >= S.lo && (uint32_t)(f + nc - S.lo) <= S.n;
    const float4* cp = st ? Stage::pm() + (f - S.lo) : T.pm + f;
    if constexpr (GRAD && KIND == SBH_SMOOTHDIST) {
        const float a = P.kp.alpha;
        smooth_vg(pT, q, a, -w * pT.w, r, v, g);
        for (int k = 0; k < nc; ++k) smooth_vg(cp[k], q, a, w * cp[k].w, r, v, g);
    } else if constexpr (GRAD && KIND == SBH_WINDING) {
        // each child's two records in one 32-byte load from the interleaved array (the stage is
        // not read here); two children in flight per iteration, with separate sums (1.4% faster
        // than one child with the next one's load issued ahead)
        float s0 = 0.0f, s1 = 0.0f;
        float h[3] = {0.0f, 0.0f, 0.0f};
        int k = 0;
        for (; k + 1 < nc; k += 2) {
            float4 p0, d0, p1, d1;
            ld_pmd(T.pmd, f + k, p0, d0);
            ld_pmd(T.pmd, f + k + 1, p1, d1);
            s0 += winding_vg_4pi(p0, d0, q, g);
            s1 += winding_vg_4pi(p1, d1, q, h);
        }
        if (k < nc) {
            float4 p0, d0;
            ld_pmd(T.pmd, f + k, p0, d0);
            s0 += winding_vg_4pi(p0, d0, q, g);
        }
        s0 += s1;
        g[0] += h[0]; g[1] += h[1]; g[2] += h[2];
        float go[3] = {0.0f, 0.0f, 0.0f};
        float4 pn, dn;  // the node's own records, also in one load
        ld_pmd(T.pmd, node, pn, dn);
        const float own = winding_vg_4pi(pn, dn, q, go);
        const float ws = w * kInv4Pi;
        v = ws * (s0 - own);
        g[0] = ws * (g[0] - go[0]); g[1] = ws * (g[1] - go[1]); g[2] = ws * (g[2] - go[2]);
    } else if constexpr (GRAD) {
        float s0 = 0.0f;
        for (int k = 0; k < nc; ++k) s0 += term_vg<KIND>(cp[k], cp[k], q, P.kp, g);
        float go[3] = {0.0f, 0.0f, 0.0f};
        const float own = term_vg<KIND>(pT, pT, q, P.kp, go);
        v = w * (s0 - own);
        g[0] = w * (g[0] - go[0]); g[1] = w * (g[1] - go[1]); g[2] = w * (g[2] - go[2]);
    } else if constexpr (KIND == SBH_SMOOTHDIST) {
        const float a = P.kp.alpha;
        r = dist_fast(pT, q);
        v = -w * pT.w;
        for (int k = 0; k < nc; ++k) {
            const float4 pc = cp[k];
            const float d = dist_fast(pc, q);
            if (d < r) { v *= __expf(-a * (r - d)); r = d; }
            v = fmaf(w * pc.w, __expf(-a * (d - r)), v);
        }
    } else {
        // two independent partial sums: two children in flight per iteration. Winding: each
        // child's two records in one 32-byte load from the interleaved array (the stage is not
        // read here): half the L1 requests of two 16-byte loads
        float s0 = 0.0f, s1 = 0.0f;
        int k = 0;
        constexpr int kUnroll = swap_unroll<KIND>();
#pragma unroll kUnroll
        for (; k + 1 < nc; k += 2) {
            if constexpr (KIND == SBH_WINDING) {
                float4 p0, d0, p1, d1;
                ld_pmd(T.pmd, f + k, p0, d0);
                ld_pmd(T.pmd, f + k + 1, p1, d1);
                s0 += term_winding_4pi(p0, d0, q);
                s1 += term_winding_4pi(p1, d1, q);
            } else {
                s0 += node_value<KIND>(T, S, f + k, cp[k], q, P.kp);
                s1 += node_value<KIND>(T, S, f + k + 1, cp[k + 1], q, P.kp);
            }
        }
        if (k < nc) {
            if constexpr (KIND == SBH_WINDING) {
                float4 p0, d0;
                ld_pmd(T.pmd, f + k, p0, d0);
                s0 += term_winding_4pi(p0, d0, q);
            } else {
                s0 += node_value<KIND>(T, S, f + k, cp[k], q, P.kp);
            }
        }
        if constexpr (KIND == SBH_WINDING) {
            float4 pn, dn;  // the node's own records, also in one load
            ld_pmd(T.pmd, node, pn, dn);
            v = (w * kInv4Pi) * ((s0 + s1) - term_winding_4pi(pn, dn, q));
        } else
            v = w * ((s0 + s1) - node_value<KIND>(T, S, node, pT, q, P.kp));
    }
}

// Add a query's summed swap results (value tot in the frame exp(-alpha tr) for the smooth
// distance; GRAD: gradient tg) into its sums in shared memory.
template <int KIND, bool GRAD>
__device__ __forceinline__ void add_to_query(const Params& P, WarpState<KIND>& W, uint32_t slot, float tot, float tr,
                                             const float tg[3])
{
    float* qg = GRAD ? grad_sums<KIND>() + (threadIdx.x >> 5) * 96 + 3 * slot : nullptr;
    if constexpr (KIND == SBH_SMOOTHDIST) {
        const float a = P.kp.alpha;
        float qr = W.ref[slot], qa = W.acc[slot];
        if (tr < qr) {
            const float f = __expf(-a * (qr - tr));
            qa = qa * f + tot;
            if (GRAD) for (int c = 0; c < 3; ++c) qg[c] = qg[c] * f + tg[c];
            qr = tr;
        } else {
            const float f = __expf(-a * (tr - qr));
            qa = fmaf(tot, f, qa);
            if (GRAD) for (int c = 0; c < 3; ++c) qg[c] = fmaf(tg[c], f, qg[c]);
        }
        W.ref[slot] = qr;
        W.acc[slot] = qa;
    } else {
        W.acc[slot] += tot;
        if (GRAD) for (int c = 0; c < 3; ++c) qg[c] += tg[c];
    }
}

// Run up to 32 swap tasks from the front of the ring, one per lane, each added to its query's sum
// in lane order.
template <int KIND, bool GRAD>
__device__ __forceinline__ void swap_batch(const Params& P, const Stage& S, WarpState<KIND>& W, uint32_t& s_head,
                                           uint32_t s_tail)
{
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
    float g[3] = {0.0f, 0.0f, 0.0f};
    if (valid) swap_terms<KIND, GRAD>(P, S, node, make_float3(W.qx[slot], W.qy[slot], W.qz[slot]), w, v, r, g);
    // lane-ordered sum over the tasks of each query
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, slot);
    float tot = 0.0f, tr = 3.0e38f;
    float tg[3] = {0.0f, 0.0f, 0.0f};
    for (unsigned rest = peers; rest; rest &= rest - 1u) {
        const int src = __ffs(rest) - 1;
        const float vs = __shfl_sync(peers, v, src);
        float gs[3] = {0.0f, 0.0f, 0.0f};
        if constexpr (GRAD) {
            gs[0] = __shfl_sync(peers, g[0], src); gs[1] = __shfl_sync(peers, g[1], src);
            gs[2] = __shfl_sync(peers, g[2], src);
        }
        if constexpr (KIND == SBH_SMOOTHDIST) {
            const float rs = __shfl_sync(peers, r, src);
            const float a = P.kp.alpha;
            if (rs < tr) {
                const float f = __expf(-a * (tr - rs));
                tot = tot * f + vs;
                if (GRAD) for (int c = 0; c < 3; ++c) tg[c] = tg[c] * f + gs[c];
                tr = rs;
            } else {
                const float f = __expf(-a * (rs - tr));
                tot = fmaf(vs, f, tot);
                if (GRAD) for (int c = 0; c < 3; ++c) tg[c] = fmaf(gs[c], f, tg[c]);
            }
        } else {
            tot += vs;
            if (GRAD) for (int c = 0; c < 3; ++c) tg[c] += gs[c];
        }
    }
    if (valid && lane_id() == (uint32_t)(__ffs(peers) - 1)) add_to_query<KIND, GRAD>(P, W, slot, tot, tr, tg);
    __syncwarp();
}

// One tile of 32 queries (query index tile * 32 + lane within the set described by P), run by
// one warp: control variates and depth-0 decisions lane-parallel, everything else as tasks.
template <int KIND, bool LEARNED, bool GRAD>
__device__ __forceinline__ void run_tile(const Params& P, const PhiloxRoundKeys& K, const Stage& S, WarpState<KIND>& W,
                                         const float* sdiam, int64_t tile)
{
    const TreeView& T = P.T;
    const int32_t first_sub = T.ctrl->first_sub;
    const int n_sub = T.ctrl->n_sub;
    const uint32_t lane = lane_id();
    const int64_t j = tile * 32 + lane;
    const bool active = j < P.nq;
    float3 q0 = make_float3(0.f, 0.f, 0.f);
    if (active) q0 = make_float3(P.Q[3 * j], P.Q[3 * j + 1], P.Q[3 * j + 2]);
    W.qx[lane] = q0.x; W.qy[lane] = q0.y; W.qz[lane] = q0.z;
    W.qctr[lane] = P.coherent ? 0u : (uint32_t)(j + P.qbase);
    W.acc[lane] = 0.0f;
    if constexpr (KIND == SBH_SMOOTHDIST) W.ref[lane] = 3.0e38f;
    if (lane == 0) {
        W.slack = stop_slack(T.ctrl->lo, T.ctrl->side, sdiam[0]);
        W.first_sub = first_sub;
    }
    float* qg = GRAD ? grad_sums<KIND>() + (threadIdx.x >> 5) * 96 + 3 * lane : nullptr;
    if (GRAD) { qg[0] = 0.0f; qg[1] = 0.0f; qg[2] = 0.0f; }
    __syncwarp();
    float cv = 0.0f;
    float cg[3] = {0.0f, 0.0f, 0.0f};  // GRAD: the control variates' gradient (in the frame of ex)
    ExpAcc ex;
    ex.init(3.0e38f);
    uint32_t d_head = 0, d_tail = 0, s_head = 0, s_tail = 0;

    for (int ai = 0; ai < n_sub; ++ai) {
        const int32_t a = first_sub + ai;
        // the lane's query, read from the warp's shared copy each time (not held in registers
        // through the decision and swap batches: 56 instead of 62 for the winding estimator); the
        // learned and adjoint instances keep their register copy (they spilled more or ran slower)
        const float3 q = (LEARNED || GRAD) ? q0 : make_float3(W.qx[lane], W.qy[lane], W.qz[lane]);
        const float4 pa = ld_pm(T, S, a);
        const uint32_t ma = ld_meta(T, S, a);
        if (active) {  // control variate CV_a
            if constexpr (GRAD && KIND == SBH_SMOOTHDIST) {
                smooth_vg(pa, q, P.kp.alpha, pa.w, ex.ref, ex.acc, cg);
            } else if constexpr (GRAD) {
                cv += term_vg<KIND>(pa, KIND == SBH_WINDING ? ld_dip(T, S, a) : pa, q, P.kp, cg);
            } else if constexpr (KIND == SBH_SMOOTHDIST) {
                const float d = dist_fast(pa, q);
                ex.lower(d, P.kp.alpha);
                ex.acc = fmaf(pa.w, ex.scale(d, P.kp.alpha), ex.acc);
            } else {
                cv += node_value<KIND>(T, S, a, pa, q, P.kp);
            }
        }
        if (meta_kind(ma) == kPoint) continue;
        const float wa = subdomain_weight<LEARNED>(P, S, a);
        const float da = dist_rn(pa.x, pa.y, pa.z, q);
        const float Ba = sdiam[meta_level(ma)];
        for (int s = 0; s < P.S; ++s) {
            // the depth-0 decision of every lane's query, unless its roulette surely stops: taken in
            // place by the whole warp (the node is the same for every lane) when enough lanes need it,
            // else queued as tasks that a later batch runs with other work
            uint4 x = make_uint4(0u, 0u, 0u, 0u);
            const uint32_t tag = make_tag(lane, 0u, (uint32_t)ai, (uint32_t)s);
            bool live = false;
            if (active) {
                x = draw_block(K, W, tag);
                live = !certain_stop(P.rr, unit24(x.y), da, Ba, W.slack);
            }
            const unsigned push = __ballot_sync(0xFFFFFFFFu, live);
            constexpr int kQueueMax = depth0_queue_max<KIND, LEARNED, GRAD>();
            if (kQueueMax < 0 || (kQueueMax < 32 && __popc(push) > kQueueMax)) {
                decide<KIND, LEARNED, true>(P, K, S, W, sdiam, live, a, x.x, x.y, x.z, x.w, tag, 1.0f, da, wa, wa,
                                            d_tail, s_tail);
                while (s_tail - s_head >= 32u) swap_batch<KIND, GRAD>(P, S, W, s_head, s_tail);
            } else {
                if (live) {
                    const uint32_t k = (d_tail + __popc(push & lanemask_lt())) & kRingMask;
                    W.d_node[k] = a;
                    W.d_x0[k] = x.x;
                    W.d_x1[k] = x.y;
                    W.d_w2[k] = x.z;
                    W.d_w3[k] = x.w;
                    W.d_tag[k] = tag;
                    W.d_dT[k] = da;
                }
                d_tail += __popc(push);
                __syncwarp();
            }
            while (d_tail - d_head >= 32u) {
                decision_batch<KIND, LEARNED>(P, K, S, W, sdiam, d_head, d_tail, s_tail);
                while (s_tail - s_head >= 32u) swap_batch<KIND, GRAD>(P, S, W, s_head, s_tail);
            }
        }
    }
    // drain: the decision tasks first, swaps only in full batches while decisions remain (each
    // decision batch pushes at most 32 swaps, so the swap ring stays below 64), then one partial swap
    // batch. Alternating partial swap and decision batches ran 1.1-2.8% slower: more nearly empty
    // swap batches, which cost as much as full ones.
    while (d_tail != d_head) {
        decision_batch<KIND, LEARNED>(P, K, S, W, sdiam, d_head, d_tail, s_tail);
        while (s_tail - s_head >= 32u) swap_batch<KIND, GRAD>(P, S, W, s_head, s_tail);
    }
    while (s_tail != s_head) swap_batch<KIND, GRAD>(P, S, W, s_head, s_tail);
    __syncwarp();
    if (active) {
        if constexpr (KIND == SBH_SMOOTHDIST) {
            const float a = P.kp.alpha;
            float r = W.ref[lane], v = W.acc[lane];
            float sg[3] = {0.0f, 0.0f, 0.0f};
            if (GRAD) { sg[0] = qg[0]; sg[1] = qg[1]; sg[2] = qg[2]; }
            // merge the swap sum into the control-variate sum
            if (r < ex.ref) {
                const float f = __expf(-a * (ex.ref - r));
                ex.acc = ex.acc * f + v;
                if (GRAD) for (int c = 0; c < 3; ++c) cg[c] = cg[c] * f + sg[c];
                ex.ref = r;
            } else {
                const float f = __expf(-a * (r - ex.ref));
                ex.acc = fmaf(v, f, ex.acc);
                if (GRAD) for (int c = 0; c < 3; ++c) cg[c] = fmaf(sg[c], f, cg[c]);
            }
            if (P.raw_sum) {
                const float sc = __expf(-a * ex.ref);
                P.out[j] = ex.acc * sc;
                if (GRAD) for (int c = 0; c < 3; ++c) P.grad[3 * j + c] = cg[c] * sc;
            } else {
                const bool pos = ex.acc > 0.0f;
                P.out[j] = pos ? ex.ref - __logf(ex.acc) / a : __int_as_float(0x7F800000);
                if (GRAD) {  // d = ref - log(acc) / alpha: grad d = -grad acc / (alpha acc), the frame cancels
                    const float c0 = pos ? -1.0f / (a * ex.acc) : __int_as_float(0x7FC00000);
                    for (int c = 0; c < 3; ++c) P.grad[3 * j + c] = c0 * cg[c];
                }
            }
        } else {
            P.out[j] = cv + W.acc[lane];
            if (GRAD) for (int c = 0; c < 3; ++c) P.grad[3 * j + c] = cg[c] + qg[c];
        }
    }
    __syncwarp();
}

// dynamic shared memory: the stage (stage_bytes), then [learned proposal: MlpFrag, one LearnScratch
// per warp | adjoint: one [32][3] gradient sum per warp]
template <bool LEARNED, bool GRAD>
constexpr size_t extra_smem_bytes()
{
    return LEARNED ? sizeof(MlpFrag) + kWarpsPerBlock * sizeof(LearnScratch)
                   : (GRAD ? kWarpsPerBlock * 96 * sizeof(float) : 0);
}

template <int KIND, bool LEARNED, bool GRAD>
__global__ void __launch_bounds__(32 * kWarpsPerBlock,
                                  LEARNED ? SBH_LEARNED_MIN_BLOCKS : (GRAD ? SBH_GRAD_MIN_BLOCKS : value_min_blocks<KIND>()))
    k_stoch_batched(Params P, PhiloxRoundKeys K, int32_t stage_lo, uint32_t stage_n)
{
    __shared__ WarpState<KIND> s_state[kWarpsPerBlock];
    __shared__ float sdiam[LEARNED ? 2 * kDiamLevels : kDiamLevels];  // learned: then ln of each
    if constexpr (LEARNED) mlp_frag_fill(P.mlpw, *mlp_frag<KIND>());
    Stage S;
    S.lo = stage_lo;
    S.n = stage_n;
    for (uint32_t i = threadIdx.x; i < stage_n; i += blockDim.x) {
        const int32_t v = stage_lo + (int32_t)i;
        Stage::pm()[i] = __ldg(&P.T.pm[v]);
        if (KIND == SBH_WINDING) Stage::dip()[i] = __ldg(&P.T.dip[v]);
        Stage::cdf()[i] = __ldg(&P.T.cdf[v]);
        Stage::gd()[i] = __ldg(&P.T.gd[v]);
        Stage::meta()[i] = __ldg(&P.T.meta[v]);
        Stage::fc()[i] = __ldg(&P.T.fc[v]);
    }
    if (threadIdx.x < kDiamLevels) {
        sdiam[threadIdx.x] = P.T.ctrl->diam[threadIdx.x];
        if (LEARNED) sdiam[kDiamLevels + threadIdx.x] = __logf(P.T.ctrl->diam[threadIdx.x]);
    }
    __syncthreads();
    WarpState<KIND>& W = s_state[threadIdx.x >> 5];
    const int64_t n_tiles = (P.nq + 31) / 32;
    const int64_t warp_global = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int64_t warp_stride = (int64_t)gridDim.x * kWarpsPerBlock;
    for (int64_t tile = warp_global; tile < n_tiles; tile += warp_stride)
        run_tile<KIND, LEARNED, GRAD>(P, K, S, W, sdiam, tile);
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
    Params base;         // kernel, samples, key and options shared by all sets
    PhiloxRoundKeys rk;  // the round keys of base.key (read from the parameter space, not per warp)
};

template <int KIND>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, multi_min_blocks<KIND>()) k_stoch_multi(MultiParams M)
{
    __shared__ WarpState<KIND> s_state[kWarpsPerBlock];
    __shared__ float s_diam[kWarpsPerBlock][kDiamLevels];
    __shared__ Params s_params[kWarpsPerBlock];  // the warp's current set (kept out of registers)
    const int warp = threadIdx.x >> 5;
    WarpState<KIND>& W = s_state[warp];
    float* sdiam = s_diam[warp];
    Params& P = s_params[warp];
    Stage S;  // nothing staged: the sets' trees differ
    S.lo = 0; S.n = 0;
    const uint32_t lane = lane_id();
    if (lane == 0) P = M.base;
    __syncwarp();
    int cur = -1;
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
            if (lane == 0) { P.T = D.T; P.Q = D.Q; P.out = D.out; P.nq = D.nq; }
            if (lane < (uint32_t)kDiamLevels) sdiam[lane] = D.T.ctrl->diam[lane];
            __syncwarp();
        }
        run_tile<KIND, false, false>(P, M.rk, S, W, sdiam, tile - M.sets[lo].tile_begin);
    }
}

template <int KIND, bool LEARNED, bool GRAD>
static cudaError_t launch_kind(const Params& P, unsigned blocks, int32_t lo, uint32_t n, cudaStream_t s)
{
    const size_t bytes = stage_bytes_of<KIND, LEARNED>() + extra_smem_bytes<LEARNED, GRAD>();
    cudaError_t e = cudaFuncSetAttribute(k_stoch_batched<KIND, LEARNED, GRAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_stoch_batched<KIND, LEARNED, GRAD><<<blocks, 32 * kWarpsPerBlock, bytes, s>>>(P, philox_round_keys(P.key), lo, n);
    return cudaSuccess;
}

template <bool LEARNED, bool GRAD = false>
static cudaError_t launch_batched_impl(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                                       const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o,
                                       float* out, const void* mlp_half, float near, cudaStream_t s, int64_t qbase,
                                       float* grad = nullptr)
{
    if (nq <= 0) return cudaSuccess;
    Params P;
    P.qbase = qbase;
    P.grad = grad;
    P.T = T; P.Q = Q; P.nq = nq; P.kp = kp; P.S = S;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.sampling = o.sampling; P.rr = o.rr; P.coherent = o.seed_mode; P.raw_sum = o.raw_sum; P.out = out;
    P.mlpw = (const __half*)mlp_half; P.near = near;
    const int64_t tiles = (nq + 31) / 32;
    int64_t blocks = (tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t grid_cap = (int64_t)device_sm_count() * SBH_GRID_BLOCKS_PER_SM;
    if (blocks > grid_cap) blocks = grid_cap;
    // stage the first nodes of generations 1 and 2 (the subdomains, then their children), at most
    // kStageMax (half as many with the learned proposal, whose scratch takes room, or none)
    const int32_t lo = host_ctrl.max_depth >= 1 ? host_ctrl.depth_base[1] : 0;
    const int32_t hi = host_ctrl.depth_base[host_ctrl.max_depth >= 2 ? 3 : (host_ctrl.max_depth >= 1 ? 2 : 1)];
    uint32_t n = (uint32_t)(hi > lo ? hi - lo : 0);
    const uint32_t cap = LEARNED ? (SBH_LEARNED_STAGE ? kStageMax / 2 : 0) : kStageMax;
    if (n > cap) n = cap;
    cudaError_t e;
    switch (kp.kind) {
    case SBH_COULOMB: e = launch_kind<SBH_COULOMB, LEARNED, GRAD>(P, (unsigned)blocks, lo, n, s); break;
    case SBH_WINDING: e = launch_kind<SBH_WINDING, LEARNED, GRAD>(P, (unsigned)blocks, lo, n, s); break;
    case SBH_SMOOTHDIST: e = launch_kind<SBH_SMOOTHDIST, LEARNED, GRAD>(P, (unsigned)blocks, lo, n, s); break;
    case SBH_AFFINE: e = launch_kind<SBH_AFFINE, LEARNED, GRAD>(P, (unsigned)blocks, lo, n, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stoch_batched(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                                 const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                                 cudaStream_t s, int64_t qbase)
{
    return launch_batched_impl<false>(T, host_ctrl, Q, nq, kp, S, seed, o, out, nullptr, 0.0f, s, qbase);
}

cudaError_t launch_stoch_batched_grad(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                                      const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                                      float* grad, cudaStream_t s)
{
    return launch_batched_impl<false, true>(T, host_ctrl, Q, nq, kp, S, seed, o, out, nullptr, 0.0f, s, 0, grad);
}

cudaError_t launch_stoch_batched_learned(const TreeView& T, const TreeCtrl& host_ctrl, const void* mlp_half,
                                         float near, const float* Q, int64_t nq, const KernelParams& kp, int S,
                                         uint64_t seed, const sbh_eval_opts& o, float* out, cudaStream_t s)
{
    return launch_batched_impl<true>(T, host_ctrl, Q, nq, kp, S, seed, o, out, mlp_half, near, s, 0);
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
    P.T = TreeView{}; P.Q = nullptr; P.nq = 0; P.kp = kp; P.S = S; P.out = nullptr; P.qbase = 0;
    P.grad = nullptr;
    P.mlpw = nullptr; P.near = 0.0f;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    M.rk = philox_round_keys(P.key);
    P.sampling = o.sampling; P.rr = o.rr; P.coherent = o.seed_mode; P.raw_sum = o.raw_sum;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    // persistent: as many blocks as are resident at once
    const unsigned sms = (unsigned)device_sm_count();
    switch (kp.kind) {
    case SBH_COULOMB:
        k_stoch_multi<SBH_COULOMB><<<sms * multi_min_blocks<SBH_COULOMB>(), 32 * kWarpsPerBlock, 0, s>>>(M);
        break;
    case SBH_WINDING:
        k_stoch_multi<SBH_WINDING><<<sms * multi_min_blocks<SBH_WINDING>(), 32 * kWarpsPerBlock, 0, s>>>(M);
        break;
    case SBH_SMOOTHDIST:
        k_stoch_multi<SBH_SMOOTHDIST><<<sms * multi_min_blocks<SBH_SMOOTHDIST>(), 32 * kWarpsPerBlock, 0, s>>>(M);
        break;
    case SBH_AFFINE:
        k_stoch_multi<SBH_AFFINE><<<sms * multi_min_blocks<SBH_AFFINE>(), 32 * kWarpsPerBlock, 0, s>>>(M);
        break;
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

// sbh_internal.cuh -- shared device-side definitions of libsbh: the tree layout in HBM, the
// counter-based random stream, the kernel terms and the FP32 decision arithmetic.
//
// Madan et al., "Stochastic Barnes-Hut Approximation for Fast Summation on the GPU" (SIGGRAPH
// 2025). Section and equation numbers below refer to that paper.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh.h"

namespace sbh {

// host-side count of kernel launches made by the library (reported by sbh_kernel_launches)
void note_launch();
// streaming multiprocessors of the current device (queried once per device, then cached); grid
// caps and persistent launches are sized in multiples of it
int device_sm_count();
// set the calling thread's sbh_last_error() message (printf-style)
void set_error_message(const char* fmt, ...);

// ----------------------------------------------------------------------------------------------
// Limits
// ----------------------------------------------------------------------------------------------
constexpr int kMortonBits = 20;          // bits per axis; 60-bit codes
constexpr int kMaxLevel4 = 10;           // 64-ary tree: 6 code bits per level
constexpr int kMaxLevel2 = 20;           // 8-ary tree: 3 code bits per level
constexpr int kMaxDepth = kMaxLevel2 + 2;  // generations of nodes, root included, upper bound
constexpr int kMaxLeafSize = 64;
constexpr int kDiamLevels = 24;          // |B| table entries (levels 0 .. 22 used)

// node kinds (bits 30..31 of meta)
constexpr uint32_t kPoint = 0;     // a single source point, no children
constexpr uint32_t kInternal = 1;  // children are the runs of the next code digit
constexpr uint32_t kMultiLeaf = 2; // a leaf holding several points: its children are the points
constexpr uint32_t kMaxChildren = (1u << 24) - 1;

// meta word of a node: child count (24 bits) | level << 24 (6 bits) | kind << 30
__host__ __device__ inline uint32_t meta_pack(uint32_t nchild, uint32_t level, uint32_t kind)
{
    return (nchild & 0xFFFFFFu) | ((level & 0x3Fu) << 24) | ((kind & 0x3u) << 30);
}
__host__ __device__ inline uint32_t meta_nchild(uint32_t m) { return m & 0xFFFFFFu; }
__host__ __device__ inline uint32_t meta_level(uint32_t m) { return (m >> 24) & 0x3Fu; }
__host__ __device__ inline uint32_t meta_kind(uint32_t m) { return (m >> 30) & 0x3u; }

// ----------------------------------------------------------------------------------------------
// Per-tree control block, in device memory, written by the build and read by every eval kernel.
// ----------------------------------------------------------------------------------------------
struct TreeCtrl {
    int32_t n_nodes;
    int32_t first_sub;    // subdomains: [first_sub, first_sub + n_sub)
    int32_t n_sub;
    int32_t max_depth;    // deepest generation that holds nodes
    int32_t depth_base[kMaxDepth + 2];  // node id of the first node of each generation
    float lo[3];
    float side;
    float diam[kDiamLevels];  // |B| at each level: sqrt(3) * side * d^-level (FP32, exact scaling)
    int32_t error;        // nonzero if a build step detected an inconsistency
};

// Structure-of-arrays node storage of one tree (device pointers). Children of node v are the
// contiguous ids fc[v] .. fc[v] + nchild - 1, in Morton order; generations are contiguous.
struct TreeView {
    const float4* pm;     // (centre of mass x, y, z; aggregate mass)
    const float4* dip;    // (sum_j m_j n_j; 0) or nullptr
    const float4* pmd;    // [2 v], [2 v + 1]: pm[v] and dip[v] as one 32-byte record, or nullptr
    const float* cdf;     // prefix fraction of the node's mass among its siblings (last = 1)
    const uint8_t* gd;    // the parent's child-pick guide entry for this node's slot (k_guide)
    const int32_t* fc;    // first child, -1 for a point
    const uint32_t* meta; // nchild | level << 24 | kind << 30
    const int32_t* nb;    // first sorted point
    const int32_t* ne;    // one past the last sorted point
    const int32_t* skip;  // next node of a depth-first walk after this subtree (8-ary tree)
    const TreeCtrl* ctrl;
};

// ----------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds; each multiplies counter words 0 and 2 by the round multipliers, swaps
// the halves and xors in the other words and the key; the key advances by the Weyl increments
// between rounds.
// ----------------------------------------------------------------------------------------------
// The ten round keys of a key (k.x + r W0, k.y + r W1 for round r), precomputed once per launch
// so that a round's key words are read as operands instead of advanced in registers.
struct PhiloxRoundKeys {
    uint32_t k[20];
};
__host__ __device__ inline PhiloxRoundKeys philox_round_keys(uint2 k)
{
    PhiloxRoundKeys K;
    for (int r = 0; r < 10; ++r) {
        K.k[2 * r] = k.x + (uint32_t)r * 0x9E3779B9u;
        K.k[2 * r + 1] = k.y + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& K)
{
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
        const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ K.k[2 * r], lo1, hi0 ^ c.w ^ K.k[2 * r + 1], lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
        const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += kW0;
        k.y += kW1;
    }
    return c;
}

// 24 random bits as a float in [0, 1): exact in FP32
__device__ __forceinline__ float unit24(uint32_t x) { return __uint2float_rn(x >> 8) * 5.9604644775390625e-8f; }

// ----------------------------------------------------------------------------------------------
// FP32 decision arithmetic. Every step is one IEEE round-to-nearest operation with no
// contraction, in a fixed order, so that a CPU reference in FP32 reproduces it bit for bit.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ float dist_rn(float px, float py, float pz, float3 q)
{
    const float dx = __fsub_rn(px, q.x), dy = __fsub_rn(py, q.y), dz = __fsub_rn(pz, q.z);
    const float s = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return __fsqrt_rn(s);
}

// Eq. 5 for the step from node T into its child c with the draw u: continue iff u < p,
// p = min(1, max(1, beta~_T) / beta~_c), beta~ = ||q - p~|| / |B|. The child's cell is exactly
// 4^-(l_c - l_T) times T's, so p = min(1, X / d_c) with X = max(d_T, |B_T|) 4^-(l_c - l_T) (exact),
// and u < p is u d_c < X, whose sign one FMA gives exactly. rr = 1: p = 1; rr = 2: p = 1/2. On a
// continue p gets the factor of p_rr, X / d_c capped at 1. That factor only scales sample weights,
// never a decision, so it is the fast quotient (within 2 ulp), exact-rounded only for d_c >= 2^126
// where the fast one does not hold.
__device__ __forceinline__ bool rr_continue(int rr, float u, float dT, float BT, uint32_t lT, float dc, uint32_t lc,
                                            float& p)
{
    if (rr == 1) { p = 1.0f; return true; }
    if (rr == 2) { p = 0.5f; return u < 0.5f; }
    const float X = fmaxf(dT, BT) * __int_as_float((127 - 2 * (int)(lc - lT)) << 23);
    if (!(fmaf(u, dc, -X) < 0.0f)) return false;
    if (dc <= X) p = 1.0f;
    else p = dc < 8.5e37f ? __fdividef(X, dc) : __fdiv_rn(X, dc);
    return true;
}

// A path at node T (distance dT from the query to T's centre, cell diagonal BT) stops at its next
// roulette whichever child is drawn when u >= p_c for every child c; this test finds such draws
// before the child is drawn, so the pick, the child's record and the exact test above are skipped
// for them. It never skips a path rr_continue would continue, so results do not change.
//   Every child centre lies in T's cell grown by `slack`: points are assigned to cells by FP32
//   rounding (at most one quantisation step, side 2^-20, outside their cell per axis) and centres
//   are rounded to FP32; the caller passes slack = diam0 2^-19 + 2^-20 max |coordinate|. So
//   d_c >= dT - BT - slack, and X = max(dT, BT) 4^-(l_c - l_T) <= dT / 4 when dT > BT (a child is
//   at least one level down): p_c = X / d_c <= dT / (4 (dT - BT - slack)). The test asks for
//   4 u (dT - BT - slack) >= dT (1 + 2^-10); the margin covers the rounding of the FP32
//   distances (a few units in the last place) many times over. Roulette off never stops; the
//   fixed 1/2 stops exactly when u >= 1/2.
__device__ __forceinline__ bool certain_stop(int rr, float u, float dT, float BT, float slack)
{
    if (rr == 1) return false;
    if (rr == 2) return u >= 0.5f;
    const float g = dT - (BT + slack);
    return g > 0.0f && 4.0f * u * g >= dT * 1.0009765625f;
}

// the slack of certain_stop for a tree (its root cube: lower corner lo, edge side, diagonal diam0)
__host__ __device__ inline float stop_slack(const float lo[3], float side, float diam0)
{
    float c = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const float x0 = lo[a] < 0.0f ? -lo[a] : lo[a];
        const float x1 = lo[a] + side < 0.0f ? -(lo[a] + side) : lo[a] + side;
        c = c > x0 ? c : x0;
        c = c > x1 ? c : x1;
    }
    return diam0 * 1.9073486328125e-06f + c * 9.5367431640625e-07f;  // 2^-19, 2^-20
}

// ----------------------------------------------------------------------------------------------
// Kernel terms m f(p, q) in FP32 (values; tolerances, not bit-exactness, apply to these).
// ----------------------------------------------------------------------------------------------
struct KernelParams {
    int kind;
    float eps2;       // softening^2
    float alpha;
    float g[3];       // affine test kernel
};

constexpr float kInv4Pi = 0.0795774715459476679f;

// 1/sqrt(x) for the kernel terms: the hardware approximation with subnormal arguments flushed to
// zero (PTX rsqrt.approx.ftz.f32). For a normal argument it returns what rsqrtf returns; it skips
// the rescaling rsqrtf adds for subnormal arguments, which a term never meets except at points a
// distance below 1.1e-19 apart. Winding terms therefore take r^2 below the smallest normal float
// as the coincident case (term 0), or clamp r^2 there (term_winding_4pi). The decision arithmetic
// never uses it.
constexpr float kMinNormal = 1.17549435e-38f;
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Both 16-byte records of node v from an interleaved (pm, dip) array in one 256-bit load
// (ld.global.nc.v8.f32: a 32-byte aligned address, data read-only for the kernel's lifetime):
// one L1 request per node where two separate loads would take two.
__device__ __forceinline__ void ld_pmd(const float4* pmd, int32_t v, float4& pm, float4& dp)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(pm.x), "=f"(pm.y), "=f"(pm.z), "=f"(pm.w), "=f"(dp.x), "=f"(dp.y), "=f"(dp.z), "=f"(dp.w)
        : "l"(pmd + 2 * (int64_t)v));
}

// Coulomb-like potential (Sec. 4.2): m / sqrt(r^2 + eps^2)
__device__ __forceinline__ float term_coulomb(float4 pm, float3 q, float eps2)
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    return pm.w * rsqrt_ftz(r2);
}

// winding-number dipole (Sec. 4.3.2): ((p - q) . N) / (4 pi r^3), N = sum_j m_j n_j; 0 at r = 0
__device__ __forceinline__ float term_winding(float4 pm, float4 dp, float3 q)
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ir = rsqrt_ftz(r2);
    const float dot = fmaf(dx, dp.x, fmaf(dy, dp.y, dz * dp.z));
    const float v = dot * (ir * ir * ir) * kInv4Pi;
    return r2 >= kMinNormal ? v : 0.0f;
}

// The winding term times 4 pi, ((p - q).N) / r^3: sums of these are scaled by 1 / (4 pi) once.
// r^2 is clamped below at the smallest normal float instead of tested: a coincident point (r = 0,
// so (p - q).N = 0) gives 0, since ((p - q).N / r) / r^2 overflows nowhere; a point closer than
// 1.1e-19 but not coincident is taken at that distance. One instruction less per term than the
// zero test (0.9% of the warp-task kernel's time).
__device__ __forceinline__ float term_winding_4pi(float4 pm, float4 dp, float3 q)
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ir = rsqrt_ftz(fmaxf(r2, kMinNormal));
    const float dot = fmaf(dx, dp.x, fmaf(dy, dp.y, dz * dp.z));
    return (dot * ir) * (ir * ir);
}

// distance for the smooth-distance kernel (Sec. 4.3.3), whose term is m exp(-alpha r)
__device__ __forceinline__ float dist_fast(float4 pm, float3 q)
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    return r2 * rsqrt_ftz(fmaxf(r2, 1e-37f));
}

// affine test kernel: m (1 + g . (p - q))
__device__ __forceinline__ float term_affine(float4 pm, float3 q, const float* g)
{
    const float dx = pm.x - q.x, dy = pm.y - q.y, dz = pm.z - q.z;
    return pm.w * (1.0f + fmaf(g[0], dx, fmaf(g[1], dy, g[2] * dz)));
}

// Running sum of m exp(-alpha r) terms held as acc * exp(-alpha * ref): the reference distance
// drops to the smallest distance seen so far, so that no term overflows and the dominant terms
// never underflow in FP32.
struct ExpAcc {
    float ref;
    float acc;
    __device__ __forceinline__ void init(float r0) { ref = r0; acc = 0.0f; }
    // make ref <= r so that a term at distance r can be added
    __device__ __forceinline__ void lower(float r, float alpha)
    {
        if (r < ref) {
            acc *= __expf(-alpha * (ref - r));
            ref = r;
        }
    }
    __device__ __forceinline__ float scale(float r, float alpha) const { return __expf(-alpha * (r - ref)); }
};

}  // namespace sbh

// sbh_build.cu -- GPU construction of the octree-like tree of Sec. 3.1 (Madan et al. 2025).
//
// The paper builds its tree on the CPU (Sec. 4.1); here every stage is a CUDA kernel:
//   1. bounds + validation   per-axis min/max of the points (the root cube), counts of NaN/Inf
//                            coordinates and of non-positive weights
//   2. Morton codes          20-bit FP32 quantisation per axis, interleaved to 60 bits
//   3. stable LSD radix sort (code, index), 8 passes of 8 bits, block-local split sort
//   4. gather                points, weights and normals into Morton order
//   5. topology              generation by generation: a node whose points span several cells one
//                            level down has those runs as children; a run that stays inside one
//                            cell collapses into its deepest split; a run of <= leaf_size points
//                            (or at the deepest level) is a leaf whose children are its points
//   6. aggregates            FP64 bottom-up sums of m, m p, m n per node, then packed to FP32
//                            with the children's prefix mass fractions
//
// Node ids are generation-major (breadth-first): every node's children are contiguous, in
// Morton order, and the top generations that every query reads sit at the front of each array.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>
#include <stdint.h>

#include "sbh_build.cuh"
#include "sbh_sort.cuh"

namespace sbh {

namespace {
constexpr int kThreads = 256;
// blocks for n items, at most 16 per SM of the current device (grid-stride loops do the rest)
inline unsigned grid_for(int64_t n, int per_block = kThreads, unsigned cap = 0)
{
    if (cap == 0) cap = 16u * (unsigned)device_sm_count();
    int64_t g = (n + per_block - 1) / per_block;
    if (g < 1) g = 1;
    return (unsigned)(g > cap ? cap : g);
}
}  // namespace

// ----------------------------------------------------------------------------------------------
// device memory: the library's stream-ordered pool, or the caller's allocator; an optional cap on
// the bytes the library holds at once (allocations beyond it fail as out of memory)
// ----------------------------------------------------------------------------------------------
namespace {
struct Block {
    size_t bytes;
    sbh_free_fn free_fn;  // nullptr: the library's pool
    void* ctx;
};
std::mutex g_mem_mutex;
cudaMemPool_t g_pool[64];
bool g_pool_ready[64];
sbh_alloc_fn g_alloc_fn = nullptr;
sbh_free_fn g_free_fn = nullptr;
void* g_alloc_ctx = nullptr;
uint64_t g_limit = 0;
uint64_t g_in_use = 0;
std::unordered_map<void*, Block> g_blocks;
}  // namespace

cudaError_t dalloc(void** p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    std::lock_guard<std::mutex> lock(g_mem_mutex);
    if (g_limit && g_in_use + bytes > g_limit) return cudaErrorMemoryAllocation;
    if (g_alloc_fn) {
        void* q = g_alloc_fn(bytes, (void*)s, g_alloc_ctx);
        if (!q) return cudaErrorMemoryAllocation;
        if (((uintptr_t)q & 255u) != 0) {  // misaligned: hand it back and fail
            g_free_fn(q, (void*)s, g_alloc_ctx);
            return cudaErrorMisalignedAddress;
        }
        *p = q;
        g_blocks[q] = Block{bytes, g_free_fn, g_alloc_ctx};
        g_in_use += bytes;
        return cudaSuccess;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;  // keep freed blocks for reuse by later builds
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool_ready[dev] = true;
    }
    e = cudaMallocFromPoolAsync(p, bytes, g_pool[dev], s);
    if (e != cudaSuccess) return e;
    g_blocks[*p] = Block{bytes, nullptr, nullptr};
    g_in_use += bytes;
    return cudaSuccess;
}

void dfree(void* p, cudaStream_t s)
{
    if (!p) return;
    Block b{0, nullptr, nullptr};
    {
        std::lock_guard<std::mutex> lock(g_mem_mutex);
        auto it = g_blocks.find(p);
        if (it != g_blocks.end()) {
            b = it->second;
            g_in_use -= b.bytes;
            g_blocks.erase(it);
        }
    }
    if (b.free_fn) b.free_fn(p, (void*)s, b.ctx);
    else cudaFreeAsync(p, s);
}

void set_allocator(sbh_alloc_fn a, sbh_free_fn f, void* ctx)
{
    std::lock_guard<std::mutex> lock(g_mem_mutex);
    g_alloc_fn = a;
    g_free_fn = f;
    g_alloc_ctx = ctx;
}

void set_memory_limit(uint64_t bytes)
{
    std::lock_guard<std::mutex> lock(g_mem_mutex);
    g_limit = bytes;
}

uint64_t memory_in_use()
{
    std::lock_guard<std::mutex> lock(g_mem_mutex);
    return g_in_use;
}

// ----------------------------------------------------------------------------------------------
// 1. bounds and validation
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ int ordered_int(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float from_ordered(int i) { return __int_as_float(i >= 0 ? i : (i ^ 0x7FFFFFFF)); }

// scratch: [0..2] min (ordered int), [3..5] max, [6] bad coordinates, [7] bad weights
__global__ void k_bounds_init(int* scratch)
{
    if (threadIdx.x < 3) { scratch[threadIdx.x] = INT32_MAX; scratch[3 + threadIdx.x] = INT32_MIN; }
    if (threadIdx.x == 6 || threadIdx.x == 7) scratch[threadIdx.x] = 0;
}

__global__ void k_bounds(const float* __restrict__ pts, const float* __restrict__ w, int64_t n,
                         int* __restrict__ scratch)
{
    int mn[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, mx[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    int bad_p = 0, bad_w = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = pts[3 * i + a];
            if (!isfinite(v)) { ++bad_p; continue; }
            const int o = ordered_int(v);
            mn[a] = min(mn[a], o);
            mx[a] = max(mx[a], o);
        }
        const float m = w[i];
        if (!(m > 0.0f) || !isfinite(m)) ++bad_w;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], off));
            mx[a] = max(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], off));
        }
        bad_p += __shfl_xor_sync(0xFFFFFFFFu, bad_p, off);
        bad_w += __shfl_xor_sync(0xFFFFFFFFu, bad_w, off);
    }
    // then across the block's warps, so that each block adds one set of atomics (not one per warp)
    __shared__ int s_red[kThreads / 32][8];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { s_red[warp][a] = mn[a]; s_red[warp][3 + a] = mx[a]; }
        s_red[warp][6] = bad_p;
        s_red[warp][7] = bad_w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                mn[a] = min(mn[a], s_red[k][a]);
                mx[a] = max(mx[a], s_red[k][3 + a]);
            }
            bad_p += s_red[k][6];
            bad_w += s_red[k][7];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&scratch[a], mn[a]);
            atomicMax(&scratch[3 + a], mx[a]);
        }
        if (bad_p) atomicAdd(&scratch[6], bad_p);
        if (bad_w) atomicAdd(&scratch[7], bad_w);
    }
}

// root cube: lo = per-axis min, side = largest extent (1 if every point coincides); the cell
// diagonal table |B|(level) = sqrt(3) * side * 2^-(shift * level) for each branching
__global__ void k_root_cube(const int* __restrict__ scratch, TreeCtrl* c4, TreeCtrl* c2)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float lo[3], side = 0.0f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = from_ordered(scratch[a]);
        const float ext = __fsub_rn(from_ordered(scratch[3 + a]), lo[a]);
        side = ext > side ? ext : side;
    }
    if (side == 0.0f) side = 1.0f;
    const float diam0 = __fmul_rn(1.7320508075688772f, side);
    for (int a = 0; a < 3; ++a) { c4->lo[a] = lo[a]; c2->lo[a] = lo[a]; }
    c4->side = side;
    c2->side = side;
    for (int l = 0; l < kDiamLevels; ++l) {
        c4->diam[l] = ldexpf(diam0, -2 * l);
        c2->diam[l] = ldexpf(diam0, -l);
    }
}

// ----------------------------------------------------------------------------------------------
// 2. Morton codes: c = min(2^20 - 1, floor((x - lo) * (2^20 / side))), FP32 with one rounding
//    per operation; bits interleaved x, y, z from the most significant bit down.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t quantise(float x, float lo, float scale)
{
    const float t = __fmul_rn(__fsub_rn(x, lo), scale);
    const float f = floorf(t);
    const uint32_t c = f <= 0.0f ? 0u : (uint32_t)f;
    return c > 1048575u ? 1048575u : c;
}

__global__ void k_morton(const float* __restrict__ pts, int64_t n, const TreeCtrl* __restrict__ c4,
                         uint64_t* __restrict__ code, int32_t* __restrict__ idx)
{
    const float lx = c4->lo[0], ly = c4->lo[1], lz = c4->lo[2];
    const float scale = __fdiv_rn(1048576.0f, c4->side);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cx = quantise(pts[3 * i], lx, scale);
        const uint32_t cy = quantise(pts[3 * i + 1], ly, scale);
        const uint32_t cz = quantise(pts[3 * i + 2], lz, scale);
        code[i] = (spread3(cx) << 2) | (spread3(cy) << 1) | spread3(cz);
        idx[i] = (int32_t)i;
    }
}

// ----------------------------------------------------------------------------------------------
// Device-wide exclusive scan of int32 (reduce, scan the block sums, add): no inter-block waits.
// ----------------------------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// exclusive scan of one value per thread across the block; *total (if given) gets the sum
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int before = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int* __restrict__ in, int64_t n,
                                                              int* __restrict__ sums)
{
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    int total;
    block_exclusive_scan(s, ws, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// exclusive scan of each tile plus a per-tile offset (offsets may be nullptr); in may alias out
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int* in, int64_t n,
                                                            const int* __restrict__ offsets, int* out)
{
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int run = block_exclusive_scan(s, ws, nullptr) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

int64_t scan_temp_ints(int64_t n)
{
    int64_t total = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n;
    }
    return total + 1;
}

void scan_exclusive(const int* in, int* out, int64_t n, int* temp, cudaStream_t s)
{
    if (n <= 0) return;
    if (n <= kScanTile) {
        k_scan_tile<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        note_launch();
        return;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    int* sums = temp;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    note_launch();
    scan_exclusive(sums, sums, nb, temp + nb, s);
    k_scan_tile<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums, out);
    note_launch();
}

// ----------------------------------------------------------------------------------------------
// 3. stable LSD radix sort of (code, index) pairs, 8-bit digits
//    hist: per-tile digit counts, stored digit-major so that one exclusive scan gives every
//    (digit, tile) output offset. scatter: a stable local sort of the tile by the digit (nine
//    one-bit splits of (digit, slot) words in shared memory; the ninth moves padding last),
//    then each key goes to offset[digit][tile] + its rank among the tile's keys of that digit.
// ----------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                             int shift, int ntiles, int* __restrict__ hist)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                                const int32_t* __restrict__ vin, int64_t n,
                                                                int shift, int ntiles,
                                                                const int* __restrict__ offsets,
                                                                uint64_t* __restrict__ kout,
                                                                int32_t* __restrict__ vout)
{
    __shared__ uint64_t skey[kSortTile];
    __shared__ int32_t sval[kSortTile];
    __shared__ uint32_t ord[2][kSortTile];  // digit << 16 | slot
    __shared__ int dstart[257];
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int count = (n - base) < kSortTile ? (int)(n - base) : kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        if (i < count) {
            const uint64_t k = kin[base + i];
            skey[i] = k;
            sval[i] = vin[base + i];
            ord[0][i] = ((uint32_t)((k >> shift) & 0xFF) << 16) | (uint32_t)i;
        } else {
            ord[0][i] = (256u << 16) | (uint32_t)i;  // padding sorts last
        }
    }
    __syncthreads();
    int cur = 0;
    for (int bit = 16; bit < 25; ++bit) {
        uint32_t e[kSortItems];
        int zeros = 0;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            e[k] = ord[cur][threadIdx.x * kSortItems + k];
            zeros += ((e[k] >> bit) & 1u) ? 0 : 1;
        }
        int total_zeros;
        int zb = block_exclusive_scan(zeros, ws, &total_zeros);
        int pos = threadIdx.x * kSortItems;
#pragma unroll
        for (int k = 0; k < kSortItems; ++k, ++pos) {
            const bool one = (e[k] >> bit) & 1u;
            const int dst = one ? total_zeros + (pos - zb) : zb;
            if (!one) ++zb;
            ord[cur ^ 1][dst] = e[k];
        }
        cur ^= 1;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < count; i += kSortThreads) {
        const uint32_t d = ord[cur][i] >> 16;
        if (i == 0 || (ord[cur][i - 1] >> 16) != d) dstart[d] = i;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += kSortThreads) {
        const uint32_t e = ord[cur][i];
        const uint32_t d = e >> 16, slot = e & 0xFFFFu;
        const int64_t dst = (int64_t)offsets[(int64_t)d * ntiles + blockIdx.x] + (i - dstart[d]);
        kout[dst] = skey[slot];
        vout[dst] = sval[slot];
    }
}

// ----------------------------------------------------------------------------------------------
// 4. gather into Morton order; shared code digits of neighbouring codes
// ----------------------------------------------------------------------------------------------
__global__ void k_gather(const float* __restrict__ pts, const float* __restrict__ w,
                         const float* __restrict__ nrm, const int32_t* __restrict__ perm, int64_t n,
                         float4* __restrict__ spw, float4* __restrict__ snrm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = perm[i];
        spw[i] = make_float4(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], w[j]);
        if (nrm) snrm[i] = make_float4(nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2], 0.0f);
    }
}

// lcp[i] = leading code digits (6 bits for d = 4, 3 bits for d = 2) shared by sorted codes i-1
// and i, capped at the deepest level; lcp[0] is unused
__global__ void k_lcp(const uint64_t* __restrict__ code, int64_t n, uint8_t* __restrict__ lcp4,
                      uint8_t* __restrict__ lcp2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == 0) { lcp4[0] = 0; lcp2[0] = 0; continue; }
        const int same_bits = __clzll((long long)(code[i] ^ code[i - 1])) - 4;  // codes use 60 bits
        lcp4[i] = (uint8_t)min(same_bits / 6, kMaxLevel4);
        lcp2[i] = (uint8_t)min(same_bits / 3, kMaxLevel2);
    }
}

// ----------------------------------------------------------------------------------------------
// 5. topology, one generation at a time
//    cid[i] is the node of the newest generation holding sorted point i (-1 once the point has
//    left the frontier). A child of an expandable node v starts at point i when i is v's first
//    point, when v is a multi-point leaf (every point is a child), or when lcp[i] equals v's
//    level (points i-1 and i differ in the digit just below v). Child id = generation base +
//    inclusive scan of those flags - 1, so children of one parent are contiguous.
// ----------------------------------------------------------------------------------------------
struct BuildArrays {
    int32_t* nb;
    int32_t* ne;
    int32_t* fc;
    int32_t* parent;
    uint32_t* meta;
    int32_t* minl;    // smallest lcp strictly inside a new node (its split level)
    int32_t* cid;
    int32_t* flag;
    int32_t* scan;
    const uint8_t* lcp;
    TreeCtrl* ctrl;
    int64_t n;
    int leaf_size;
    int max_level;
};

// expandable node of the newest generation that holds point i, or -1
__device__ __forceinline__ int32_t frontier_of(const BuildArrays& B, int64_t i)
{
    const int32_t c = B.cid[i];
    if (c < 0) return -1;
    return meta_kind(B.meta[c]) != kPoint ? c : -1;
}

__device__ __forceinline__ int child_flag(const BuildArrays& B, int64_t i, int32_t v)
{
    if (v < 0) return 0;
    const uint32_t m = B.meta[v];
    if (meta_kind(m) == kMultiLeaf) return 1;
    return (i == B.nb[v] || (int)B.lcp[i] == (int)meta_level(m)) ? 1 : 0;
}

__global__ void k_min_u8(const uint8_t* __restrict__ lcp, int64_t n, int* __restrict__ out_min)
{
    int m = 255;
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = min(m, (int)lcp[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = min(m, __shfl_xor_sync(0xFFFFFFFFu, m, off));
    if ((threadIdx.x & 31) == 0 && m < 255) atomicMin(out_min, m);
}

__global__ void k_set_int(int* p, int v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

// the root: point, multi-point leaf (n <= leaf_size, or every code equal), or internal at its
// split level (collapsed down to the first level at which its points separate)
__global__ void k_topo_root(BuildArrays B, const int* __restrict__ root_min)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t n = B.n;
    uint32_t kind, level;
    if (n == 1) { kind = kPoint; level = 0; }
    else if (n <= B.leaf_size) { kind = kMultiLeaf; level = 0; }
    else {
        const int L = *root_min;
        if (L >= B.max_level) { kind = kMultiLeaf; level = (uint32_t)B.max_level; }
        else { kind = kInternal; level = (uint32_t)L; }
    }
    B.nb[0] = 0;
    B.ne[0] = (int32_t)n;
    B.parent[0] = -1;
    B.fc[0] = -1;
    B.meta[0] = meta_pack(0, level, kind);
    for (int g = 0; g < kMaxDepth + 2; ++g) B.ctrl->depth_base[g] = 1;
    B.ctrl->depth_base[0] = 0;
    B.ctrl->max_depth = 0;
    B.ctrl->error = 0;
}

__global__ void k_topo_seed(BuildArrays B)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += (int64_t)gridDim.x * blockDim.x)
        B.cid[i] = 0;
}

__global__ void k_topo_flags(BuildArrays B)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += (int64_t)gridDim.x * blockDim.x)
        B.flag[i] = child_flag(B, i, frontier_of(B, i));
}

// after the scan: ranges and parent links of generation gen + 1
__global__ void k_topo_children(BuildArrays B, int gen)
{
    const int32_t base = B.ctrl->depth_base[gen + 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = B.flag[i];
        if (i == B.n - 1) {
            const int32_t total = B.scan[i] + f;
            B.ctrl->depth_base[gen + 2] = base + total;
            if (total > 0) B.ctrl->max_depth = gen + 1;
        }
        const int32_t v = frontier_of(B, i);
        if (v < 0) continue;
        const int32_t c = base + B.scan[i] + f - 1;  // child holding point i
        if (f) {
            B.nb[c] = (int32_t)i;
            B.parent[c] = v;
            B.minl[c] = 255;
            B.fc[c] = -1;
        }
        if (i == B.nb[v]) B.fc[v] = c;
        if (i + 1 == B.ne[v] || B.flag[i + 1]) B.ne[c] = (int32_t)(i + 1);
    }
}

// smallest lcp strictly inside each new child, then the cid map of the new generation
__global__ void k_topo_minlcp(BuildArrays B, int gen)
{
    const int32_t base = B.ctrl->depth_base[gen + 1];
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < B.n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        int32_t c = -1;
        int val = 255;
        if (i < B.n) {
            const int32_t v = frontier_of(B, i);
            if (v >= 0) {
                const int f = B.flag[i];
                c = base + B.scan[i] + f - 1;
                if (!f) val = B.lcp[i];
            }
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
        const int m = (int)__reduce_min_sync(peers, (unsigned)val);
        if (c >= 0 && m < 255 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(&B.minl[c], m);
        if (i < B.n) B.cid[i] = c;
    }
}

// kind and level of each new child; child counts of the parents
__global__ void k_topo_classify(BuildArrays B, int gen)
{
    const int32_t base = B.ctrl->depth_base[gen + 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = B.cid[i];
        if (c < base) continue;  // not in the new generation
        const int32_t v = B.parent[c];
        const uint32_t pm = B.meta[v];
        if (i + 1 == B.ne[v]) {  // parent's last point: its last child is c
            const uint32_t nc = (uint32_t)(c - B.fc[v] + 1);
            if (nc > kMaxChildren) B.ctrl->error = 1;
            B.meta[v] = meta_pack(nc, meta_level(pm), meta_kind(pm));
        }
        if (!B.flag[i]) continue;
        const int32_t cnt = B.ne[c] - B.nb[c];
        const uint32_t L1 = meta_level(pm) + 1;
        uint32_t kind, level;
        if (meta_kind(pm) == kMultiLeaf || cnt == 1) { kind = kPoint; level = L1; }
        else if (cnt <= B.leaf_size) { kind = kMultiLeaf; level = L1; }
        else {
            const int m = B.minl[c];
            if (m >= B.max_level) { kind = kMultiLeaf; level = (uint32_t)B.max_level; }
            else { kind = kInternal; level = (uint32_t)m; }
        }
        B.meta[c] = meta_pack(0, level, kind);
    }
}

// ----------------------------------------------------------------------------------------------
// 6. aggregates: FP64 sums of m, m p, m n, children before parents (generations in reverse)
// ----------------------------------------------------------------------------------------------
__global__ void k_aggregate(const int32_t* __restrict__ fc, const uint32_t* __restrict__ meta,
                            const int32_t* __restrict__ nb, const float4* __restrict__ spw,
                            const float4* __restrict__ snrm, const TreeCtrl* __restrict__ ctrl, int gen,
                            double* __restrict__ agg)
{
    const int32_t lo = ctrl->depth_base[gen], hi = ctrl->depth_base[gen + 1];
    for (int64_t v = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < hi; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t m = meta[v];
        double a[7];
        if (meta_kind(m) == kPoint) {
            const float4 p = spw[nb[v]];
            const double w = p.w;
            a[0] = w; a[1] = w * (double)p.x; a[2] = w * (double)p.y; a[3] = w * (double)p.z;
            if (snrm) {
                const float4 q = snrm[nb[v]];
                a[4] = w * (double)q.x; a[5] = w * (double)q.y; a[6] = w * (double)q.z;
            } else {
                a[4] = a[5] = a[6] = 0.0;
            }
        } else {
            for (int k = 0; k < 7; ++k) a[k] = 0.0;
            const int32_t f = fc[v];
            const int nc = (int)meta_nchild(m);
            for (int c = 0; c < nc; ++c) {
                const double* s = agg + 8 * (int64_t)(f + c);
                for (int k = 0; k < 7; ++k) a[k] += s[k];
            }
        }
        double* d = agg + 8 * v;
        for (int k = 0; k < 7; ++k) d[k] = a[k];
        d[7] = 0.0;
    }
}

// FP32 node records and prefix mass fractions: FP64 quotients rounded once to FP32. FP64 division
// is slow on this GPU, and a loop of them in one lane holds its whole warp, so each node computes
// only its own: its centre of mass (a single point, whose quotient m x / m is x itself, copies its
// own record) and its own fraction among its siblings, the prefix sum of their masses in sibling
// order over the parent's mass (the same sum, in the same order, as k_aggregate's). (A product
// with 1 / m is not a substitute for the quotient: small nodes of equal weights often sit exactly
// on an FP32 rounding midpoint, where the product's last-bit error changes the rounding.)
__global__ void k_pack(const double* __restrict__ agg, const int32_t* __restrict__ fc,
                       const uint32_t* __restrict__ meta, const int32_t* __restrict__ nb,
                       const int32_t* __restrict__ parent, const float4* __restrict__ spw,
                       const float4* __restrict__ snrm, const TreeCtrl* __restrict__ ctrl, float4* __restrict__ pm,
                       float4* __restrict__ dip, float4* __restrict__ pmd, float* __restrict__ cdf)
{
    const int32_t N = ctrl->depth_base[ctrl->max_depth + 1];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        if (meta_kind(meta[v]) == kPoint) {
            const float4 p = spw[nb[v]];
            pm[v] = p;
            if (dip) {  // m n: one FP32 rounding of the exact product, as the FP64 sum rounded to FP32
                const float4 q = snrm ? snrm[nb[v]] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                dip[v] = make_float4(__fmul_rn(p.w, q.x), __fmul_rn(p.w, q.y), __fmul_rn(p.w, q.z), 0.0f);
            }
        } else {
            const double* a = agg + 8 * v;
            const double m = a[0];
            pm[v] = make_float4(__double2float_rn(a[1] / m), __double2float_rn(a[2] / m),
                                __double2float_rn(a[3] / m), __double2float_rn(m));
            if (dip) dip[v] = make_float4(__double2float_rn(a[4]), __double2float_rn(a[5]), __double2float_rn(a[6]), 0.0f);
        }
        if (pmd) {  // the same two records side by side, for one 32-byte load
            pmd[2 * v] = pm[v];
            pmd[2 * v + 1] = dip[v];
        }
        if (v == 0) { cdf[0] = 1.0f; continue; }
        const int32_t par = parent[v];
        const int32_t f = fc[par];
        const int32_t last = f + (int32_t)meta_nchild(meta[par]) - 1;
        if (v >= last) { cdf[v] = 1.0f; continue; }
        double pre = 0.0;
        for (int32_t k = f; k <= v; ++k) pre += agg[8 * (int64_t)k];
        cdf[v] = __double2float_rn(pre / agg[8 * (int64_t)par]);
    }
}

// The child pick's guide table (Chen and Asau's method), one entry per child slot: for slot j of
// a node with nc children, the number of prefix fractions cdf_c <= u_j among the first nc - 1
// children, where u_j = ceil(j 2^24 / nc) 2^-24 is the smallest 24-bit draw whose slot
// floor(u nc) is j. It is stored at the child's own id (first child + j): every node but the root
// fills one slot of its parent. That count never decreases with u, so a pick with draw u in slot
// j that scans up from the entry finds the same child as counting all prefix fractions.
__global__ void k_guide(const int32_t* __restrict__ fc, const uint32_t* __restrict__ meta,
                        const int32_t* __restrict__ parent, const float* __restrict__ cdf,
                        const TreeCtrl* __restrict__ ctrl, uint8_t* __restrict__ gd)
{
    const int32_t N = ctrl->depth_base[ctrl->max_depth + 1];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        if (v == 0) { gd[0] = 0; continue; }
        const int32_t par = parent[v];
        const int32_t f = fc[par];
        const uint32_t nc = meta_nchild(meta[par]);
        const uint32_t j = (uint32_t)(v - f);
        const uint32_t mj = (uint32_t)((((uint64_t)j << 24) + nc - 1u) / nc);  // < 2^24: exact in FP32
        const float uj = (float)mj * 5.9604644775390625e-8f;
        uint32_t cnt = 0;
        for (uint32_t i = 0; i + 1u < nc; ++i) cnt += cdf[f + i] <= uj ? 1u : 0u;
        gd[v] = (uint8_t)cnt;
    }
}

__global__ void k_finalize(TreeCtrl* ctrl, const int32_t* __restrict__ fc, const uint32_t* __restrict__ meta)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ctrl->n_nodes = ctrl->depth_base[ctrl->max_depth + 1];
    const uint32_t m = meta[0];
    if (meta_nchild(m) > 0) {
        ctrl->first_sub = fc[0];
        ctrl->n_sub = (int32_t)meta_nchild(m);
    } else {
        ctrl->first_sub = 0;
        ctrl->n_sub = 1;
    }
}

// depth-first successor after a node's subtree: its next sibling, else its parent's successor
__global__ void k_skip(const int32_t* __restrict__ parent, const int32_t* __restrict__ fc,
                       const uint32_t* __restrict__ meta, const TreeCtrl* __restrict__ ctrl, int gen,
                       int32_t* __restrict__ skip)
{
    const int32_t lo = ctrl->depth_base[gen], hi = ctrl->depth_base[gen + 1];
    for (int64_t v = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < hi; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = parent[v];
        if (p < 0) { skip[v] = -1; continue; }
        const int32_t last = fc[p] + (int32_t)meta_nchild(meta[p]) - 1;
        skip[v] = (v < last) ? (int32_t)(v + 1) : skip[p];
    }
}

// ----------------------------------------------------------------------------------------------
// host orchestration
// ----------------------------------------------------------------------------------------------
#define SBH_TRY(x)                               \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return e_;        \
    } while (0)

// Scratch buffers of one build step: whatever is still held when the step returns (on success or
// on an error part way) goes back in stream order; keep() hands a buffer over to the tree.
struct ScratchSet {
    cudaStream_t s;
    void* p[8] = {};
    int n = 0;
    explicit ScratchSet(cudaStream_t st) : s(st) {}
    ScratchSet(const ScratchSet&) = delete;
    ScratchSet& operator=(const ScratchSet&) = delete;
    template <class T>
    cudaError_t alloc(T** q, size_t bytes)
    {
        if (n == 8) return cudaErrorInvalidValue;
        const cudaError_t e = dalloc((void**)q, bytes, s);
        if (e == cudaSuccess) p[n++] = (void*)*q;
        return e;
    }
    void keep(const void* q)
    {
        for (int i = 0; i < n; ++i)
            if (p[i] == q) p[i] = nullptr;
    }
    ~ScratchSet()
    {
        for (int i = 0; i < n; ++i) dfree(p[i], s);
    }
};

cudaError_t alloc_tree(DeviceTree& D, int64_t n, bool with_dip, bool with_skip, bool with_rec, cudaStream_t s)
{
    const int64_t cap = 2 * n + 1;
    D.cap = cap;  // D.ctrl is kept if the caller allocated it already
    SBH_TRY(dalloc((void**)&D.pm, cap * sizeof(float4), s));
    if (with_dip) SBH_TRY(dalloc((void**)&D.dip, cap * sizeof(float4), s));
    if (with_dip && with_rec) SBH_TRY(dalloc((void**)&D.pmd, 2 * cap * sizeof(float4), s));
    SBH_TRY(dalloc((void**)&D.cdf, cap * sizeof(float), s));
    SBH_TRY(dalloc((void**)&D.gd, cap * sizeof(uint8_t), s));
    SBH_TRY(dalloc((void**)&D.fc, cap * sizeof(int32_t), s));
    SBH_TRY(dalloc((void**)&D.meta, cap * sizeof(uint32_t), s));
    SBH_TRY(dalloc((void**)&D.nb, cap * sizeof(int32_t), s));
    SBH_TRY(dalloc((void**)&D.ne, cap * sizeof(int32_t), s));
    SBH_TRY(dalloc((void**)&D.parent, cap * sizeof(int32_t), s));
    if (with_skip) SBH_TRY(dalloc((void**)&D.skip, cap * sizeof(int32_t), s));
    SBH_TRY(dalloc((void**)&D.minl, cap * sizeof(int32_t), s));
    SBH_TRY(dalloc((void**)&D.agg, cap * 8 * sizeof(double), s));
    if (!D.ctrl) SBH_TRY(dalloc((void**)&D.ctrl, sizeof(TreeCtrl), s));
    return cudaSuccess;
}

void free_tree(DeviceTree& D, cudaStream_t s)
{
    dfree(D.pm, s); dfree(D.dip, s); dfree(D.pmd, s); dfree(D.cdf, s); dfree(D.gd, s); dfree(D.fc, s); dfree(D.meta, s); dfree(D.nb, s);
    dfree(D.ne, s); dfree(D.parent, s); dfree(D.skip, s); dfree(D.minl, s); dfree(D.agg, s); dfree(D.ctrl, s);
    D = DeviceTree();
}

cudaError_t build_sorted(sbh_tree* T, const float* pts, const float* w, const float* nrm, cudaStream_t s,
                         int* bad_points, int* bad_weights)
{
    const int64_t n = T->n;
    ScratchSet guard(s);
    int* scratch = nullptr;
    SBH_TRY(guard.alloc(&scratch, 8 * sizeof(int)));
    k_bounds_init<<<1, 32, 0, s>>>(scratch);
    note_launch();
    k_bounds<<<grid_for(n), kThreads, 0, s>>>(pts, w, n, scratch);
    note_launch();
    int host[8];
    SBH_TRY(cudaMemcpyAsync(host, scratch, sizeof(host), cudaMemcpyDeviceToHost, s));
    SBH_TRY(cudaStreamSynchronize(s));
    *bad_points = host[6];
    *bad_weights = host[7];
    if (host[6] || host[7]) return cudaSuccess;
    k_root_cube<<<1, 32, 0, s>>>(scratch, T->t4.ctrl, T->t2.ctrl);
    note_launch();
    SBH_TRY(cudaGetLastError());

    uint64_t *k0 = nullptr, *k1 = nullptr;
    int32_t *v0 = nullptr, *v1 = nullptr;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t nhist = (int64_t)256 * ntiles;
    int *hist = nullptr, *tmp = nullptr;
    SBH_TRY(guard.alloc(&k0, n * sizeof(uint64_t)));
    SBH_TRY(guard.alloc(&k1, n * sizeof(uint64_t)));
    SBH_TRY(guard.alloc(&v0, n * sizeof(int32_t)));
    SBH_TRY(guard.alloc(&v1, n * sizeof(int32_t)));
    SBH_TRY(guard.alloc(&hist, nhist * sizeof(int)));
    SBH_TRY(guard.alloc(&tmp, scan_temp_ints(nhist) * sizeof(int)));
    k_morton<<<grid_for(n), kThreads, 0, s>>>(pts, n, T->t4.ctrl, k0, v0);
    note_launch();
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        k_radix_hist<<<ntiles, kSortThreads, 0, s>>>(k0, n, shift, ntiles, hist);
        note_launch();
        scan_exclusive(hist, hist, nhist, tmp, s);
        k_radix_scatter<<<ntiles, kSortThreads, 0, s>>>(k0, v0, n, shift, ntiles, hist, k1, v1);
        note_launch();
        uint64_t* tk = k0; k0 = k1; k1 = tk;
        int32_t* tv = v0; v0 = v1; v1 = tv;
    }
    SBH_TRY(cudaGetLastError());
    T->code = k0;
    T->perm = v0;
    guard.keep(k0);
    guard.keep(v0);

    SBH_TRY(dalloc((void**)&T->spw, n * sizeof(float4), s));
    if (nrm) SBH_TRY(dalloc((void**)&T->snrm, n * sizeof(float4), s));
    SBH_TRY(dalloc((void**)&T->lcp4, n, s));
    SBH_TRY(dalloc((void**)&T->lcp2, n, s));
    k_gather<<<grid_for(n), kThreads, 0, s>>>(pts, w, nrm, T->perm, n, T->spw, T->snrm);
    note_launch();
    k_lcp<<<grid_for(n), kThreads, 0, s>>>(T->code, n, T->lcp4, T->lcp2);
    note_launch();
    return cudaGetLastError();
}

cudaError_t build_tree(sbh_tree* T, DeviceTree& D, const uint8_t* lcp, int max_level, int level_shift,
                       bool with_skip, cudaStream_t s)
{
    const int64_t n = T->n;
    D.max_level = max_level;
    D.level_shift = level_shift;
    ScratchSet guard(s);
    int32_t *cid = nullptr, *flag = nullptr, *scan = nullptr, *tmp = nullptr, *rmin = nullptr;
    SBH_TRY(guard.alloc(&cid, n * sizeof(int32_t)));
    SBH_TRY(guard.alloc(&flag, n * sizeof(int32_t)));
    SBH_TRY(guard.alloc(&scan, n * sizeof(int32_t)));
    SBH_TRY(guard.alloc(&tmp, scan_temp_ints(n) * sizeof(int32_t)));
    SBH_TRY(guard.alloc(&rmin, sizeof(int32_t)));

    BuildArrays B;
    B.nb = D.nb; B.ne = D.ne; B.fc = D.fc; B.parent = D.parent; B.meta = D.meta; B.minl = D.minl;
    B.cid = cid; B.flag = flag; B.scan = scan; B.lcp = lcp; B.ctrl = D.ctrl; B.n = n;
    B.leaf_size = T->leaf_size; B.max_level = max_level;

    const unsigned g = grid_for(n);
    k_set_int<<<1, 32, 0, s>>>(rmin, 255);
    note_launch();
    k_min_u8<<<g, kThreads, 0, s>>>(lcp, n, rmin);
    note_launch();
    k_topo_root<<<1, 32, 0, s>>>(B, rmin);
    note_launch();
    k_topo_seed<<<g, kThreads, 0, s>>>(B);
    note_launch();
    const int generations = max_level + 2;  // levels strictly increase; points end one below the deepest level
    for (int gen = 0; gen < generations; ++gen) {
        k_topo_flags<<<g, kThreads, 0, s>>>(B);
        note_launch();
        scan_exclusive(flag, scan, n, tmp, s);
        k_topo_children<<<g, kThreads, 0, s>>>(B, gen);
        note_launch();
        k_topo_minlcp<<<g, kThreads, 0, s>>>(B, gen);
        note_launch();
        k_topo_classify<<<g, kThreads, 0, s>>>(B, gen);
        note_launch();
    }
    SBH_TRY(cudaGetLastError());
    for (int gen = generations; gen >= 0; --gen) {
        k_aggregate<<<grid_for(n), kThreads, 0, s>>>(D.fc, D.meta, D.nb, T->spw, T->snrm, D.ctrl, gen, D.agg);
        note_launch();
    }
    k_pack<<<grid_for(2 * n), kThreads, 0, s>>>(D.agg, D.fc, D.meta, D.nb, D.parent, T->spw, T->snrm, D.ctrl, D.pm,
                                                D.dip, D.pmd, D.cdf);
    note_launch();
    k_guide<<<grid_for(2 * n), kThreads, 0, s>>>(D.fc, D.meta, D.parent, D.cdf, D.ctrl, D.gd);
    note_launch();
    k_finalize<<<1, 32, 0, s>>>(D.ctrl, D.fc, D.meta);
    note_launch();
    if (with_skip) {
        for (int gen = 0; gen <= generations; ++gen) {
            k_skip<<<grid_for(n), kThreads, 0, s>>>(D.parent, D.fc, D.meta, D.ctrl, gen, D.skip);
            note_launch();
        }
    }
    SBH_TRY(cudaGetLastError());
    D.built = true;
    return cudaSuccess;
}

}  // namespace sbh

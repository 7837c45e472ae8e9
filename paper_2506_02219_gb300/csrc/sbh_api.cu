// sbh_api.cu -- the extern "C" entry points declared in include/sbh.h: argument checks, error
// reporting, ownership of the tree object, and dispatch to the build and evaluation kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <vector>
#include <new>

#include "sbh.h"
#include "sbh_build.cuh"
#include "sbh_eval.cuh"
#include "sbh_learned.cuh"

namespace sbh {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<int> g_sm_count[64];
int device_sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int n = g_sm_count[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = 1;  // no usable device: the launch that follows reports the error
    }
    g_sm_count[dev].store(n, std::memory_order_relaxed);
    return n;
}
}  // namespace sbh

namespace {

thread_local char g_err[512] = "";

sbh_status fail(sbh_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

}  // namespace

void sbh::set_error_message(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

namespace {

sbh_status cuda_fail(cudaError_t e, const char* what)
{
    const sbh_status st = (e == cudaErrorMemoryAllocation) ? SBH_ENOMEM : SBH_ECUDA;
    return fail(st, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// nonzero if p is usable from the current device (device or managed memory)
bool device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

sbh_status check_kernel(const sbh_kernel& k, sbh::KernelParams* kp)
{
    if (k.kind < SBH_COULOMB || k.kind > SBH_AFFINE) return fail(SBH_EINVAL, "unknown kernel kind %d", (int)k.kind);
    if (k.kind == SBH_COULOMB && !(k.softening >= 0.0f && isfinite(k.softening)))
        return fail(SBH_EINVAL, "softening must be finite and >= 0");
    if (k.kind == SBH_SMOOTHDIST && !(k.alpha > 0.0f && isfinite(k.alpha)))
        return fail(SBH_EINVAL, "alpha must be finite and > 0");
    kp->kind = k.kind;
    kp->eps2 = k.softening * k.softening;
    kp->alpha = k.alpha;
    for (int i = 0; i < 3; ++i) kp->g[i] = k.affine[i];
    return SBH_OK;
}

void release(sbh_tree* T, cudaStream_t s)
{
    sbh::free_tree(T->t4, s);
    sbh::free_tree(T->t2, s);
    sbh::dfree(T->code, s);
    sbh::dfree(T->perm, s);
    sbh::dfree(T->spw, s);
    sbh::dfree(T->snrm, s);
    sbh::dfree(T->lcp4, s);
    sbh::dfree(T->lcp2, s);
    cudaStreamSynchronize(s);
    delete T;
}

constexpr int64_t kMaxPoints = (int64_t)1 << 28;

bool opts_ok(const sbh_eval_opts& o)
{
    return o.sampling >= 0 && o.sampling <= 1 && o.rr >= 0 && o.rr <= 2 && o.seed_mode >= 0 && o.seed_mode <= 1 &&
           o.raw_sum >= 0 && o.raw_sum <= 1 && o.schedule >= 0 && o.schedule <= 1;
}

}  // namespace

extern "C" {

int32_t sbh_version(void) { return SBH_VERSION; }

const char* sbh_last_error(void) { return g_err; }

sbh_status sbh_build(const float* points, const float* weights, const float* normals, int64_t n, int32_t leaf_size,
                     void* stream, sbh_tree** out)
{
    g_err[0] = 0;
    if (!out) return fail(SBH_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > kMaxPoints) return fail(SBH_EINVAL, "n = %lld outside [1, 2^28]", (long long)n);
    if (leaf_size < 1 || leaf_size > sbh::kMaxLeafSize)
        return fail(SBH_EINVAL, "leaf_size = %d outside [1, %d]", (int)leaf_size, sbh::kMaxLeafSize);
    if (!device_ptr(points) || !device_ptr(weights))
        return fail(SBH_EINVAL, "points and weights must be device memory");
    if (normals && !device_ptr(normals)) return fail(SBH_EINVAL, "normals must be device memory or NULL");
    cudaStream_t s = (cudaStream_t)stream;
    sbh_tree* T = new (std::nothrow) sbh_tree();
    if (!T) return fail(SBH_ENOMEM, "host allocation failed");
    T->n = n;
    T->leaf_size = leaf_size;
    T->has_normals = normals != nullptr;
    T->stream = s;
    cudaGetDevice(&T->device);
    cudaError_t e = sbh::alloc_tree(T->t4, n, normals != nullptr, false, normals != nullptr, s);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&T->t2.ctrl, sizeof(sbh::TreeCtrl), s);
    if (e != cudaSuccess) {
        release(T, s);
        return cuda_fail(e, "sbh_build allocation");
    }
    int bad_p = 0, bad_w = 0;
    e = sbh::build_sorted(T, points, weights, normals, s, &bad_p, &bad_w);
    if (e != cudaSuccess) {
        release(T, s);
        return cuda_fail(e, "sbh_build sort");
    }
    if (bad_p || bad_w) {
        release(T, s);
        return fail(SBH_EINVAL, "sbh_build: %d non-finite coordinates, %d weights not finite and > 0", bad_p, bad_w);
    }
    e = sbh::build_tree(T, T->t4, T->lcp4, sbh::kMaxLevel4, 2, false, s);
    if (e != cudaSuccess) {
        release(T, s);
        return cuda_fail(e, "sbh_build tree");
    }
    e = cudaMemcpyAsync(&T->host_ctrl4, T->t4.ctrl, sizeof(sbh::TreeCtrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        release(T, s);
        return cuda_fail(e, "sbh_build");
    }
    if (T->host_ctrl4.error) {
        release(T, s);
        return fail(SBH_EUNSUPPORTED, "sbh_build: more than 2^24 - 1 points share one deepest-level cell");
    }
    *out = T;
    return SBH_OK;
}

sbh_status sbh_eval(const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                    int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts, float* out, void* stream)
{
    g_err[0] = 0;
    if (!tree || !tree->t4.built) return fail(SBH_EINVAL, "tree is NULL or not built");
    if (nq < 0) return fail(SBH_EINVAL, "nq < 0");
    if (samples_per_subdomain < 1 || samples_per_subdomain > SBH_MAX_SAMPLES_PER_SUBDOMAIN)
        return fail(SBH_EINVAL, "samples_per_subdomain = %d outside [1, %d]", (int)samples_per_subdomain,
                    (int)SBH_MAX_SAMPLES_PER_SUBDOMAIN);
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    sbh_eval_opts o = {0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (!opts_ok(o))
        return fail(SBH_EINVAL, "sbh_eval_opts out of range");
    if (nq == 0) return SBH_OK;
    if (!device_ptr(queries) || !device_ptr(out)) return fail(SBH_EINVAL, "queries and out must be device memory");
    cudaError_t e = sbh::launch_stoch_eval(tree->t4.view(), tree->host_ctrl4, queries, nq, kp, samples_per_subdomain,
                                           seed, o, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval launch");
    return SBH_OK;
}

namespace {
// per-device copy streams of sbh_solve_host (created on first use, kept for the process)
std::mutex g_copy_mutex;
cudaStream_t g_copy_in[64], g_copy_out[64];

cudaError_t copy_streams(cudaStream_t* ci, cudaStream_t* co)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_copy_mutex);
    if (!g_copy_in[dev]) {
        e = cudaStreamCreateWithFlags(&g_copy_in[dev], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g_copy_out[dev], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    *ci = g_copy_in[dev];
    *co = g_copy_out[dev];
    return cudaSuccess;
}
}  // namespace

sbh_status sbh_solve_host(const float* points, const float* weights, const float* normals, int64_t n,
                          int32_t leaf_size, const float* queries, int64_t nq, sbh_kernel kernel,
                          int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts, int64_t chunk,
                          float* out, void* stream)
{
    g_err[0] = 0;
    if (!points || !weights || (nq > 0 && (!queries || !out))) return fail(SBH_EINVAL, "NULL buffer");
    if (device_ptr(points) || device_ptr(weights) || (normals && device_ptr(normals)) ||
        (nq > 0 && (device_ptr(queries) || device_ptr(out))))
        return fail(SBH_EINVAL, "sbh_solve_host takes host buffers (use sbh_build and sbh_eval for device ones)");
    if (nq < 0 || chunk < 0) return fail(SBH_EINVAL, "nq and chunk must be >= 0");
    if (samples_per_subdomain < 1 || samples_per_subdomain > SBH_MAX_SAMPLES_PER_SUBDOMAIN)
        return fail(SBH_EINVAL, "samples_per_subdomain = %d outside [1, %d]", (int)samples_per_subdomain,
                    (int)SBH_MAX_SAMPLES_PER_SUBDOMAIN);
    if (n < 1 || n > kMaxPoints) return fail(SBH_EINVAL, "n = %lld outside [1, 2^28]", (long long)n);
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !normals) return fail(SBH_EINVAL, "the winding-number kernel needs normals");
    sbh_eval_opts o = {0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (!opts_ok(o)) return fail(SBH_EINVAL, "sbh_eval_opts out of range");
    // each chunk adds a launch tail (~0.15 ms), but the first chunk's evaluation starts after half
    // of the query upload (which outlasts the build where the host link is slow) and its download
    // overlaps the second chunk: two chunks from 2^22 queries on (measured even where the link is
    // fast: 28.80 ms for one or two chunks at 2^24 queries)
    if (chunk == 0) chunk = nq >= (int64_t(1) << 22) ? (nq + 1) / 2 : std::max<int64_t>(nq, 1);
    // whole 32-query tiles: a tile's results depend on its queries only, so the chunks' tiles must
    // be those of one launch over all queries
    chunk = (chunk + 31) / 32 * 32;
    const int64_t n_chunks = nq > 0 ? (nq + chunk - 1) / chunk : 0;
    cudaStream_t s = (cudaStream_t)stream, ci = nullptr, co = nullptr;
    cudaError_t e = copy_streams(&ci, &co);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_solve_host streams");
    float *dP = nullptr, *dW = nullptr, *dN = nullptr, *dQ = nullptr, *dO = nullptr;
    std::vector<cudaEvent_t> ev((size_t)(2 * n_chunks + 2), nullptr);
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&dP, (size_t)n * 3 * sizeof(float), s);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&dW, (size_t)n * sizeof(float), s);
    if (e == cudaSuccess && normals) e = sbh::dalloc((void**)&dN, (size_t)n * 3 * sizeof(float), s);
    if (e == cudaSuccess && nq > 0) e = sbh::dalloc((void**)&dQ, (size_t)nq * 3 * sizeof(float), s);
    if (e == cudaSuccess && nq > 0) e = sbh::dalloc((void**)&dO, (size_t)nq * sizeof(float), s);
    // the sources go first (the build needs them; uploads share the copy engine), then the
    // queries chunk by chunk on the copy stream, overlapping the build
    if (e == cudaSuccess) e = cudaMemcpyAsync(dP, points, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dW, weights, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && normals)
        e = cudaMemcpyAsync(dN, normals, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ci, ev[0], 0);
    for (int64_t k = 0; k < n_chunks && e == cudaSuccess; ++k) {
        const int64_t b = k * chunk, m = std::min(chunk, nq - b);
        e = cudaMemcpyAsync(dQ + 3 * b, queries + 3 * b, (size_t)m * 3 * sizeof(float), cudaMemcpyHostToDevice, ci);
        if (e == cudaSuccess) e = cudaEventRecord(ev[(size_t)(1 + k)], ci);
    }
    sbh_tree* tree = nullptr;
    if (e == cudaSuccess) {
        st = sbh_build(dP, dW, dN, n, leaf_size, (void*)s, &tree);  // synchronises s
        if (st != SBH_OK) {
            cudaStreamSynchronize(ci);
            sbh::dfree(dP, s); sbh::dfree(dW, s); sbh::dfree(dN, s); sbh::dfree(dQ, s); sbh::dfree(dO, s);
            cudaStreamSynchronize(s);
            for (auto& x : ev) if (x) cudaEventDestroy(x);
            return st;
        }
    }
    // evaluate each chunk as it lands; its results go out on the second copy stream
    for (int64_t k = 0; k < n_chunks && e == cudaSuccess; ++k) {
        const int64_t b = k * chunk, m = std::min(chunk, nq - b);
        e = cudaStreamWaitEvent(s, ev[(size_t)(1 + k)], 0);
        if (e == cudaSuccess)
            e = sbh::launch_stoch_eval(tree->t4.view(), tree->host_ctrl4, dQ + 3 * b, m, kp, samples_per_subdomain,
                                       seed, o, dO + b, s, b);
        if (e == cudaSuccess) e = cudaEventRecord(ev[(size_t)(1 + n_chunks + k)], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(co, ev[(size_t)(1 + n_chunks + k)], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out + b, dO + b, (size_t)m * sizeof(float), cudaMemcpyDeviceToHost, co);
    }
    // everything done before the buffers go back to the pool
    const cudaError_t e_in = cudaStreamSynchronize(ci), e_out = cudaStreamSynchronize(co);
    if (e == cudaSuccess) e = e_in != cudaSuccess ? e_in : e_out;
    if (tree) sbh_tree_free(tree);
    sbh::dfree(dP, s); sbh::dfree(dW, s); sbh::dfree(dN, s); sbh::dfree(dQ, s); sbh::dfree(dO, s);
    const cudaError_t e_s = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e_s;
    for (auto& x : ev) if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_solve_host");
    return SBH_OK;
}

sbh_status sbh_eval_count(const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                          int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                          unsigned long long* counts, void* stream)
{
    g_err[0] = 0;
    if (!tree || !tree->t4.built) return fail(SBH_EINVAL, "tree is NULL or not built");
    if (nq < 0) return fail(SBH_EINVAL, "nq < 0");
    if (samples_per_subdomain < 1 || samples_per_subdomain > SBH_MAX_SAMPLES_PER_SUBDOMAIN)
        return fail(SBH_EINVAL, "samples_per_subdomain = %d outside [1, %d]", (int)samples_per_subdomain,
                    (int)SBH_MAX_SAMPLES_PER_SUBDOMAIN);
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    sbh_eval_opts o = {0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (!opts_ok(o))
        return fail(SBH_EINVAL, "sbh_eval_opts out of range");
    if (!device_ptr(counts)) return fail(SBH_EINVAL, "counts must be device memory");
    if (nq == 0) return SBH_OK;
    if (!device_ptr(queries)) return fail(SBH_EINVAL, "queries must be device memory");
    cudaError_t e = sbh::launch_stoch_count(tree->t4.view(), queries, nq, kp, samples_per_subdomain, seed, o, counts,
                                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval_count launch");
    return SBH_OK;
}

sbh_status sbh_eval_grad(const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                         int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts, float* out,
                         float* grad, void* stream)
{
    g_err[0] = 0;
    if (!tree || !tree->t4.built) return fail(SBH_EINVAL, "tree is NULL or not built");
    if (nq < 0) return fail(SBH_EINVAL, "nq < 0");
    if (samples_per_subdomain < 1 || samples_per_subdomain > SBH_MAX_SAMPLES_PER_SUBDOMAIN)
        return fail(SBH_EINVAL, "samples_per_subdomain = %d outside [1, %d]", (int)samples_per_subdomain,
                    (int)SBH_MAX_SAMPLES_PER_SUBDOMAIN);
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    sbh_eval_opts o = {0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (!opts_ok(o))
        return fail(SBH_EINVAL, "sbh_eval_opts out of range");
    if (nq == 0) return SBH_OK;
    if (!device_ptr(queries) || !device_ptr(out) || !device_ptr(grad))
        return fail(SBH_EINVAL, "queries, out and grad must be device memory");
    cudaError_t e = sbh::launch_stoch_grad(tree->t4.view(), tree->host_ctrl4, queries, nq, kp, samples_per_subdomain, seed, o, out, grad,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval_grad launch");
    return SBH_OK;
}

}  // extern "C"

struct sbh_multi_plan {
    int device = 0;
    int32_t n_sets = 0;
    int64_t total_tiles = 0;
    void* descs = nullptr;                  // device array of set descriptors
    unsigned long long* counter = nullptr;  // device tile counter
    sbh::KernelParams kp;
    int32_t S = 1;
    uint64_t seed = 0;
    sbh_eval_opts opts;
};

extern "C" {

sbh_status sbh_multi_plan_create(const sbh_tree* const* trees, const float* const* queries, const int64_t* nq,
                                 float* const* outs, int32_t n_sets, sbh_kernel kernel, int32_t samples_per_subdomain,
                                 uint64_t seed, const sbh_eval_opts* opts, void* stream, sbh_multi_plan** plan)
{
    g_err[0] = 0;
    if (!plan) return fail(SBH_EINVAL, "plan is NULL");
    *plan = nullptr;
    if (n_sets < 1 || !trees || !queries || !nq || !outs) return fail(SBH_EINVAL, "n_sets >= 1 and non-NULL arrays");
    if (samples_per_subdomain < 1 || samples_per_subdomain > SBH_MAX_SAMPLES_PER_SUBDOMAIN)
        return fail(SBH_EINVAL, "samples_per_subdomain = %d outside [1, %d]", (int)samples_per_subdomain,
                    (int)SBH_MAX_SAMPLES_PER_SUBDOMAIN);
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    sbh_eval_opts o = {0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (!opts_ok(o)) return fail(SBH_EINVAL, "sbh_eval_opts out of range");
    const size_t db = sbh::multi_set_desc_bytes();
    unsigned char* host = new (std::nothrow) unsigned char[db * (size_t)n_sets];
    if (!host) return fail(SBH_ENOMEM, "host allocation failed");
    int64_t tiles = 0;
    for (int32_t i = 0; i < n_sets; ++i) {
        const sbh_tree* t = trees[i];
        if (!t || !t->t4.built) { delete[] host; return fail(SBH_EINVAL, "set %d: tree is NULL or not built", i); }
        if (nq[i] < 0) { delete[] host; return fail(SBH_EINVAL, "set %d: nq < 0", i); }
        if (kernel.kind == SBH_WINDING && !t->has_normals) {
            delete[] host;
            return fail(SBH_EINVAL, "set %d: the winding-number kernel needs a tree built with normals", i);
        }
        if (nq[i] > 0 && (!device_ptr(queries[i]) || !device_ptr(outs[i]))) {
            delete[] host;
            return fail(SBH_EINVAL, "set %d: queries and out must be device memory", i);
        }
        sbh::multi_fill_desc(host + db * (size_t)i, t->t4.view(), queries[i], outs[i], nq[i], tiles);
        tiles += (nq[i] + 31) / 32;
    }
    sbh_multi_plan* P = new (std::nothrow) sbh_multi_plan();
    if (!P) { delete[] host; return fail(SBH_ENOMEM, "host allocation failed"); }
    cudaStream_t s = (cudaStream_t)stream;
    cudaGetDevice(&P->device);
    cudaError_t e = sbh::dalloc(&P->descs, db * (size_t)n_sets, s);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&P->counter, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->descs, host, db * (size_t)n_sets, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] host;
    if (e != cudaSuccess) {
        sbh::dfree(P->descs, s);
        sbh::dfree(P->counter, s);
        cudaStreamSynchronize(s);
        delete P;
        return cuda_fail(e, "sbh_multi_plan_create");
    }
    P->n_sets = n_sets;
    P->total_tiles = tiles;
    P->kp = kp;
    P->S = samples_per_subdomain;
    P->seed = seed;
    P->opts = o;
    *plan = P;
    return SBH_OK;
}

sbh_status sbh_multi_plan_launch(const sbh_multi_plan* plan, void* stream)
{
    g_err[0] = 0;
    if (!plan) return fail(SBH_EINVAL, "plan is NULL");
    cudaError_t e = sbh::launch_stoch_multi(plan->descs, plan->n_sets, plan->total_tiles, plan->counter, plan->kp,
                                            plan->S, plan->seed, plan->opts, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_multi_plan_launch");
    return SBH_OK;
}

void sbh_multi_plan_free(sbh_multi_plan* plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    sbh::dfree(plan->descs, nullptr);
    sbh::dfree(plan->counter, nullptr);
    cudaStreamSynchronize(nullptr);
    delete plan;
}

}  // extern "C"

struct sbh_mlp {
    int device = 0;
    sbh::MlpState M;
};

namespace {
// deterministic host initialisation: He-scaled normals from splitmix64 + Box-Muller
uint64_t splitmix64(uint64_t& x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unit_open(uint64_t& st) { return ((double)(splitmix64(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
double normal(uint64_t& st)
{
    const double u = unit_open(st), v = unit_open(st);
    return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
}
}  // namespace

extern "C" {

sbh_status sbh_mlp_create(uint64_t seed, void* stream, sbh_mlp** out)
{
    g_err[0] = 0;
    if (!out) return fail(SBH_EINVAL, "out is NULL");
    *out = nullptr;
    sbh_mlp* N = new (std::nothrow) sbh_mlp();
    if (!N) return fail(SBH_ENOMEM, "host allocation failed");
    cudaStream_t s = (cudaStream_t)stream;
    cudaGetDevice(&N->device);
    std::vector<float> w(sbh::kMlpParams, 0.0f);
    uint64_t st = seed;
    for (int i = 0; i < 32 * 6; ++i) w[i] = (float)(normal(st) * std::sqrt(2.0 / 6.0));
    for (int i = 0; i < 32 * 32; ++i) w[224 + i] = (float)(normal(st) * std::sqrt(2.0 / 32.0));
    for (int i = 0; i < 32; ++i) w[1280 + i] = (float)(normal(st) * std::sqrt(1.0 / 32.0));
    cudaError_t e = sbh::mlp_alloc(N->M, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(N->M.w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sbh::mlp_sync_half(N->M, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        sbh::mlp_release(N->M, s);
        delete N;
        return cuda_fail(e, "sbh_mlp_create");
    }
    *out = N;
    return SBH_OK;
}

sbh_status sbh_mlp_set_weights(sbh_mlp* net, const float* host_weights, void* stream)
{
    g_err[0] = 0;
    if (!net || !host_weights) return fail(SBH_EINVAL, "net and weights must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(net->M.w, host_weights, sbh::kMlpParams * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sbh::mlp_sync_half(net->M, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_set_weights");
    return SBH_OK;
}

sbh_status sbh_mlp_get_weights(const sbh_mlp* net, float* host_weights, int64_t* adam_step, void* stream)
{
    g_err[0] = 0;
    if (!net || !host_weights) return fail(SBH_EINVAL, "net and weights must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(host_weights, net->M.w, sbh::kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_get_weights");
    if (adam_step) *adam_step = net->M.step;
    return SBH_OK;
}

sbh_status sbh_mlp_get_state(const sbh_mlp* net, float* host_state, int64_t* adam_step, void* stream)
{
    g_err[0] = 0;
    if (!net || !host_state || !adam_step) return fail(SBH_EINVAL, "net, state and step must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b = sbh::kMlpParams * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(host_state, net->M.w, b, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_state + sbh::kMlpParams, net->M.m, b, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_state + 2 * sbh::kMlpParams, net->M.v, b, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_get_state");
    *adam_step = net->M.step;
    return SBH_OK;
}

sbh_status sbh_mlp_set_state(sbh_mlp* net, const float* host_state, int64_t adam_step, void* stream)
{
    g_err[0] = 0;
    if (!net || !host_state || adam_step < 0) return fail(SBH_EINVAL, "net and state must be non-NULL, step >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b = sbh::kMlpParams * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(net->M.w, host_state, b, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->M.m, host_state + sbh::kMlpParams, b, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->M.v, host_state + 2 * sbh::kMlpParams, b, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sbh::mlp_sync_half(net->M, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_set_state");
    net->M.step = adam_step;
    return SBH_OK;
}

sbh_status sbh_mlp_scores(const sbh_mlp* net, const float* feats, int64_t n, float* scores, void* stream)
{
    g_err[0] = 0;
    if (!net || n < 0) return fail(SBH_EINVAL, "net is NULL or n < 0");
    if (n == 0) return SBH_OK;
    if (!device_ptr(feats) || !device_ptr(scores)) return fail(SBH_EINVAL, "feats and scores must be device memory");
    cudaError_t e = sbh::mlp_scores(net->M, feats, n, scores, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_scores");
    return SBH_OK;
}

sbh_status sbh_mlp_loss_grad(sbh_mlp* net, const float* feats, const float* targets, const int64_t* offsets,
                             int64_t n_sets, float* grad, float* loss, void* stream)
{
    g_err[0] = 0;
    if (!net || n_sets < 1) return fail(SBH_EINVAL, "net is NULL or n_sets < 1");
    if (!device_ptr(feats) || !device_ptr(targets) || !device_ptr(offsets) || !device_ptr(grad) || !device_ptr(loss))
        return fail(SBH_EINVAL, "all buffers must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = sbh::mlp_loss_grad(net->M, feats, targets, offsets, n_sets, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad, net->M.grad, sbh::kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, net->M.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_loss_grad");
    return SBH_OK;
}

sbh_status sbh_mlp_dataset(const sbh_tree* tree, const float* queries, sbh_kernel kernel, const int32_t* set_query,
                           const int32_t* set_node, const int64_t* set_offsets, int64_t n_sets, float* feats,
                           float* targets, void* stream)
{
    g_err[0] = 0;
    if (!tree || !tree->t4.built) return fail(SBH_EINVAL, "tree missing");
    if (n_sets < 0) return fail(SBH_EINVAL, "n_sets < 0");
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    if (n_sets == 0) return SBH_OK;
    if (!device_ptr(queries) || !device_ptr(set_query) || !device_ptr(set_node) || !device_ptr(set_offsets) ||
        !device_ptr(feats) || !device_ptr(targets))
        return fail(SBH_EINVAL, "all buffers must be device memory");
    cudaError_t e = sbh::mlp_dataset(tree, queries, set_query, set_node, n_sets, set_offsets, kp, feats, targets,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_dataset");
    return SBH_OK;
}

namespace {
constexpr int kTrainPaths = 4;            // paths per subdomain walked by each training query
constexpr int kTrainSetsPerQuery = 4096;  // cap on the decision sets one training query contributes
constexpr uint64_t kTrainSeed = 0x7EA1ull;
}  // namespace

sbh_status sbh_mlp_train(sbh_mlp* net, const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                         float near, int32_t steps, float lr, float* losses, void* stream)
{
    g_err[0] = 0;
    if (!net || !tree || !tree->t4.built) return fail(SBH_EINVAL, "net or tree missing");
    if (nq < 1 || nq > (1 << 20) || steps < 0 || !(lr > 0.0f)) return fail(SBH_EINVAL, "need 1 <= nq <= 2^20, steps >= 0, lr > 0");
    if (!(near >= 0.0f)) return fail(SBH_EINVAL, "near must be >= 0");
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    if (!device_ptr(queries)) return fail(SBH_EINVAL, "queries must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    const sbh::TreeView T = tree->t4.view();
    // 1. the decision sets the estimator's own paths reach (count, offsets, fill)
    int32_t* dcount = nullptr;
    int64_t* dbase = nullptr;
    int32_t *set_q = nullptr, *set_node = nullptr;
    int64_t *rows = nullptr, *doff = nullptr;
    float *feats = nullptr, *targets = nullptr;
    std::vector<int32_t> count((size_t)nq);
    std::vector<int64_t> base((size_t)nq);
    cudaError_t e = sbh::dalloc((void**)&dcount, nq * sizeof(int32_t), s);
    if (e == cudaSuccess) e = sbh::mlp_visit(T, queries, (int)nq, kTrainPaths, kTrainSeed, near, kTrainSetsPerQuery,
                                             dcount, nullptr, nullptr, nullptr, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(count.data(), dcount, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int64_t n_sets = 0;
    for (int64_t j = 0; j < nq; ++j) { base[(size_t)j] = n_sets; n_sets += count[(size_t)j]; }
    std::vector<int64_t> off;
    if (e == cudaSuccess && n_sets == 0) {
        sbh::dfree(dcount, s);
        return fail(SBH_EUNSUPPORTED, "no decision set within reach of the training queries (raise near)");
    }
    if (e == cudaSuccess) e = sbh::dalloc((void**)&dbase, nq * sizeof(int64_t), s);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&set_q, n_sets * sizeof(int32_t), s);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&set_node, n_sets * sizeof(int32_t), s);
    if (e == cudaSuccess) e = sbh::dalloc((void**)&rows, (n_sets + 1) * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbase, base.data(), nq * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sbh::mlp_visit(T, queries, (int)nq, kTrainPaths, kTrainSeed, near, kTrainSetsPerQuery,
                                             nullptr, dbase, set_q, set_node, s);
    if (e == cudaSuccess) e = sbh::mlp_set_rows(T, set_node, n_sets, rows, s);
    if (e == cudaSuccess) {
        off.resize((size_t)n_sets + 1);
        e = cudaMemcpyAsync(off.data() + 1, rows, n_sets * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int64_t total = 0;
    if (e == cudaSuccess) {
        off[0] = 0;
        for (int64_t i = 1; i <= n_sets; ++i) off[(size_t)i] += off[(size_t)i - 1];
        total = off[(size_t)n_sets];
    }
    bool too_large = e == cudaSuccess && total > (int64_t(1) << 26);
    // 2. features and |exact child residual| targets
    if (e == cudaSuccess && !too_large) {
        doff = rows;  // reuse: n_sets + 1 entries
        e = cudaMemcpyAsync(doff, off.data(), (n_sets + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = sbh::dalloc((void**)&feats, total * 6 * sizeof(float), s);
        if (e == cudaSuccess) e = sbh::dalloc((void**)&targets, total * sizeof(float), s);
        if (e == cudaSuccess) e = sbh::mlp_dataset(tree, queries, set_q, set_node, n_sets, doff, kp, feats, targets, s);
        // 3. full-batch Adam steps
        for (int32_t k = 0; k < steps && e == cudaSuccess; ++k) {
            e = sbh::mlp_loss_grad(net->M, feats, targets, doff, n_sets, s);
            if (e == cudaSuccess && losses)
                e = cudaMemcpyAsync(&losses[k], net->M.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = sbh::mlp_adam_step(net->M, lr, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host copies of `losses` are complete
    }
    sbh::dfree(dcount, s);
    sbh::dfree(dbase, s);
    sbh::dfree(set_q, s);
    sbh::dfree(set_node, s);
    sbh::dfree(rows, s);
    sbh::dfree(feats, s);
    sbh::dfree(targets, s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_mlp_train");
    if (too_large) return fail(SBH_EINVAL, "training set too large (more than 2^26 rows): use fewer training queries");
    return SBH_OK;
}

sbh_status sbh_eval_learned(const sbh_tree* tree, const sbh_mlp* net, const float* queries, int64_t nq,
                            sbh_kernel kernel, int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                            float near, float* out, void* stream)
{
    g_err[0] = 0;
    if (!tree || !tree->t4.built || !net) return fail(SBH_EINVAL, "tree or net missing");
    if (nq < 0) return fail(SBH_EINVAL, "nq < 0");
    if (samples_per_subdomain < 1 || samples_per_subdomain > SBH_MAX_SAMPLES_PER_SUBDOMAIN)
        return fail(SBH_EINVAL, "samples_per_subdomain = %d outside [1, %d]", (int)samples_per_subdomain,
                    (int)SBH_MAX_SAMPLES_PER_SUBDOMAIN);
    if (!(near >= 0.0f)) return fail(SBH_EINVAL, "near must be >= 0");
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    sbh_eval_opts o = {0, 0, 0, 0, 0};
    if (opts) o = *opts;
    if (!opts_ok(o)) return fail(SBH_EINVAL, "sbh_eval_opts out of range");
    if (o.sampling != 0) return fail(SBH_EINVAL, "the learned proposal replaces the path-index sampling: sampling must be 0");
    if (nq == 0) return SBH_OK;
    if (!device_ptr(queries) || !device_ptr(out)) return fail(SBH_EINVAL, "queries and out must be device memory");
    cudaError_t e = sbh::launch_stoch_learned(tree->t4.view(), tree->host_ctrl4, net->M.wh, near, queries, nq, kp,
                                              samples_per_subdomain, seed, o, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval_learned launch");
    return SBH_OK;
}

void sbh_mlp_free(sbh_mlp* net)
{
    if (!net) return;
    cudaDeviceSynchronize();
    sbh::mlp_release(net->M, nullptr);
    cudaStreamSynchronize(nullptr);
    delete net;
}

sbh_status sbh_set_allocator(sbh_alloc_fn alloc, sbh_free_fn free_fn, void* ctx)
{
    g_err[0] = 0;
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(SBH_EINVAL, "set both allocator functions or neither");
    sbh::set_allocator(alloc, free_fn, ctx);
    return SBH_OK;
}

sbh_status sbh_set_memory_limit(uint64_t bytes)
{
    g_err[0] = 0;
    sbh::set_memory_limit(bytes);
    return SBH_OK;
}

uint64_t sbh_memory_in_use(void) { return sbh::memory_in_use(); }

unsigned long long sbh_kernel_launches(void) { return sbh::g_launches.load(std::memory_order_relaxed); }

sbh_status sbh_eval_bh(sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel, float theta,
                       int32_t warp_vote, float* out, void* stream)
{
    g_err[0] = 0;
    if (!tree || !tree->t4.built) return fail(SBH_EINVAL, "tree is NULL or not built");
    if (nq < 0) return fail(SBH_EINVAL, "nq < 0");
    if (!(theta >= 0.0f) || !isfinite(theta)) return fail(SBH_EINVAL, "theta must be finite and >= 0");
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (kernel.kind == SBH_WINDING && !tree->has_normals)
        return fail(SBH_EINVAL, "the winding-number kernel needs a tree built with normals");
    cudaStream_t s = (cudaStream_t)stream;
    if (!tree->t2.built) {
        // the root cube of t2.ctrl was written by sbh_build; alloc_tree keeps that block
        cudaError_t e = sbh::alloc_tree(tree->t2, tree->n, tree->has_normals != 0, true, false, s);
        if (e == cudaSuccess) e = sbh::build_tree(tree, tree->t2, tree->lcp2, sbh::kMaxLevel2, 1, true, s);
        if (e != cudaSuccess) {  // give back what was taken, keep the control block with the root cube
            sbh::TreeCtrl* ctrl = tree->t2.ctrl;
            tree->t2.ctrl = nullptr;
            sbh::free_tree(tree->t2, s);
            tree->t2.ctrl = ctrl;
            return cuda_fail(e, "sbh_eval_bh tree build");
        }
        tree->stream = s;
    }
    if (nq == 0) return SBH_OK;
    if (!device_ptr(queries) || !device_ptr(out)) return fail(SBH_EINVAL, "queries and out must be device memory");
    const float beta = theta > 0.0f ? 1.0f / theta : INFINITY;
    cudaError_t e = sbh::launch_bh_eval(tree->t2.view(), queries, nq, kp, beta, warp_vote ? 1 : 0, out, s);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval_bh launch");
    return SBH_OK;
}

sbh_status sbh_eval_brute(const float* points, const float* weights, const float* normals, int64_t n,
                          const float* queries, int64_t nq, sbh_kernel kernel, int32_t fp64_accum, float* out,
                          void* stream)
{
    g_err[0] = 0;
    if (n < 0 || nq < 0) return fail(SBH_EINVAL, "n and nq must be >= 0");
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (nq == 0) return SBH_OK;
    if (n > 0 && (!device_ptr(points) || !device_ptr(weights)))
        return fail(SBH_EINVAL, "points and weights must be device memory");
    if (kernel.kind == SBH_WINDING && n > 0 && !device_ptr(normals))
        return fail(SBH_EINVAL, "the winding-number kernel needs normals");
    if (!device_ptr(queries) || !device_ptr(out)) return fail(SBH_EINVAL, "queries and out must be device memory");
    cudaError_t e = sbh::launch_brute(points, weights, normals, n, queries, nq, kp, fp64_accum ? 1 : 0, out,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval_brute launch");
    return SBH_OK;
}

sbh_status sbh_eval_brute_grad(const float* points, const float* weights, const float* normals, int64_t n,
                               const float* queries, int64_t nq, sbh_kernel kernel, float* out, float* grad,
                               void* stream)
{
    g_err[0] = 0;
    if (n < 0 || nq < 0) return fail(SBH_EINVAL, "n and nq must be >= 0");
    sbh::KernelParams kp;
    sbh_status st = check_kernel(kernel, &kp);
    if (st != SBH_OK) return st;
    if (nq == 0) return SBH_OK;
    if (n > 0 && (!device_ptr(points) || !device_ptr(weights)))
        return fail(SBH_EINVAL, "points and weights must be device memory");
    if (kernel.kind == SBH_WINDING && n > 0 && !device_ptr(normals))
        return fail(SBH_EINVAL, "the winding-number kernel needs normals");
    if (!device_ptr(queries) || !device_ptr(out) || !device_ptr(grad))
        return fail(SBH_EINVAL, "queries, out and grad must be device memory");
    cudaError_t e = sbh::launch_brute_grad(points, weights, normals, n, queries, nq, kp, out, grad,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_eval_brute_grad launch");
    return SBH_OK;
}

sbh_status sbh_tree_info(const sbh_tree* tree, int32_t which, sbh_tree_meta* meta)
{
    g_err[0] = 0;
    if (!tree || !meta) return fail(SBH_EINVAL, "tree or meta is NULL");
    if (which != 0 && which != 1) return fail(SBH_EINVAL, "which must be 0 or 1");
    const sbh::DeviceTree& D = which == 0 ? tree->t4 : tree->t2;
    if (!D.built) return fail(SBH_EUNSUPPORTED, "the 8-ary tree has not been built (call sbh_eval_bh first)");
    sbh::TreeCtrl c;
    cudaError_t e = cudaMemcpyAsync(&c, D.ctrl, sizeof(c), cudaMemcpyDeviceToHost, tree->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(tree->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sbh_tree_info copy");
    memset(meta, 0, sizeof(*meta));
    meta->n_points = tree->n;
    meta->n_nodes = c.n_nodes;
    meta->leaf_size = tree->leaf_size;
    meta->has_normals = tree->has_normals;
    meta->max_depth = c.max_depth;
    meta->first_sub = c.first_sub;
    meta->n_sub = c.n_sub;
    for (int a = 0; a < 3; ++a) meta->lo[a] = c.lo[a];
    meta->side = c.side;
    meta->diam0 = c.diam[0];
    if (c.error) return fail(SBH_ECUDA, "tree build reported an internal inconsistency (%d)", c.error);
    return SBH_OK;
}

sbh_status sbh_tree_export(const sbh_tree* tree, int32_t which, const sbh_tree_export_buffers* buf)
{
    sbh_tree_meta meta;
    sbh_status st = sbh_tree_info(tree, which, &meta);
    if (st != SBH_OK) return st;
    if (!buf) return fail(SBH_EINVAL, "buf is NULL");
    const sbh::DeviceTree& D = which == 0 ? tree->t4 : tree->t2;
    const int64_t n = tree->n, N = meta.n_nodes;
    cudaStream_t s = tree->stream;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    };
    cp(buf->perm, tree->perm, n * sizeof(int32_t));
    cp(buf->code, tree->code, n * sizeof(uint64_t));
    cp(buf->begin, D.nb, N * sizeof(int32_t));
    cp(buf->end, D.ne, N * sizeof(int32_t));
    cp(buf->first_child, D.fc, N * sizeof(int32_t));
    cp(buf->parent, D.parent, N * sizeof(int32_t));
    cp(buf->com_mass, D.pm, N * sizeof(float4));
    cp(buf->cdf, D.cdf, N * sizeof(float));
    cp(buf->guide, D.gd, N * sizeof(uint8_t));
    uint32_t* meta_h = nullptr;
    double* agg_h = nullptr;
    float4* dip_h = nullptr;
    if (buf->nchild || buf->level) {
        meta_h = new (std::nothrow) uint32_t[N];
        if (!meta_h) return fail(SBH_ENOMEM, "host allocation failed");
        cp(meta_h, D.meta, N * sizeof(uint32_t));
    }
    if (buf->com_mass64) {
        agg_h = new (std::nothrow) double[8 * N];
        if (!agg_h) { delete[] meta_h; return fail(SBH_ENOMEM, "host allocation failed"); }
        cp(agg_h, D.agg, 8 * N * sizeof(double));
    }
    if (buf->dipole && D.dip) {
        dip_h = new (std::nothrow) float4[N];
        if (!dip_h) { delete[] meta_h; delete[] agg_h; return fail(SBH_ENOMEM, "host allocation failed"); }
        cp(dip_h, D.dip, N * sizeof(float4));
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        for (int64_t v = 0; v < N; ++v) {
            if (meta_h && buf->nchild) buf->nchild[v] = (int32_t)sbh::meta_nchild(meta_h[v]);
            if (meta_h && buf->level) buf->level[v] = (int32_t)sbh::meta_level(meta_h[v]);
            if (agg_h) {
                const double m = agg_h[8 * v];
                buf->com_mass64[4 * v + 0] = agg_h[8 * v + 1] / m;
                buf->com_mass64[4 * v + 1] = agg_h[8 * v + 2] / m;
                buf->com_mass64[4 * v + 2] = agg_h[8 * v + 3] / m;
                buf->com_mass64[4 * v + 3] = m;
            }
            if (buf->dipole) {
                for (int a = 0; a < 3; ++a)
                    buf->dipole[3 * v + a] = dip_h ? (&dip_h[v].x)[a] : 0.0f;
            }
        }
    }
    delete[] meta_h;
    delete[] agg_h;
    delete[] dip_h;
    if (e != cudaSuccess) return cuda_fail(e, "sbh_tree_export copy");
    return SBH_OK;
}

void sbh_tree_free(sbh_tree* tree)
{
    if (!tree) return;
    cudaStreamSynchronize(tree->stream);
    release(tree, tree->stream);
}

}  // extern "C"

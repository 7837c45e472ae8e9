/*
 * sbh.h -- C ABI of the GB300 stochastic Barnes-Hut library (libsbh.so).
 *
 * The library evaluates kernel sums F(q) = sum_i m_i f(p_i, q) over a source point set for many
 * query points (Madan, Sharp, Williams, Museth, Levin, "Stochastic Barnes-Hut Approximation for
 * Fast Summation on the GPU", SIGGRAPH 2025, Sec. 3, Eq. 1), with
 *   - sbh_build:       the octree-like tree with aggregate mass and centre of mass (Sec. 3.1),
 *                      built on the GPU from Morton codes;
 *   - sbh_eval:        the stratified, unbiased path estimator (Sec. 3.3, Eq. 5-7, Algorithm 2);
 *   - sbh_eval_bh:     deterministic Barnes-Hut (Sec. 3.1, Eq. 2, Algorithm 1), the GPU baseline;
 *   - sbh_eval_brute:  the exact sum by tiled brute force (Eq. 1).
 *
 * Conventions shared by every entry point:
 *   - Buffers are caller-owned, contiguous, C order, FP32 unless stated. Points and queries are
 *     [n][3] (x, y, z interleaved). "device" buffers must be device (or managed) memory of the
 *     current CUDA device; nothing is read from or written to host memory unless stated.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is enqueued on it and
 *     the call returns without synchronising, except where a call says it synchronises.
 *   - Every call returns an sbh_status; nothing throws across the ABI. On failure
 *     sbh_last_error() returns a message for the calling thread, and output buffers are left in
 *     an unspecified state.
 *   - Results are bitwise reproducible for the same inputs, seed and device.
 */
#ifndef SBH_H
#define SBH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SBH_VERSION 1

#if defined(__GNUC__)
#define SBH_API __attribute__((visibility("default")))
#else
#define SBH_API
#endif

typedef enum {
    SBH_OK = 0,
    SBH_EINVAL = 1,       /* an argument is out of its documented range */
    SBH_ENOMEM = 2,       /* device memory could not be allocated */
    SBH_ECUDA = 3,        /* a CUDA runtime call failed; see sbh_last_error() */
    SBH_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
    SBH_EUNSUPPORTED = 5  /* the request needs something this tree or device does not have */
} sbh_status;

/* Kernel f(p, q) of the sum (Sec. 4.2, 4.3). Each source contributes m_i f(p_i, q):
 *   SBH_COULOMB     f = 1 / sqrt(|p - q|^2 + softening^2)              (Sec. 4.2, sign +)
 *   SBH_WINDING     m f = m ((p - q) . n) / (4 pi |p - q|^3), 0 at p = q (Sec. 4.3.2); a node
 *                   uses its dipole sum_j m_j n_j at its centre of mass. Needs normals.
 *   SBH_SMOOTHDIST  f = exp(-alpha |p - q|); the output is the smooth distance
 *                   -log(F) / alpha (Sec. 4.3.3), +inf where the estimate of F is <= 0.
 *   SBH_AFFINE      f = 1 + g . (p - q) with g = affine[0..2]: a test kernel, affine in p, for
 *                   which every contribution swap is zero and the estimator is exact. */
typedef enum { SBH_COULOMB = 0, SBH_WINDING = 1, SBH_SMOOTHDIST = 2, SBH_AFFINE = 3 } sbh_kernel_kind;

typedef struct {
    int32_t kind;       /* sbh_kernel_kind */
    float softening;    /* SBH_COULOMB: epsilon >= 0 */
    float alpha;        /* SBH_SMOOTHDIST: alpha > 0 */
    float affine[3];    /* SBH_AFFINE: g */
} sbh_kernel;

/* Estimator options. Pass NULL for the defaults (all zero). */
typedef struct {
    int32_t sampling;   /* 0: child picked with probability m_c / m_T (aggregate mass);
                           1: |T_c| / |T| (uniform path index, the paper's Algorithm 2) */
    int32_t rr;         /* 0: Eq. 5; 1: no Russian roulette (p = 1); 2: fixed p = 1/2 */
    int32_t seed_mode;  /* 0: random stream keyed by query index; 1: every query uses index 0
                           (coherent across queries, the paper's identical per-warp seeding) */
    int32_t raw_sum;    /* SBH_SMOOTHDIST only: 1 returns the signed estimate of
                           sum_i m_i exp(-alpha |p_i - q|) itself (FP32; underflows to 0 beyond
                           alpha |p - q| ~ 87) instead of the distance -log(F) / alpha */
    int32_t schedule;   /* how sbh_eval maps work to threads (same result up to FP32 summation order):
                           0: a warp runs 32 queries, later path steps run as per-warp task batches;
                           1: one thread walks each query's paths on its own */
} sbh_eval_opts;

typedef struct sbh_tree sbh_tree;  /* opaque, library-owned */

/* Tree summary, filled by sbh_tree_info (host memory). `which`: 0 = the 64-ary tree used by the
 * estimator (per-dimension branching d = 4), 1 = the 8-ary tree used by Barnes-Hut (d = 2). */
typedef struct {
    int64_t n_points;
    int64_t n_nodes;
    int32_t leaf_size;
    int32_t has_normals;
    int32_t max_depth;       /* number of node generations below the root */
    int32_t reserved;
    int64_t first_sub;       /* subdomains (Sec. 3.3.1): node ids [first_sub, first_sub + n_sub) */
    int64_t n_sub;
    float lo[3];             /* root cube lower corner */
    float side;              /* root cube edge */
    float diam0;             /* |B| of the root cell: sqrt(3) * side, FP32 */
    float reserved_f;
} sbh_tree_meta;

/* Host copy of one tree for inspection. Every pointer may be NULL (skipped); arrays hold
 * n_points or n_nodes entries (x4 / x3 where stated). Node ids are breadth-first: the children
 * of node v are first_child[v] .. first_child[v] + nchild[v] - 1, in Morton order. */
typedef struct {
    int32_t* perm;         /* [n_points] input index of the i-th point in Morton order */
    uint64_t* code;        /* [n_points] sorted 60-bit Morton codes */
    int32_t* begin;        /* [n_nodes] first sorted point of the node */
    int32_t* end;          /* [n_nodes] one past the last sorted point */
    int32_t* first_child;  /* [n_nodes] -1 for a source point */
    int32_t* nchild;       /* [n_nodes] 0 for a source point */
    int32_t* level;        /* [n_nodes] cell level (|B| = diam0 * d^-level) */
    int32_t* parent;       /* [n_nodes] -1 for the root */
    float* com_mass;       /* [n_nodes][4] centre of mass x, y, z and aggregate mass (FP32) */
    double* com_mass64;    /* [n_nodes][4] the same in FP64, before rounding */
    float* dipole;         /* [n_nodes][3] sum_j m_j n_j (zeros without normals) */
    float* cdf;            /* [n_nodes] prefix fraction of the node's mass among its siblings */
    uint8_t* guide;        /* [n_nodes] the child pick's guide entry of the node's slot j among its
                            * parent's nc children: the number of the first nc - 1 siblings' cdf
                            * values <= ceil(j 2^24 / nc) 2^-24 (0 at the root) */
} sbh_tree_export_buffers;

/* Build the tree over n sources (Sec. 3.1).
 *   points   device [n][3]   finite
 *   weights  device [n]      masses m_i > 0 and finite (the child pick divides by them)
 *   normals  device [n][3] or NULL; required by SBH_WINDING evaluations
 *   n        1 <= n <= 2^28
 *   leaf_size 1 <= leaf_size <= 64: nodes with at most this many points are leaves
 * Builds the 64-ary estimator tree now; the 8-ary Barnes-Hut tree is built from the same sorted
 * codes on the first sbh_eval_bh call. The input buffers are not retained. On success *out owns
 * device memory until sbh_tree_free. Validation of the inputs synchronises the stream once; the
 * build itself is enqueued on `stream` and the call synchronises once more at its end. Returns
 * SBH_EINVAL for a bad size, NaN/Inf coordinates or a non-positive weight, SBH_ENOMEM when
 * device memory runs out, SBH_EUNSUPPORTED when more than 2^24 - 1 points share one cell of the
 * deepest level (2^-20 of the root cube per axis). */
SBH_API sbh_status sbh_build(const float* points, const float* weights, const float* normals, int64_t n,
                     int32_t leaf_size, void* stream, sbh_tree** out);

/* Most paths per subdomain any evaluation takes (the sample index is carried in 16 bits of a
 * task tag): every entry point taking samples_per_subdomain returns SBH_EINVAL beyond it. */
#define SBH_MAX_SAMPLES_PER_SUBDOMAIN (1 << 16)

/* Stochastic estimate of F at nq queries (Algorithm 2 with Eq. 5-7; Sec. 3.3.1 subdomains are
 * the root's children), S = samples_per_subdomain paths per subdomain, 1 <= S <=
 * SBH_MAX_SAMPLES_PER_SUBDOMAIN, random stream Philox4x32-10 keyed by `seed`: the decision at depth k
 * of a path uses the block counted by (query index, subdomain, sample, k - k mod 2), words 0 and 1
 * at even k, 2 and 3 at odd k (first word: child pick, second: roulette).
 *   queries device [nq][3]; out device [nq]: the estimate of F (the smooth distance for
 *   SBH_SMOOTHDIST). nq = 0 is a no-op. SBH_EINVAL if the kernel is SBH_WINDING and the tree
 *   has no normals, if S is out of range, or if an option is out of range. */
SBH_API sbh_status sbh_eval(const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                    int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                    float* out, void* stream);

/* Adjoint of sbh_eval with respect to the query positions, under the same random stream: the paths
 * and their weights 1 / (p(I in T) p(K >= k)) drawn exactly as sbh_eval draws them are held fixed
 * and every term m f(p, q) of Eq. 7 is replaced by its gradient in q. The weights are a valid
 * sampling of the same telescoping sums (Eq. 3-4), so E[grad] = grad F exactly; the decisions
 * themselves (Eq. 5 depends on q) are not differentiated.
 *   out  device [nq]: the estimate, equal to sbh_eval's up to FP32 summation order
 *   grad device [nq][3]: d out / d q. For SBH_SMOOTHDIST, d = -log(F)/alpha gives
 *        grad d = -grad F / (alpha F) (NaN where the estimate of F is <= 0); with opts->raw_sum
 *        both outputs are the sum F and its gradient. */
SBH_API sbh_status sbh_eval_grad(const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                                 int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                                 float* out, float* grad, void* stream);

/* One-shot build and evaluation from HOST buffers (the call for callers without device memory
 * of their own): points [n][3], weights [n], normals [n][3] or NULL, queries [nq][3] and out [nq] are
 * host memory. The points go up and the tree is built (as sbh_build) while the queries go up chunk
 * by chunk (chunk queries each, rounded up to a multiple of 32; 0 = half of nq from 2^22 on, else nq) on a copy
 * stream; each chunk is evaluated
 * (as sbh_eval, with the random stream of its place in the whole set, so out equals sbh_eval on
 * all queries bit for bit) as soon as it has landed, and its results come back on a second copy
 * stream while the next chunk runs. Page-locked host memory lets the copies overlap; pageable
 * memory works, without the overlap. The tree is freed before returning. Synchronises. */
SBH_API sbh_status sbh_solve_host(const float* points, const float* weights, const float* normals, int64_t n,
                                  int32_t leaf_size, const float* queries, int64_t nq, sbh_kernel kernel,
                                  int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                                  int64_t chunk, float* out, void* stream);

/* The work sbh_eval does for the same arguments, counted instead of evaluated: the same paths
 * are walked (same decisions) and no output is written. counts: device [4] unsigned 64-bit,
 * accumulated into (the caller zeroes them): [0] kernel terms evaluated (control variates, every
 * child of a swap and the swapped node), [1] node records read for those terms, [2] decisions
 * (child pick + roulette; one Philox block per two depths), [3] child prefix fractions read by the
 * picks.
 * Used to turn a measured time into achieved work for the roofline. */
SBH_API sbh_status sbh_eval_count(const sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                                  int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                                  unsigned long long* counts, void* stream);

/* Many independent problems in one launch: a plan holds n_sets (tree, queries, output) triples
 * sharing one kernel, S, seed and options; each launch runs every set in one persistent kernel
 * whose warps take 32-query tiles from a global counter. Set i's output equals sbh_eval on set i
 * alone (query indices are local to each set) up to FP32 summation order. Query sets may be empty.
 *   trees, queries, nq, outs: host arrays of n_sets entries (queries / outs are device buffers)
 * sbh_multi_plan_create copies the set descriptors to the device and synchronises `stream`; the
 * buffers must stay valid while the plan is used. sbh_multi_plan_launch enqueues a counter reset
 * and the kernel on `stream` and allocates nothing. */
typedef struct sbh_multi_plan sbh_multi_plan;
SBH_API sbh_status sbh_multi_plan_create(const sbh_tree* const* trees, const float* const* queries,
                                         const int64_t* nq, float* const* outs, int32_t n_sets, sbh_kernel kernel,
                                         int32_t samples_per_subdomain, uint64_t seed, const sbh_eval_opts* opts,
                                         void* stream, sbh_multi_plan** plan);
SBH_API sbh_status sbh_multi_plan_launch(const sbh_multi_plan* plan, void* stream);
/* Release a plan's device memory (NULL is a no-op); synchronises the device first. */
SBH_API void sbh_multi_plan_free(sbh_multi_plan* plan);

/* Learned child proposal (the paper samples the path index uniformly and leaves importance
 * sampling to future work, Sec. 3.3; this is the project's extension). A 6-32-32-1 ReLU network
 * (SBH_MLP_PARAMS values: W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3) scores each child c
 * of a node from query-relative features: ln(d_c/|B_c|), ln(m_c/m_T), ln(|B_c|/|B_T|),
 * ln(d_c/d_T), and for dipoles |N_c|/m_c and cos(p_c - q, N_c). The pick probability is
 * pi_c = 0.9 softmax(s)_c + 0.1 m_c/m_T (every pi_c > 0, so the estimator stays unbiased with
 * p(I in T) the product of the pi's); nodes with more than 64 children pick by mass. Inference
 * uses FP16 weights with FP32 accumulation; training keeps FP32 master weights (Adam). */
#define SBH_MLP_PARAMS 1313
typedef struct sbh_mlp sbh_mlp;
/* New network with He-scaled normal weights drawn from `seed`, zero biases. Synchronises. */
SBH_API sbh_status sbh_mlp_create(uint64_t seed, void* stream, sbh_mlp** out);
/* Host [SBH_MLP_PARAMS] FP32 weights in/out (the FP16 inference copy follows). Synchronise.
 * adam_step (may be NULL) receives the number of training steps taken, for resuming. */
SBH_API sbh_status sbh_mlp_set_weights(sbh_mlp* net, const float* host_weights, void* stream);
SBH_API sbh_status sbh_mlp_get_weights(const sbh_mlp* net, float* host_weights, int64_t* adam_step, void* stream);
/* The whole training state, for checkpoints: host [3 * SBH_MLP_PARAMS] FP32 = the master weights,
 * then Adam's first and second moment estimates, and the number of Adam steps taken. Restoring it
 * and training on the same queries continues the same optimisation (the training sets come from a
 * fixed random stream). Synchronise. */
SBH_API sbh_status sbh_mlp_get_state(const sbh_mlp* net, float* host_state, int64_t* adam_step, void* stream);
SBH_API sbh_status sbh_mlp_set_state(sbh_mlp* net, const float* host_state, int64_t adam_step, void* stream);
/* Scores of feature rows (device [n][6] -> device [n]) with the estimator's tensor-core scorer
 * (FP16 features, weights and hidden activations; FP32 accumulation). */
SBH_API sbh_status sbh_mlp_scores(const sbh_mlp* net, const float* feats, int64_t n, float* scores, void* stream);
/* Training loss and its gradient in the FP32 master weights: the mean over decision sets s (rows
 * offsets[s] .. offsets[s+1]-1, 2..64 rows each; device int64 offsets) of the cross-entropy between
 * softmax(scores) and the set's targets (>= 0) normalised to sum 1; a set whose targets are all 0
 * takes uniform targets. Only each set's ratios matter: targets at any scale, FP32 denormals
 * included, give the same loss up to their rounding. grad device [SBH_MLP_PARAMS], loss device [1]. */
SBH_API sbh_status sbh_mlp_loss_grad(sbh_mlp* net, const float* feats, const float* targets, const int64_t* offsets,
                                     int64_t n_sets, float* grad, float* loss, void* stream);
/* Training rows of explicit decision sets: set s is node set_node[s] at query set_query[s]
 * (device int32, queries device [.][3]); its rows set_offsets[s] .. set_offsets[s+1]-1 (device int64,
 * n_sets + 1 entries, set_offsets[s+1] - set_offsets[s] = the node's child count) receive each
 * child's features (feats, device [rows][6]) and target |R_c(q)|, the exact residual of the child's
 * subtree: the FP64 sum over its points minus its own centre-of-mass term (targets, device [rows]). */
SBH_API sbh_status sbh_mlp_dataset(const sbh_tree* tree, const float* queries, sbh_kernel kernel,
                                   const int32_t* set_query, const int32_t* set_node, const int64_t* set_offsets,
                                   int64_t n_sets, float* feats, float* targets, void* stream);
/* Train on the residuals the method itself produces: each of the nq training queries (device,
 * 1 <= nq <= 2^20) walks 4 paths of Algorithm 2 per subdomain (mass picks, Eq. 5 roulette, a
 * fixed training stream) and every node it decides at where the network is used (2..64 children,
 * d_T < near |B_T|; at most 4096 per query) becomes a decision set (sbh_mlp_dataset); at most 2^26
 * rows in all, else SBH_EINVAL; SBH_EUNSUPPORTED if there is none. Then `steps` full-batch Adam
 * steps with learning rate lr; losses (host [steps] or NULL) gets the loss before each step.
 * Synchronises. */
SBH_API sbh_status sbh_mlp_train(sbh_mlp* net, const sbh_tree* tree, const float* queries, int64_t nq,
                                 sbh_kernel kernel, float near, int32_t steps, float lr, float* losses, void* stream);
/* sbh_eval with the learned proposal, used at nodes with 2..64 children whose centre is nearer to
 * the query than `near` cell diagonals (d_T < near |B_T|, FP32; +inf: everywhere, 0: nowhere, which
 * is the mass-proportional estimator); elsewhere the pick is by mass. Same random stream layout;
 * opts->sampling must be 0. schedule 0 scores the children of a warp's gated decisions together on
 * the tensor cores (mma.sync m16n8k16: FP16 features and activations, FP16 weights, FP32
 * accumulation); schedule 1 is one thread per query with FP32 features and activations. */
SBH_API sbh_status sbh_eval_learned(const sbh_tree* tree, const sbh_mlp* net, const float* queries, int64_t nq,
                                    sbh_kernel kernel, int32_t samples_per_subdomain, uint64_t seed,
                                    const sbh_eval_opts* opts, float near, float* out, void* stream);
/* Release a network's device memory (NULL is a no-op); synchronises the device first. */
SBH_API void sbh_mlp_free(sbh_mlp* net);

/* Device memory. Every buffer the library holds (trees, scratch, plans, networks) comes from a
 * stream-ordered pool of its own, or, once set, from the caller's allocator: alloc(bytes, stream,
 * ctx) returns a device pointer aligned to 256 bytes that is usable in stream order on `stream`
 * (NULL: out of memory, reported as SBH_ENOMEM); free(ptr, stream, ctx) gives it back in stream
 * order. Both functions or neither (NULL, NULL: back to the pool); a block is always returned to
 * the allocator that gave it. Set the allocator while no library call is in flight. */
typedef void* (*sbh_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*sbh_free_fn)(void* ptr, void* stream, void* ctx);
SBH_API sbh_status sbh_set_allocator(sbh_alloc_fn alloc, sbh_free_fn free_fn, void* ctx);
/* Cap on the bytes the library holds at once (0: none). An allocation that would pass it fails
 * and the call returns SBH_ENOMEM with nothing leaked. */
SBH_API sbh_status sbh_set_memory_limit(uint64_t bytes);
/* Bytes the library holds now. */
SBH_API uint64_t sbh_memory_in_use(void);

/* Deterministic Barnes-Hut (Algorithm 1) on the 8-ary tree: a node is used whole when it is a
 * single point or ||q - p_a|| / |B_a| >= beta = 1 / theta (theta = 0 gives the exact sum).
 * warp_vote = 1 takes the decision jointly for the 32 queries of a warp (a node is opened when
 * any of them needs it); 0 decides per query, exactly as Algorithm 1. The first call builds the
 * 8-ary tree (enqueued on `stream`). */
SBH_API sbh_status sbh_eval_bh(sbh_tree* tree, const float* queries, int64_t nq, sbh_kernel kernel,
                       float theta, int32_t warp_vote, float* out, void* stream);

/* Exact sum (Eq. 1) by tiled brute force: every query against every source.
 *   points/weights/normals as in sbh_build (normals may be NULL unless SBH_WINDING);
 *   fp64_accum = 1 accumulates each tile's FP32 partial sum in FP64 (the error reference),
 *   0 keeps everything in FP32. out device [nq]. */
SBH_API sbh_status sbh_eval_brute(const float* points, const float* weights, const float* normals, int64_t n,
                          const float* queries, int64_t nq, sbh_kernel kernel, int32_t fp64_accum,
                          float* out, void* stream);

/* The exact sum and its gradient with respect to the query position (tiled brute force, FP32
 * per-tile partials added in FP64), in the conventions of sbh_eval_grad: out [nq] is F (the
 * distance d for the smooth distance), grad [nq][3] its gradient (grad d = -grad F / (alpha F)). */
SBH_API sbh_status sbh_eval_brute_grad(const float* points, const float* weights, const float* normals, int64_t n,
                                       const float* queries, int64_t nq, sbh_kernel kernel, float* out, float* grad,
                                       void* stream);

/* Tree summary (host struct). Synchronises the tree's build stream. which: 0 or 1 (see above);
 * SBH_EUNSUPPORTED when the 8-ary tree has not been built yet. */
SBH_API sbh_status sbh_tree_info(const sbh_tree* tree, int32_t which, sbh_tree_meta* meta);

/* Copy a tree to host buffers sized from sbh_tree_info. Synchronises. */
SBH_API sbh_status sbh_tree_export(const sbh_tree* tree, int32_t which, const sbh_tree_export_buffers* buf);

/* Release the tree's device memory (NULL is a no-op). Synchronises the tree's build stream. */
SBH_API void sbh_tree_free(sbh_tree* tree);

/* Message describing the calling thread's most recent failure ("" if none). */
SBH_API const char* sbh_last_error(void);

/* Allocation-free Morton ordering. The paper has no counterpart: this serves callers that cannot
 * allocate device memory -- real-time loops that cannot afford the implicit synchronisation of an
 * allocation, and applications that give the library a fixed memory budget and own every
 * allocation. It computes the same 60-bit codes and the same stable order sbh_build uses (what
 * sbh_tree_export reports as `code` and `perm`) without calling cudaMalloc, cudaFree or any
 * allocating routine.
 *   points  device [n][3], finite (not checked: a check would need a device-to-host read)
 *   codes   device [n] out: sorted codes;  perm device [n] out: input index of each sorted point
 *   n       1 <= n <= SBH_NOALLOC_MAX_POINTS; larger n returns SBH_EINVAL with a message
 * Scratch lives in one static device array of about 0.8 MB that every GPU loading the library
 * holds until the process exits; all calls share it and it keeps the last call's contents, so
 * calls whose GPU work overlaps (on different streams, or from different threads) race and must
 * be ordered by the caller. Every call looks up the array's device address in the current
 * device's context (cudaGetSymbolAddress, no allocation), so the address is never stale after a
 * device reset; the first call on a device also loads the library's device code there, so make
 * that first call before any stream capture. Enqueued on `stream`, no synchronisation. */
#define SBH_NOALLOC_MAX_POINTS 65536
SBH_API sbh_status sbh_morton_sort_noalloc(const float* points, int64_t n, uint64_t* codes, int32_t* perm,
                                           void* stream);

/* Number of CUDA kernels this library has launched in this process so far (host-side count). */
SBH_API unsigned long long sbh_kernel_launches(void);

/* SBH_VERSION of the loaded library. */
SBH_API int32_t sbh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SBH_H */

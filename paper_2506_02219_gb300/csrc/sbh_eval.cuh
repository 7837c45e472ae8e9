// sbh_eval.cuh -- launchers of the evaluation kernels (estimator, Barnes-Hut, brute force).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sbh_internal.cuh"

namespace sbh {

// host_ctrl: the host copy of the tree's control block (node counts per generation); qbase: the
// index of Q[0] in the caller's whole query set, so that a chunk draws the random stream the whole
// set would give it
cudaError_t launch_stoch_eval(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                              const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                              cudaStream_t s, int64_t qbase = 0);

cudaError_t launch_stoch_batched(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                                 const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                                 cudaStream_t s, int64_t qbase = 0);

// many sets in one launch: set_descs is a device array of n_sets descriptors filled with
// multi_fill_desc (host side) and copied to the device; counter is one device word
cudaError_t launch_stoch_multi(const void* set_descs, int n_sets, int64_t total_tiles, unsigned long long* counter,
                               const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, cudaStream_t s);
size_t multi_set_desc_bytes();
void multi_fill_desc(void* dst, const TreeView& T, const float* Q, float* out, int64_t nq, int64_t tile_begin);

cudaError_t launch_stoch_lane(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                              uint64_t seed, const sbh_eval_opts& o, float* out, cudaStream_t s);

// the estimator with the learned child proposal (mlp_half: device FP16 weights; the network is
// used at nodes nearer to the query than `near` cell diagonals); schedule 1 = one thread per query
cudaError_t launch_stoch_learned(const TreeView& T, const TreeCtrl& host_ctrl, const void* mlp_half, float near,
                                 const float* Q, int64_t nq, const KernelParams& kp, int S, uint64_t seed,
                                 const sbh_eval_opts& o, float* out, cudaStream_t s);
cudaError_t launch_stoch_batched_learned(const TreeView& T, const TreeCtrl& host_ctrl, const void* mlp_half,
                                         float near, const float* Q, int64_t nq, const KernelParams& kp, int S,
                                         uint64_t seed, const sbh_eval_opts& o, float* out, cudaStream_t s);

cudaError_t launch_stoch_count(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, int S,
                               uint64_t seed, const sbh_eval_opts& o, unsigned long long* counts, cudaStream_t s);

// the adjoint: schedule 0 = the warp-task kernel, 1 = one thread per query
cudaError_t launch_stoch_grad(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                              const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                              float* grad, cudaStream_t s);
cudaError_t launch_stoch_batched_grad(const TreeView& T, const TreeCtrl& host_ctrl, const float* Q, int64_t nq,
                                      const KernelParams& kp, int S, uint64_t seed, const sbh_eval_opts& o, float* out,
                                      float* grad, cudaStream_t s);

cudaError_t launch_bh_eval(const TreeView& T, const float* Q, int64_t nq, const KernelParams& kp, float beta,
                           int warp_vote, float* out, cudaStream_t s);

cudaError_t launch_brute(const float* P, const float* W, const float* N, int64_t n, const float* Q, int64_t nq,
                         const KernelParams& kp, int fp64_accum, float* out, cudaStream_t s);
cudaError_t launch_brute_grad(const float* P, const float* W, const float* N, int64_t n, const float* Q, int64_t nq,
                              const KernelParams& kp, float* out, float* grad, cudaStream_t s);

}  // namespace sbh

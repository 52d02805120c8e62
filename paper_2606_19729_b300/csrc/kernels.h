// Kernel argument blocks and launcher declarations (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace voila {

constexpr int kSimtRows = 32;
constexpr int kMaxPlanners = VOILA_MAX_PLANNERS;
constexpr int kSimtThreads = 256;

struct RolloutArgs {
  MlpDev g;
  MlpDev r;
  int reward_kind;
  int goal_dims;
  float goal[VOILA_MAX_GOAL];
  const float* particles;
  const float* actions;
  int N, K, H, d_s, d_a, d_omega;
  double gamma;
  uint32_t key0, key1, planner;
  uint32_t n_off, k_off;  // a shard's offsets in the whole problem: noise counters (n + n_off, k + k_off, t)
  double* G;  // [K][N]
  int ld;     // shared-memory row stride (floats)
};

struct BeliefArgs {
  MlpDev g;
  MlpDev l;
  int lik_kind;
  float sigma;
  const float* particles;
  const float* action;
  const float* obs;
  int N, d_s, d_a, d_o, d_omega;
  uint32_t key0, key1, planner, step;
  float* s_prop;  // [N][d_s]
  double* ell;    // [N]
  int ld;
};

// Resampling runs in one CTA up to kResampleSingleCta particles, above that
// in CTAs of kResampleSegElems particles each (at most kResampleMaxSegs).
constexpr int kResampleSingleCta = 2048;
constexpr int kResampleSegElems = 4096;
constexpr int kResampleMaxSegs = 64;

struct ResampleArgs {
  const double* ell;
  const double* logw;
  const float* s_prop;
  int N, d_s;
  double lambda;
  uint32_t key0, key1, planner, step;
  double* C;          // [N] workspace
  double* part;       // [5][kResampleMaxSegs] segment partials (N > kResampleSingleCta)
  double* w_out;      // [N] or null
  int32_t* idx_out;   // [N] or null
  float* particles_out;
  double* logZ_out;
  double* ess_out;
  WsHeader* hdr;
};

struct FwdArgs {
  MlpDev m;
  const float* X;   // plain form, or null for the seeded form
  const float* S;
  const float* A;
  int a_stride;
  int B, d_s, d_a, d_omega;
  uint32_t key0, key1, planner, step, stream_id;
  float* Y;
  int ld;
};

size_t rollout_simt_smem(int ld);
size_t belief_propose_smem(int ld);
cudaError_t launch_rollout_simt(const RolloutArgs& a, cudaStream_t s);
cudaError_t launch_belief_propose(const BeliefArgs& a, cudaStream_t s);
cudaError_t launch_belief_resample(const ResampleArgs& a, cudaStream_t s);
cudaError_t launch_mlp_fwd(const FwdArgs& a, cudaStream_t s);
// J_k = sum_n w_n G[k][n] (w == NULL: the uniform weight 1 / N_total); a
// non-finite J_k sets VOILA_ERR_NONFINITE in *hdr (where = kWhereReturns).
constexpr int32_t kWhereReturns = 70;
cudaError_t launch_reduce_returns(const double* G, const double* w, int N, int N_total, int K, double* J,
                                  int32_t* best_k, WsHeader* hdr, cudaStream_t s);
// Returns of P planners in one launch: J_q[k] = sum_n w_q[n] G_q[k][n], then argmax per planner.
struct BatchedReduceArgs {
  const double* G[kMaxPlanners];
  const double* w[kMaxPlanners];
  double* J[kMaxPlanners];
  int32_t* best[kMaxPlanners];
  int N[kMaxPlanners], K[kMaxPlanners];
  long long k_end[kMaxPlanners];  // inclusive prefix sum of K
  int P;
  WsHeader* hdr;  // status word of the call's workspace (non-finite J_k)
};
cudaError_t launch_reduce_returns_batched(const BatchedReduceArgs& a, cudaStream_t s);

cudaError_t launch_philox_fill(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t* out, long long n, cudaStream_t s);
cudaError_t launch_normal_fill(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2,
                               uint32_t stream, uint32_t planner, int dim, float* out,
                               long long n, cudaStream_t s);

}  // namespace voila

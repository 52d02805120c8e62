// Tensor-core (tcgen05) rollout: host-side entry points used by the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/voila.h"
#include "kernels.h"

namespace voila {

// Scratch bytes (packed, swizzled BF16 weight stream) the tensor-core
// rollout needs inside the caller's workspace.
size_t tc_rollout_scratch_bytes(const voila_mlp* g_T, const voila_reward* R);

// One planning problem of a batched tensor-core rollout.
struct TcProblem {
  const float* particles;  // [N][d_s]
  const float* actions;    // [K][H][d_a]
  double* G;               // [K][N]
  int N, K, H;
  uint32_t planner;
  uint32_t n_off = 0, k_off = 0;  // offsets of a shard's particles and sequences in the whole problem
};

// Tile-shape and work-order flags of tc_rollout_batched.
constexpr int kShapeQueue = 1;    // work items claimed from a global counter (else c, c + clusters, ...)
constexpr int kShapeOneTile = 2;  // one 128-row tile per CTA and item, scalar outputs as MMAs (else two
                                  // tiles per CTA in flight, scalar outputs fused into the epilogue)
// The work-item counter's byte offset in the workspace header.
constexpr size_t kQueueCounterOffset = 64;

// Launches one persistent BF16 tcgen05 rollout over P problems sharing the
// MLPs. order = 1 sorts the work by descending horizon (longest first);
// max_clusters > 0 caps the number of CTA pairs; shape: kShape* flags.
voila_status tc_rollout_batched(const voila_mlp* g_T, const voila_reward* R, const TcProblem* probs, int P,
                                int d_s, int d_a, int d_omega, double gamma, uint32_t key0, uint32_t key1,
                                int order, int max_clusters, int shape, WsHeader* hdr, void* scratch,
                                cudaStream_t s);

// Launches the BF16 tcgen05 rollout; writes G [K][N]. Returns
// VOILA_ERR_UNSUPPORTED for shapes the kernel does not cover.
voila_status tc_rollout(const voila_mlp* g_T, const voila_reward* R, const RolloutArgs& a,
                        WsHeader* hdr, void* scratch, cudaStream_t s);

// DDIM teacher sampling on the tensor cores (BF16 teacher 82 -> 512 x L -> 8,
// s 8, a 2, x 8, embedding 64): whether the shape is covered, the scratch it
// needs (packed weights, biases, step embeddings; 1024-byte aligned), and the
// launch. cx[t], cv[t]: x <- cx x + cv v at launch step t (diffusion step
// T-1-t); freq[i], i < 32: embedding frequencies.
bool tc_ddim_supported(const voila_mlp* teacher, int d_s, int d_a, int d_x, int emb_dim);
size_t tc_ddim_scratch_bytes(const voila_mlp* teacher, int T);
voila_status tc_ddim_sample(const voila_mlp* teacher, const float* S, const float* A, const float* omega, int B,
                            int T, const double* cx, const double* cv, const double* freq, float* Y, WsHeader* hdr,
                            void* scratch, cudaStream_t s);

// Likelihood on all B x B pairs on the tensor cores (BF16 likelihood MLP
// 16 -> 256 x L -> 1, s' 8, a 2, o 6): out[i * B + j] = l([s'_i; a_i; o_j]).
bool tc_pairs_supported(const voila_mlp* ell, int d_s, int d_a, int d_o);
size_t tc_pairs_scratch_bytes(const voila_mlp* ell);
voila_status tc_likelihood_pairs(const voila_mlp* ell, const float* S, const float* A, const float* Ob, long long B,
                                 float* out, WsHeader* hdr, void* scratch, cudaStream_t s);
// Gather form: out[m] = l([S[m]; A[node[m]]; Ob[node[m] * C_max + branch[m]]]) for m < M
// (node outside [0, n_nodes): zero input row).
voila_status tc_likelihood_rows(const voila_mlp* ell, const float* S, const float* A, const float* Ob, long long M,
                                const int32_t* node, const int32_t* branch, int n_nodes, int C_max, float* out,
                                WsHeader* hdr, void* scratch, cudaStream_t s);

// Observation sampler of progressive widening on the tensor cores (BF16 f_Z
// 18 -> 256 x L -> d_o, s' 8, a 2, omega 8): for the first *count entries m of
// list, obs[node[m] * C_max + branch[m]][0 .. d_o) = f_Z([S[m]; act[node[m]];
// omega_Z(m)]), omega_Z the normals of stream VOILA_STREAM_OBS_OMEGA at counter
// (m, 0, step); at most M rows (the count is read on the device).
bool tc_observe_supported(const voila_mlp* g_Z, int d_s, int d_a, int d_omega, int d_o);
size_t tc_observe_scratch_bytes(const voila_mlp* g_Z);
voila_status tc_observe_rows(const voila_mlp* g_Z, const float* S, const float* act, const int32_t* list,
                             const int32_t* count, long long M, const int32_t* node, const int32_t* branch,
                             int n_nodes, int C_max, float* obs, int d_o, uint32_t key0, uint32_t key1,
                             uint32_t step, uint32_t planner, WsHeader* hdr, void* scratch, cudaStream_t s);

// Belief proposal on the tensor cores (generator 18 -> 256 x L -> 8 and
// likelihood 16 -> 256 x L -> 1, each BF16 or FP8 e4m3 with per-channel
// scales on its hidden layers): s_prop[i] = g_T([particles[i]; action;
// omega(i)]), omega the normals of stream VOILA_STREAM_BELIEF_OMEGA at counter
// (i, 0, step); ell_out[i] = l([s_prop[i]; action; obs]) (FP64 store).
bool tc_propose_supported(const voila_mlp* g_T, const voila_mlp* ell, int d_s, int d_a, int d_omega, int d_o);
size_t tc_propose_scratch_bytes(const voila_mlp* g_T, const voila_mlp* ell);
voila_status tc_belief_propose(const voila_mlp* g_T, const voila_mlp* ell, const float* particles, const float* action,
                               const float* obs, long long N, uint32_t key0, uint32_t key1, uint32_t step,
                               uint32_t planner, float* s_prop, double* ell_out, WsHeader* hdr, void* scratch,
                               cudaStream_t s);

// Self-test of the bounded waits (see voila_selftest_wait_timeout).
cudaError_t launch_wait_timeout_selftest(WsHeader* hdr, long long limit, cudaStream_t s);

}  // namespace voila

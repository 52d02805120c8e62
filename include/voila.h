/*
 * voila.h - C-ABI of the VOiLA planning-loop hot path on B300 (sm_103a).
 *
 * VOiLA (Vectorized Online planning wIth Learned diffusion model for POMDP
 * Agents) plans with a distilled feed-forward transition generator
 * s' = f_T(s, a, omega_T) (Eq. 2), an observation sampler z = f_Z(s', a, omega_Z)
 * (Eq. 5) and an unnormalised likelihood l(s', a, o) whose tempered
 * exponential exp(l / lambda) weights particles (Sec. 4.2.3). This library
 * runs the data-parallel part of that loop:
 *
 *   voila_rollout        Monte-Carlo rollout of N particles x K action
 *                        sequences x H steps and the per-sequence return
 *                        reduction (value definition of Sec. 2.1; the
 *                        Monte-Carlo estimate of R(b, a) in Eq. 1, Sec. 2.2).
 *   voila_belief_update  one SIR particle-filter step: propose with f_T,
 *                        weight with l, normalise, resample systematically
 *                        (Sec. 3, belief operator of Sec. 2.1).
 *   voila_generator_fwd  batched forward of a generator MLP (Eq. 2 / Eq. 5).
 *   voila_generator_bwd  its hand-written backward, and voila_ddim_sample the
 *                        teacher sampler, for the distillation step (Eq. 3).
 *   voila_philox_fill    raw Philox4x32-10 words, for checking the noise stream.
 *
 * Conventions shared by every call:
 *  - Every array argument is DEVICE memory owned by the caller unless the
 *    comment says "host". The library never allocates on these paths: it uses
 *    the caller's workspace, whose size the *_workspace_size calls return.
 *  - Calls are asynchronous on `stream`. The returned status reports argument
 *    validation and kernel launch only. Conditions found on the device
 *    (non-finite or all-zero weights, a wait that timed out) are written to a
 *    status word inside the workspace; voila_workspace_status() reads it.
 *  - Outputs are undefined when a call or its device status is not VOILA_OK.
 *  - Calls with distinct workspaces may run concurrently.
 *  - Layouts are row-major and densely packed.
 *
 * Random numbers: omega is drawn in-kernel by Philox4x32-10 (Salmon et al.,
 * SC'11) with key = (seed & 0xffffffff, seed >> 32) and counter
 * (c0, c1, c2, c3) = (n, k, t, stream << 28 | planner << 12 | block); each
 * block gives four uniforms u = (2 * (x >> 9) + 1) * 2^-24 and four normals
 * by Box-Muller, (r cos 2 pi u1, r sin 2 pi u1), r = sqrt(-2 ln u0), then
 * (r' cos 2 pi u3, r' sin 2 pi u3), r' = sqrt(-2 ln u2).
 * Streams: 0 rollout omega_T(n, k, t); 1 belief-update omega_T(i, 0, step);
 * 2 resampling offset (0, 0, step); 3 observation omega_Z.
 */
#ifndef VOILA_H_
#define VOILA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* voila_stream_t;

typedef enum {
  VOILA_OK = 0,
  VOILA_ERR_ARG = -1,          /* null pointer, bad enum, negative size */
  VOILA_ERR_SHAPE = -2,        /* inconsistent dimensions between arguments */
  VOILA_ERR_CUDA = -3,         /* a CUDA runtime call or launch failed */
  VOILA_ERR_NONFINITE = -4,    /* device status: a log-weight was NaN or +inf */
  VOILA_ERR_DEGENERATE = -5,   /* device status: every log-weight was -inf */
  VOILA_ERR_TIMEOUT = -6,      /* device status: a bounded wait ran out */
  VOILA_ERR_UNSUPPORTED = -7,  /* valid request the library has no kernel for */
  VOILA_ERR_WORKSPACE = -8     /* workspace missing, misaligned or too small */
} voila_status;

enum { VOILA_ACT_IDENTITY = 0, VOILA_ACT_TANH = 1, VOILA_ACT_SILU = 2 };
enum { VOILA_FP32 = 0, VOILA_BF16 = 1, VOILA_FP8E4M3 = 2 };
enum { VOILA_REWARD_GOAL = 0, VOILA_REWARD_MLP = 1 };
enum { VOILA_LIK_MLP = 0, VOILA_LIK_GAUSSIAN = 1 };
enum {
  VOILA_STREAM_ROLLOUT_OMEGA = 0,
  VOILA_STREAM_BELIEF_OMEGA = 1,
  VOILA_STREAM_RESAMPLE = 2,
  VOILA_STREAM_OBS_OMEGA = 3,
  VOILA_STREAM_PW_BRANCH = 6   /* progressive widening: choice of an existing branch */
};

#define VOILA_MAX_LAYERS 8
#define VOILA_MAX_WIDTH 512
#define VOILA_MAX_GOAL 4
#define VOILA_MAX_PLANNERS 64

/*
 * A feed-forward MLP y = L_n(act(... act(L_1(x)))), L_l(h) = h W_l^T + b_l,
 * with a linear last layer: the distilled generator form of Eq. 2 and the
 * model shapes of Sec. 5.2 (widths up to VOILA_MAX_WIDTH).
 *   W[l]  device, row-major [dims[l+1]][dims[l]] ("[out][in]"), element type
 *         float for VOILA_FP32, __nv_bfloat16 for VOILA_BF16 and VOILA_FP8E4M3.
 *         The FP8 form (rollout and tensor-core belief proposal) quantises every
 *         hidden-to-hidden layer to E4M3 with per-output-channel FP32 scales
 *         max_k|W[n][k]| / 448 and runs it on E4M3 activations (FP32
 *         accumulation); first and last layers stay BF16. It takes SiLU MLPs
 *         (act = VOILA_ACT_SILU); other activations return VOILA_ERR_UNSUPPORTED.
 *   b[l]  device, float [dims[l+1]].
 *   w_scale[l]  reserved, NULL (the FP8 form computes its channel scales).
 * The struct itself is read on the host during the call and may be freed
 * after the call returns.
 */
typedef struct {
  int32_t n_layers;                       /* 1 .. VOILA_MAX_LAYERS */
  int32_t dims[VOILA_MAX_LAYERS + 1];     /* dims[0] input width, dims[n_layers] output width */
  int32_t act;                            /* VOILA_ACT_*, applied after every layer but the last */
  int32_t prec;                           /* VOILA_FP32, VOILA_BF16 or VOILA_FP8E4M3 */
  const void* W[VOILA_MAX_LAYERS];
  const float* b[VOILA_MAX_LAYERS];
  const float* w_scale[VOILA_MAX_LAYERS];
} voila_mlp;

/*
 * Reward head R(s_{t+1}, a_t) (reward function of the POMDP tuple, Sec. 2.1;
 * the post-transition state is the one scored).
 *   GOAL: r = -sum_{d < goal_dims} (s[d] - goal[d])^2, goal given on the host.
 *   MLP:  r = R([s; a]) with mlp->dims[0] == d_s + d_a and a scalar output.
 */
typedef struct {
  int32_t kind;
  int32_t goal_dims;
  float goal[VOILA_MAX_GOAL];
  const voila_mlp* mlp;
} voila_reward;

/*
 * Likelihood l(s', a, o) (Sec. 4.2.3).
 *   MLP:      l = mlp([s'; a; o]), mlp->dims[0] == d_s + d_a + d_o, scalar output.
 *   GAUSSIAN: l = -||o - s'[:d_o]||^2 / (2 sigma^2), an analytic test kind.
 */
typedef struct {
  int32_t kind;
  float sigma;
  const voila_mlp* mlp;
} voila_likelihood;

/* Status word written by kernels into a workspace; blocks on `stream`. */
voila_status voila_workspace_status(const void* workspace, voila_stream_t stream);

/* Human-readable name of a status code (static string). */
const char* voila_status_string(voila_status s);

/*
 * Self-test of the device-side failure detection: one thread waits on an
 * mbarrier that nothing arrives on, through the bounded wait every
 * tensor-core kernel uses, and gives up after limit_cycles SM clock cycles
 * (0 .. 4e9; the kernels themselves use ~4e9, about 2 s), recording
 * VOILA_ERR_TIMEOUT in the status word of `workspace` (device, 256-byte
 * aligned, at least 256 bytes; its status word is cleared first). The wait
 * ends by itself and the context stays usable: read the result with
 * voila_workspace_status. The paper has no counterpart.
 */
voila_status voila_selftest_wait_timeout(void* workspace, int64_t limit_cycles, voila_stream_t stream);

/*
 * Workspace bytes for voila_rollout with these sizes (host call, no device work).
 */
voila_status voila_rollout_workspace_size(const voila_mlp* g_T, const voila_reward* R,
                                          int32_t N, int32_t K, int32_t H, size_t* bytes);

/*
 * Batched Monte-Carlo rollout (value definition, Sec. 2.1; R(b, a) estimate
 * of Eq. 1, Sec. 2.2; generator of Eq. 2).
 * For every particle n < N and action sequence k < K:
 *   s_0 = particles[n];  for t < H:
 *     s_{t+1} = g_T([s_t; actions[k][t]; omega_T(n, k, t)])
 *     G[k][n] += gamma^t * R(s_{t+1}, actions[k][t])
 *   J[k] = sum_n w[n] * G[k][n]   (w = 1/N when w == NULL)
 *   best_k = argmax_k J[k], lowest index on ties.
 * Arguments:
 *   particles [N][d_s] float; w [N] double or NULL; actions [K][H][d_a] float;
 *   g_T->dims[0] == d_s + d_a + d_omega, g_T output width == d_s;
 *   J [K] double (required); G [K][N] double or NULL; best_k [1] int32 or NULL.
 *   planner_id < 65536 selects an independent noise stream per planner.
 * Precision forms: VOILA_FP32 runs on CUDA cores in FP32; VOILA_BF16 runs on
 * the tcgen05 tensor cores (BF16 operands, FP32 accumulation in TMEM);
 * VOILA_FP8E4M3 runs its hidden layers as E4M3 tensor-core MMAs with
 * per-channel scales (see voila_mlp).
 * Returns are accumulated in FP64 in both forms.
 * N == 0 or K == 0 is a no-op; H == 0 gives zero returns.
 * Device status (voila_workspace_status(workspace), cleared by the call):
 * VOILA_ERR_NONFINITE if some J[k] is NaN or infinite (a non-finite weight,
 * particle, action or model value reached it; J and G are still written),
 * VOILA_ERR_TIMEOUT if a bounded wait of the tensor-core kernel ran out.
 */
voila_status voila_rollout(const voila_mlp* g_T, const voila_reward* R,
                           const float* particles, const double* w, int32_t N, int32_t d_s,
                           const float* actions, int32_t K, int32_t H, int32_t d_a,
                           int32_t d_omega, double gamma, uint64_t seed, uint32_t planner_id,
                           double* J, double* G, int32_t* best_k,
                           void* workspace, size_t ws_bytes, voila_stream_t stream);

/*
 * One shard of a rollout split over several calls or GPUs by particles and/or
 * by action sequences. The simulations of different (particle, sequence)
 * pairs are independent (Sec. 2.2: the planner runs them side by side), so a
 * shard computes exactly the rows of the whole problem that it holds.
 *   particles [N][d_s]: particles n_offset .. n_offset + N - 1 of the whole
 *     belief of N_total particles; w [N] their weights or NULL (1 / N_total each);
 *   actions [K][H][d_a]: sequences k_offset .. k_offset + K - 1 of the whole set;
 *   row (n, k) draws omega_T at counter (n + n_offset, k + k_offset, t), so G of
 *   a shard equals the matching block of the unsharded call's G bit for bit;
 *   J [K] (required): the shard's partial value J_k = sum over its particles of
 *     w_n G[k][n]. With all particles (n_offset = 0, N = N_total) this is the
 *     unsharded J of those sequences, bit for bit. Over particle shards the full
 *     J_k is the sum of the shards' partials (FP64; equal to the unsharded J up
 *     to the order of the additions);
 *   best_k [1] or NULL: argmax over this shard's J (meaningful when the shard
 *     holds every particle).
 * Requires 0 <= n_offset, n_offset + N <= N_total, 0 <= k_offset; the other
 * arguments, the workspace (voila_rollout_workspace_size(g_T, R, N, K, H)) and
 * the errors are those of voila_rollout, which is this call with n_offset =
 * k_offset = 0 and N_total = N.
 */
voila_status voila_rollout_shard(const voila_mlp* g_T, const voila_reward* R, const float* particles,
                                 const double* w, int32_t N, int32_t n_offset, int32_t N_total,
                                 int32_t d_s, const float* actions, int32_t K, int32_t k_offset,
                                 int32_t H, int32_t d_a, int32_t d_omega, double gamma, uint64_t seed,
                                 uint32_t planner_id, double* J, double* G, int32_t* best_k,
                                 void* workspace, size_t ws_bytes, voila_stream_t stream);

/*
 * One independent planning problem of a batched rollout: its own belief
 * (particles, optional weights), action sequences, horizon and noise stream,
 * sharing the generator and reward of the call. All pointers are device
 * memory; the array of voila_planner itself is host memory.
 */
typedef struct {
  const float* particles;  /* [N][d_s] */
  const double* w;         /* [N] or NULL (uniform 1/N) */
  const float* actions;    /* [K][H][d_a] */
  int32_t N, K, H;
  uint32_t planner_id;     /* < 65536, selects the noise stream */
  double* J;               /* [K], required */
  double* G;               /* [K][N] or NULL */
  int32_t* best_k;         /* [1] or NULL */
} voila_planner;

/* Schedules of voila_rollout_batched: bit 0 = order work by descending
 * horizon (longest first); bit 1 = work items claimed from an atomic counter
 * by whichever CTA pair is ready (else pair c takes items c, c + pairs, ...);
 * bit 2 = the one-tile shape: one 128-row tile per CTA and work item, reward
 * output as an MMA (else two tiles per CTA in flight and the scalar reward
 * output computed in the epilogue; the two shapes round the reward
 * differently, both within the BF16 tolerance; not available for FP8 MLPs of
 * the mid-size dimensions: VOILA_ERR_UNSUPPORTED); bits 8-15 = cap on CTA
 * pairs (0 = all resident). */
#define VOILA_SCHED_LONGEST_FIRST 1
#define VOILA_SCHED_QUEUE 2
#define VOILA_SCHED_ONE_TILE 4
#define VOILA_SCHED_CLUSTERS(n) ((n) << 8)

/* Workspace bytes for voila_rollout_batched (host call, no device work). */
voila_status voila_rollout_batched_workspace_size(const voila_mlp* g_T, const voila_reward* R,
                                                  const voila_planner* planners, int32_t P,
                                                  size_t* bytes);

/*
 * Many independent planners (uneven N, K, H) in one launch: the rollout of
 * voila_rollout for every planner, with the same generator, reward, gamma and
 * seed (the planner id separates the noise streams), as one persistent
 * tensor-core launch over all planners' work plus one reduction launch. The
 * call issues no host synchronisation and can be captured in a CUDA graph
 * once voila_rollout_batched (or voila_rollout) has run outside capture on
 * the device. P <= VOILA_MAX_PLANNERS. BF16 runs batched; FP32 runs the
 * planners one after another on CUDA cores.
 * Batched execution of VOPP's many simulations (Sec. 2.2, Sec. 4.3), with the
 * per-planner semantics of voila_rollout. One device status word for the
 * call: VOILA_ERR_NONFINITE if any planner's J has a NaN or infinite entry,
 * VOILA_ERR_TIMEOUT as for voila_rollout.
 */
voila_status voila_rollout_batched(const voila_mlp* g_T, const voila_reward* R,
                                   const voila_planner* planners, int32_t P, int32_t d_s,
                                   int32_t d_a, int32_t d_omega, double gamma, uint64_t seed,
                                   int32_t schedule, void* workspace, size_t ws_bytes,
                                   voila_stream_t stream);

/*
 * Autotuner for voila_rollout_batched: runs each candidate schedule (tile
 * shape: two tiles in flight with the fused reward output or one tile with the
 * reward output as an MMA; work order: static longest-first, table order or
 * the atomic queue; number of CTA pairs) on these inputs, times it with CUDA
 * events and writes the fastest to *best_schedule (host int32) and its time to
 * *best_ms (or NULL); a queue schedule within 0.5 % of its faster static twin
 * is taken instead (it balances CTA pairs that run at slightly different
 * speeds, which one timing per candidate cannot resolve). Candidates a form
 * has no kernel for are skipped.
 * Synchronises `stream`; do not call it during stream capture. Outputs are
 * left as the last candidate's: schedules of one tile shape compute the same
 * bits; the two shapes differ in the reward output's rounding (within the
 * BF16 tolerance), so pass the returned schedule to voila_rollout_batched to
 * reproduce a result.
 */
voila_status voila_rollout_batched_autotune(const voila_mlp* g_T, const voila_reward* R,
                                            const voila_planner* planners, int32_t P,
                                            int32_t d_s, int32_t d_a, int32_t d_omega,
                                            double gamma, uint64_t seed, void* workspace,
                                            size_t ws_bytes, int32_t* best_schedule,
                                            float* best_ms, voila_stream_t stream);

/* Workspace bytes for voila_belief_update. */
voila_status voila_belief_update_workspace_size(const voila_mlp* g_T, const voila_likelihood* ell,
                                                int32_t N, size_t* bytes);

/*
 * One SIR particle-filter step (Sec. 3; belief operator of Sec. 2.1; weights
 * exp(l / lambda), Sec. 4.2.3):
 *   s'_i = g_T([particles_in[i]; action; omega_T(i, 0, step)])
 *   lw_i = logw_in[i] + l(s'_i, action, obs) / lambda    (logw_in NULL = 0)
 *   w_i  = exp(lw_i - max lw) / sum_j exp(lw_j - max lw)
 *   q_i  = rn(w_i * 2^52) * 2^-52; C = inclusive FP64 prefix sum of q (exact)
 *   u0   = 53-bit uniform from stream 2 at counter (0, 0, step)
 *   idx_j = min{i : C_i > ((u0 + j) * C_{N-1}) / N}, or N-1 if none
 *   particles_out[j] = s'_{idx_j}
 * Arguments: particles_in [N][d_s] float; logw_in [N] double or NULL;
 *   action [d_a] and obs [d_o] float (device); particles_out [N][d_s] float;
 *   idx_out [N] int32 or NULL; w_out [N] double (the q_i) or NULL;
 *   logZ_out [1] double = log sum_i exp(lw_i), or NULL; ess_out [1] double =
 *   1 / sum_i q_i^2, or NULL. particles_out must not alias particles_in.
 * Precision: FP32 and BF16 MLPs of any supported shape run on the CUDA cores;
 * an MLP likelihood with g_T 18 -> 256 x L -> 8 and l 16 -> 256 x L -> 1
 * (d_s 8, d_a 2, d_omega 8, d_o 6), each BF16 or FP8 e4m3 (per-channel
 * scales on the hidden layers), runs on the tensor cores, proposal and
 * likelihood in one kernel. FP8 e4m3 MLPs of other shapes (or with the
 * Gaussian likelihood) return VOILA_ERR_UNSUPPORTED before any device work.
 * Device status: VOILA_ERR_NONFINITE if some lw_i is NaN or +inf,
 * VOILA_ERR_DEGENERATE if all are -inf; VOILA_ERR_TIMEOUT if a wait of the
 * tensor-core kernel ran out (the kernel then returns early). N <= 262144.
 */
voila_status voila_belief_update(const voila_mlp* g_T, const voila_likelihood* ell,
                                 const float* particles_in, const double* logw_in,
                                 int32_t N, int32_t d_s, const float* action, const float* obs,
                                 int32_t d_a, int32_t d_o, int32_t d_omega, float lambda,
                                 uint64_t seed, uint32_t step, uint32_t planner_id,
                                 float* particles_out, int32_t* idx_out, double* w_out,
                                 double* logZ_out, double* ess_out,
                                 void* workspace, size_t ws_bytes, voila_stream_t stream);

/* Size of the fixed device scratch behind voila_belief_update_noalloc (4 MiB). */
#define VOILA_NOALLOC_SCRATCH_BYTES (4u << 20)

/*
 * voila_belief_update for callers that cannot allocate device memory: a
 * control loop that forbids allocation once it runs (an allocation can block
 * or fail at an arbitrary moment), a plug-in inside a framework that owns all
 * device memory, or a caller with no way to size and keep a workspace. The
 * paper has no counterpart; this is a convenience of this library.
 *
 * Same arguments and results as voila_belief_update, without the workspace:
 * the scratch is one array of VOILA_NOALLOC_SCRATCH_BYTES compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits. N is accepted while voila_belief_update_workspace_size(g_T, ell, N)
 * fits in that array (N <= 87320 for d_s = 8 with FP32 MLPs); larger N returns
 * VOILA_ERR_WORKSPACE before any device work.
 *   status_out  device int32 or NULL: receives the device-side status
 *               (VOILA_OK, VOILA_ERR_NONFINITE, VOILA_ERR_DEGENERATE, or
 *               VOILA_ERR_TIMEOUT if a bounded wait of the tensor-core
 *               proposal expired), asynchronously on `stream`.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture. The address
 * is looked up again when the device's context has changed (after
 * cudaDeviceReset the library's device image, and the array, are loaded anew).
 * The call runs on the current device, so `stream` must belong to it.
 * All calls share the one array and it keeps the last call's contents: calls
 * whose work overlaps on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.
 */
voila_status voila_belief_update_noalloc(const voila_mlp* g_T, const voila_likelihood* ell,
                                         const float* particles_in, const double* logw_in,
                                         int32_t N, int32_t d_s, const float* action,
                                         const float* obs, int32_t d_a, int32_t d_o,
                                         int32_t d_omega, float lambda, uint64_t seed,
                                         uint32_t step, uint32_t planner_id, float* particles_out,
                                         int32_t* idx_out, double* w_out, double* logZ_out,
                                         double* ess_out, int32_t* status_out,
                                         voila_stream_t stream);

/*
 * Batched MLP forward Y = mlp(X) (Eq. 2 / Eq. 5 generator form).
 *   X [B][dims[0]] float, Y [B][dims[n_layers]] float. No workspace.
 */
voila_status voila_generator_fwd(const voila_mlp* mlp, const float* X, int32_t B, float* Y,
                                 voila_stream_t stream);

/*
 * Seeded sampler form of Eq. 2 / Eq. 5: Y[i] = mlp([S[i]; A[i]; omega(i, 0, step)])
 * with omega from Philox stream `stream_id`. S [B][d_s], A [B][d_a] float;
 * A may have row stride 0 (a_stride = 0: one action for every row).
 */
voila_status voila_generator_fwd_seeded(const voila_mlp* mlp, const float* S, const float* A,
                                        int32_t a_stride, int32_t B, int32_t d_s, int32_t d_a,
                                        int32_t d_omega, uint64_t seed, uint32_t stream_id,
                                        uint32_t step, uint32_t planner_id, float* Y,
                                        voila_stream_t stream);

/*
 * Training forward of a generator MLP, the first half of the distillation step
 * (Eq. 3): Y = mlp(X) as voila_generator_fwd, and the pre-activations of every
 * hidden layer kept for voila_generator_bwd.
 *   X [B][dims[0]], Y [B][dims[L]] float (device), L = n_layers.
 *   saved  [B][dims[1] + ... + dims[L-1]] float (device) or NULL: row b holds
 *          z_1(b), ..., z_{L-1}(b) side by side, z_l = h_{l-1} W_l^T + b_l.
 *   workspace  device, >= 2 * B * max_l dims[l] * 4 bytes (caller-owned).
 * mlp->prec FP32 or BF16 (BF16 weights, FP32 arithmetic); FP8 returns
 * VOILA_ERR_UNSUPPORTED. B = 0 returns VOILA_OK with no launch.
 */
voila_status voila_generator_fwd_train(const voila_mlp* mlp, const float* X, int32_t B, float* Y,
                                       float* saved, void* workspace, size_t ws_bytes,
                                       voila_stream_t stream);

/* Workspace of voila_generator_bwd for a batch of B rows, in bytes. */
voila_status voila_generator_bwd_workspace_size(const voila_mlp* mlp, int32_t B, size_t* bytes);

/*
 * Hand-written backward of the generator MLP for the distillation loss of
 * Eq. 3. With delta_L = dY and h_l = act(z_l) (h_0 = X):
 *   dW_l = delta_l^T h_{l-1},  db_l = sum over rows of delta_l,
 *   delta_{l-1} = (delta_l W_l) * act'(z_{l-1}),  dX = delta_1 W_1.
 *   X, saved   the inputs and `saved` of voila_generator_fwd_train (device).
 *   dY [B][dims[L]] float (device): gradient of the loss with respect to Y.
 *   dX [B][dims[0]] float (device) or NULL (not computed).
 *   dW, db     HOST arrays of L device pointers: dW[l] [dims[l+1]][dims[l]],
 *              db[l] [dims[l+1]] float, overwritten (not accumulated).
 * Batch sums run over fixed chunks of 1024 rows added in chunk order: the
 * result is the same on every run. The weights read are the ones given
 * (BF16 weights when prec is BF16); the gradients are FP32.
 */
voila_status voila_generator_bwd(const voila_mlp* mlp, const float* X, const float* saved,
                                 const float* dY, int32_t B, float* dX, float* const* dW,
                                 float* const* db, void* workspace, size_t ws_bytes,
                                 voila_stream_t stream);

/*
 * Deterministic (eta = 0) DDIM sampler of the conditional diffusion teacher
 * (Sec. 4.2.1): the targets s'_hat of Eq. 3. For each row i, x_T-1 = omega[i]
 * and for t = T-1 ... 0, with v = teacher([S[i]; A[i]; x_t; e(t)]),
 *   x0 = sqrt(abar_t) x_t - sqrt(1 - abar_t) v,
 *   eps = sqrt(1 - abar_t) x_t + sqrt(abar_t) v,
 *   x_{t-1} = sqrt(abar_{t-1}) x0 + sqrt(1 - abar_{t-1}) eps   (abar_{-1} = 1),
 * abar_t = prod_{u<=t} (1 - beta_u), beta linear from beta0 to beta1 over T
 * steps, e(t) = [sin(t f_i); cos(t f_i)], f_i = 10000^(-i / (emb_dim/2)).
 * Y[i] = x_{-1} = x0 of the last step.
 *   S [B][d_s], A [B][d_a], omega [B][d_x], Y [B][d_x] float (device).
 *   teacher dims[0] = d_s + d_a + d_x + emb_dim, dims[L] = d_x.
 * Limits: 1 <= T <= 64, 1 <= d_x <= 16, emb_dim even and <= 64, widths <= 512.
 * The paper names a cosine schedule; the linear one is the workload's.
 * Kernels: a BF16 teacher with d_s = 8, d_a = 2, d_x = 8, emb_dim = 64 and
 * hidden layers of width 512 runs on the tensor cores (BF16 operands and
 * activations, FP32 accumulation, x kept in FP32); every other teacher runs
 * on the CUDA cores in FP32.
 *   workspace  device, 1024-byte aligned, voila_ddim_sample_workspace_size
 *              bytes; it starts with the status word voila_workspace_status
 *              reads (VOILA_ERR_TIMEOUT if a tensor-core wait expired).
 */
voila_status voila_ddim_sample_workspace_size(const voila_mlp* teacher, int32_t T, size_t* bytes);

voila_status voila_ddim_sample(const voila_mlp* teacher, const float* S, const float* A,
                               const float* omega, int32_t B, int32_t d_s, int32_t d_a,
                               int32_t d_x, int32_t T, double beta0, double beta1,
                               int32_t emb_dim, float* Y, void* workspace, size_t ws_bytes,
                               voila_stream_t stream);

/*
 * One Adam step (Kingma & Ba, 2015) on a flat FP32 vector of n parameters,
 * in place: m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 * p -= lr (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps).
 * params, grads, m, v: device float [n]; m and v start at zero; step >= 1.
 * The paper does not name its optimiser; Adam is this library's choice.
 */
voila_status voila_adam_step(float* params, const float* grads, float* m, float* v, int64_t n,
                             float lr, float beta1, float beta2, float eps, int32_t step,
                             voila_stream_t stream);

typedef struct {
  int32_t T;        /* sampler steps, 1 .. 64 */
  double beta0;     /* linear beta schedule from beta0 ... */
  double beta1;     /* ... to beta1 */
  int32_t emb_dim;  /* step-embedding width, even, <= 64 */
} voila_ddim;

typedef struct {
  float lr, beta1, beta2, eps;
  int32_t step;     /* 1-based step count (bias correction) */
} voila_adam;

/* Workspace of voila_distill_step for B rows, output width d_x and T sampler
 * steps, in bytes. */
voila_status voila_distill_step_workspace_size(const voila_mlp* teacher, const voila_mlp* student,
                                               int32_t B, int32_t d_x, int32_t T, size_t* bytes);

/*
 * One distillation training step of the transition generator (Eq. 3):
 *   1. s_hat = voila_ddim_sample(teacher, S, A, omega)        (teacher targets)
 *   2. Y = student([S; A; omega])                              (Eq. 2)
 *   3. loss = (1/B) sum_b ||Y_b - s_hat_b||^2, dY = 2 (Y - s_hat) / B
 *   4. gradients by voila_generator_bwd
 *   5. voila_adam_step on `master`, then the student's W (in its precision)
 *      and b are overwritten from the updated master.
 *   master, adam_m, adam_v  device float [n_params], the flat layout
 *            [W_0, b_0, W_1, b_1, ...] with W_l [dims[l+1]][dims[l]].
 *   student  the forward copy: its W and b arrays are WRITTEN by step 5
 *            (the const in voila_mlp is not honoured here). FP32 or BF16.
 *   S [B][d_s], A [B][d_a], omega [B][d_x] float (device).
 *   loss_out  device double, the loss of step 3 (before the update).
 *   grad_out  device float [n_params] or NULL: receives the gradient.
 *   workspace device, 1024-byte aligned, voila_distill_step_workspace_size
 *            bytes; its first bytes are the teacher sampler's workspace, so
 *            voila_workspace_status(workspace) reports the sampler's status.
 * Deterministic: every reduction runs in a fixed order.
 * A BF16 student (hidden widths multiples of 16 up to 256) trains on the
 * tensor cores: BF16 operands, activations and deltas, FP32 accumulation,
 * weight gradients as split-K GEMMs over the batch; an FP32 student on the
 * CUDA cores in FP32 (voila_generator_fwd_train / voila_generator_bwd).
 */
voila_status voila_distill_step(const voila_mlp* teacher, const voila_mlp* student,
                                const voila_ddim* ddim, float* master, float* adam_m,
                                float* adam_v, const voila_adam* opt, const float* S,
                                const float* A, const float* omega, int32_t B, int32_t d_s,
                                int32_t d_a, int32_t d_x, double* loss_out, float* grad_out,
                                void* workspace, size_t ws_bytes, voila_stream_t stream);

/* voila_distill_train_step flags. SPREAD: the tensor-core GEMMs launch one CTA
 * per 128-row tile instead of one persistent CTA per SM, so that they start on
 * the SMs that other work running concurrently on the device (the teacher
 * sampler of the next batch) releases; without it they wait for whole SMs.
 * Results do not depend on the flag. */
#define VOILA_TRAIN_SPREAD 1

/* Workspace of voila_distill_train_step for B rows and output width d_x, in
 * bytes. */
voila_status voila_distill_train_step_workspace_size(const voila_mlp* student, int32_t B, int32_t d_x,
                                                     size_t* bytes);

/*
 * Steps 2-5 of voila_distill_step (the student's forward, the loss, the
 * gradients and the Adam update, Eq. 3) with the teacher targets given:
 *   s_hat  device float [B][d_x], the targets voila_ddim_sample wrote for the
 *          same S, A, omega (read only, stream-ordered: the caller orders the
 *          sampler before this call).
 * The other arguments are those of voila_distill_step; flags is 0 or
 * VOILA_TRAIN_SPREAD. The workspace (1024-byte aligned,
 * voila_distill_train_step_workspace_size bytes) is this call's alone, so a
 * sampler run for the next batch on another stream, with its own workspace,
 * can overlap it; its first bytes are the status word of the tensor-core
 * kernels (zeroed by the call; voila_workspace_status). A voila_ddim_sample
 * followed by this call gives exactly the results of voila_distill_step.
 * Errors: VOILA_ERR_ARG (null pointer, negative B, unknown flags),
 * VOILA_ERR_SHAPE (student widths), VOILA_ERR_UNSUPPORTED (precision),
 * VOILA_ERR_WORKSPACE, VOILA_ERR_CUDA.
 */
voila_status voila_distill_train_step(const voila_mlp* student, float* master, float* adam_m,
                                      float* adam_v, const voila_adam* opt, const float* S,
                                      const float* A, const float* omega, const float* s_hat,
                                      int32_t B, int32_t d_s, int32_t d_a, int32_t d_x,
                                      int32_t flags, double* loss_out, float* grad_out,
                                      void* workspace, size_t ws_bytes, voila_stream_t stream);

/*
 * Writes an MLP's weights from a flat FP32 vector [W_0, b_0, W_1, b_1, ...]
 * (W_l [dims[l+1]][dims[l]] row-major): W in the MLP's precision (BF16 by
 * round-to-nearest-even), b as FP32. The arrays the descriptor points to are
 * WRITTEN (the const in voila_mlp is not honoured here). FP32 or BF16 MLPs.
 */
voila_status voila_mlp_load_flat(const voila_mlp* mlp, const float* flat, voila_stream_t stream);

/*
 * PORPP preference backup at the root (Sec. 2.2): with the preferences
 * Psi_k = (1/eta) log pi_0(a_k | b) + J_k of the K action sequences,
 *   V = (1/eta) log sum_k exp(eta Psi_k)   (the log-sum-exp operator L_eta),
 *   pi_k = exp(eta Psi_k - eta V)          (the induced policy).
 *   J [K] double (device): the Monte-Carlo returns of voila_rollout.
 *   log_pi0 [K] double (device) or NULL: uniform reference policy (-log K).
 *   V_out  device double; pi_out [K] device double or NULL.
 * FP64, the maximum subtracted before the exponentials, one CTA in a fixed
 * summation order. eta > 0.
 */
voila_status voila_preference_backup(const double* J, const double* log_pi0, int32_t K, double eta,
                                     double* V_out, double* pi_out, voila_stream_t stream);

/* Workspace of voila_infonce_forward for a batch of B tuples, in bytes. */
voila_status voila_infonce_workspace_size(const voila_mlp* ell, int32_t B, size_t* bytes);

/*
 * InfoNCE objective of the likelihood model (Eq. 6) on B tuples
 * (s'_i, a_i, o_i): the logits of all B x B combinations
 *   L[i][j] = l([s'_i; a_i; o_j]),
 * the row log-sum-exp lse_i = log sum_j exp(L[i][j]), the loss
 * -(1/B) sum_i (L[i][i] - lse_i) and dloss/dL[i][j] = (exp(L[i][j] - lse_i)
 * - [i == j]) / B.
 *   S [B][d_s], A [B][d_a], Ob [B][d_o] float (device); ell dims[0] =
 *   d_s + d_a + d_o, scalar output. B <= 46340.
 *   L_out [B][B] float or NULL (kept in the workspace), lse_out [B] double or
 *   NULL, loss_out device double, G_out [B][B] float or NULL.
 *   workspace  device, 1024-byte aligned; starts with the status word.
 * A BF16 likelihood with d_s = 8, d_a = 2, d_o = 6 and hidden widths that are
 * multiples of 64 up to 256 runs on the tensor cores (BF16 operands and
 * activations, FP32 accumulation); any other on the CUDA cores in FP32.
 */
voila_status voila_infonce_forward(const voila_mlp* ell, const float* S, const float* A,
                                   const float* Ob, int32_t B, int32_t d_s, int32_t d_a,
                                   int32_t d_o, float* L_out, double* lse_out, double* loss_out,
                                   float* G_out, void* workspace, size_t ws_bytes,
                                   voila_stream_t stream);

/* Workspace of voila_infonce_step for a batch of B tuples, in bytes. */
voila_status voila_infonce_step_workspace_size(const voila_mlp* ell, int32_t B, size_t* bytes);

/*
 * One training step of the likelihood model on Eq. 6: the training forward
 * over the B^2 pair rows, the loss and dloss/dL as voila_infonce_forward,
 * the hand-written backward, voila_adam_step on `master` (flat FP32 layout of
 * voila_mlp_load_flat) and voila_mlp_load_flat(ell, master).
 *   loss_out  device double (the loss before the update); grad_out [n_params]
 *             float or NULL.
 *   workspace device, 1024-byte aligned. The batch of B^2 rows keeps its
 *             activations for the backward: on the order of 10 B^2 times the
 *             sum of the hidden widths bytes.
 * A BF16 likelihood trains on the tensor cores (as voila_distill_step's BF16
 * student), an FP32 one on the CUDA cores.
 */
voila_status voila_infonce_step(const voila_mlp* ell, float* master, float* adam_m, float* adam_v,
                                const voila_adam* opt, const float* S, const float* A,
                                const float* Ob, int32_t B, int32_t d_s, int32_t d_a, int32_t d_o,
                                double* loss_out, float* grad_out, void* workspace,
                                size_t ws_bytes, voila_stream_t stream);

/*
 * Action-node tensors of the belief tree that progressive widening reads and
 * updates (device memory, caller-owned).
 *   act [n_nodes][d_a] float   action of each action node
 *   N   [n_nodes] int64        visit counts N(a)            (updated)
 *   C   [n_nodes] int32        observation-branch counts    (updated)
 *   obs [n_nodes][C_max][d_o] float  branch observations    (appended)
 * n_nodes < 2^24, 1 <= C_max <= 65535.
 */
typedef struct {
  int32_t n_nodes, d_a, d_o, C_max;
  const float* act;
  int64_t* N;
  int32_t* C;
  float* obs;
} voila_pw_tree;

/* Workspace of voila_progressive_widening for the tree, observation sampler
 * g_Z (may be NULL: no room for its tensor-core form, which the call then does
 * not use), likelihood ell and M simulations, in bytes. */
voila_status voila_progressive_widening_workspace_size(const voila_pw_tree* tree, const voila_mlp* g_Z,
                                                       const voila_likelihood* ell, int32_t M,
                                                       size_t* bytes);

/*
 * Vectorised progressive widening (Sec. 4.3) for a batch of M simulations:
 * simulation m reached action node node[m] with successor state s_next[m].
 *  1. Simulations are grouped by action node, each group in batch order. The
 *     r-th simulation of node a sees n = N(a) + r + 1 visits; it WIDENS when
 *     C(a) < C_max and C(a) < k_o * pow(n, alpha_o) (FP64): it gets branch
 *     C(a), whose observation f_Z([s'; act[a]; omega_Z]) (Eq. 5, omega_Z at
 *     counter (m, 0, step) of VOILA_STREAM_OBS_OMEGA) is stored in obs[a][C(a)],
 *     and C(a) grows by one. Otherwise it JOINS branch floor(u * C(a)), u the
 *     24-bit uniform of word 0 at counter (m, step, 0) of
 *     VOILA_STREAM_PW_BRANCH. N(a) grows by the group size.
 *  2. l_m = l(s'_m, act[a], obs[a][branch_m]) (Sec. 4.2.3).
 *  3. Each (node, branch) group is resampled as voila_belief_update does:
 *     weights exp(l / lambda) normalised by log-sum-exp, quantised to
 *     multiples of 2^-52, exact prefix sum, systematic resampling with u0
 *     from counter (node, branch, step) of VOILA_STREAM_RESAMPLE (block 1);
 *     slot j of a group (its j-th simulation in batch order) receives the
 *     successor state of simulation idx_out[slot].
 *   node [M] int32 in [0, n_nodes) (others set VOILA_ERR_ARG in the status
 *        word and are skipped); s_next [M][d_s] float; M < 2^24.
 *   g_Z  dims [d_s + d_a + d_omega] -> ... -> d_o, FP32 or BF16 weights
 *        (FP32 arithmetic); ell: MLP of [s'; a; o] or GAUSSIAN (d_o <= d_s).
 *        A BF16 likelihood of the planning shapes (s' 8, a 2, o 6, hidden
 *        widths multiples of 64 up to 256) runs on the tensor cores (BF16
 *        activations, FP32 accumulation); any other on the CUDA cores in FP32.
 *   branch_out [M] int32, s_out [M][d_s] float: required.
 *   widened_out [M] uint8, ell_out [M] float, w_out [M] double, idx_out [M]
 *   int32: optional (NULL).
 *   workspace  device, 1024-byte aligned; starts with the status word
 *              (VOILA_ERR_ARG, VOILA_ERR_NONFINITE, VOILA_ERR_DEGENERATE,
 *              VOILA_ERR_TIMEOUT).
 */
voila_status voila_progressive_widening(const voila_pw_tree* tree, const int32_t* node,
                                        const float* s_next, int32_t M, int32_t d_s,
                                        const voila_mlp* g_Z, const voila_likelihood* ell,
                                        int32_t d_omega, double k_o, double alpha_o, float lambda,
                                        uint64_t seed, uint32_t step, uint32_t planner_id,
                                        int32_t* branch_out, uint8_t* widened_out, float* ell_out,
                                        double* w_out, int32_t* idx_out, float* s_out,
                                        void* workspace, size_t ws_bytes, voila_stream_t stream);

/*
 * Raw Philox4x32-10 words: out[4 i + j] = word j of counter (i, c1, c2, c3),
 * i < n. out holds 4 n uint32 (device).
 */
voila_status voila_philox_fill(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t* out, int64_t n, voila_stream_t stream);

/*
 * The normals the kernels draw: out[i][d] = component d of the noise vector
 * at counter (i, c1, c2) of stream `stream_id`, i < n, d < dim (float, device).
 */
voila_status voila_normal_fill(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t stream_id,
                               uint32_t planner_id, int32_t dim, float* out, int64_t n,
                               voila_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* VOILA_H_ */

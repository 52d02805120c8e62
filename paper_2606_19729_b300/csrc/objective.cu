// PORPP preference backup over the root's action sequences (Sec. 2.2) and the
// InfoNCE objective of the likelihood model on all B x B pairs (Eq. 6).
//
// Backup: V = (1/eta) log sum_k exp(eta J_k + lp_k), pi_k = exp(eta J_k + lp_k
// - eta V), lp_k = log pi_0(a_k) (uniform -log K when not given); FP64, the
// maximum is subtracted before the exponentials, one CTA in a fixed order.
//
// InfoNCE: L[i][j] = l([s'_i; a_i; o_j]) on the tensor cores (BF16 likelihood
// of the planning shapes) or on the CUDA cores (any other), then one CTA per
// row for lse_i = log sum_j exp(L_ij) and dloss/dL_ij = (exp(L_ij - lse_i) -
// [i == j]) / B, and one CTA for loss = -(1/B) sum_i (L_ii - lse_i). The
// training step runs the training forward and the hand-written backward over
// the B^2 pair rows (tensor cores for a BF16 likelihood, CUDA cores in FP32
// otherwise), then Adam.
#include <math.h>
#include <string.h>

#include "../../include/voila.h"
#include "trace.h"
#include "common.cuh"
#include "kernels.h"
#include "reduce.cuh"
#include "simt_mlp.cuh"
#include "tc.h"
#include "train_tc.h"

namespace voila {
namespace {

__global__ void __launch_bounds__(1024) backup_kernel(const double* __restrict__ J, const double* __restrict__ lp0,
                                                      int K, double eta, double* __restrict__ V,
                                                      double* __restrict__ pi) {
  __shared__ double red[33];
  const double lpu = -log((double)K);
  double m = -INFINITY;
  for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, eta * J[k] + (lp0 ? lp0[k] : lpu));
  m = block_max(m, red);
  double z = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) z += exp(eta * J[k] + (lp0 ? lp0[k] : lpu) - m);
  z = block_sum(z, red);
  const double lz = log(z);
  if (threadIdx.x == 0) *V = (m + lz) / eta;
  if (pi)
    for (int k = threadIdx.x; k < K; k += blockDim.x) pi[k] = exp(eta * J[k] + (lp0 ? lp0[k] : lpu) - m - lz);
}

// The pair rows [s'_i; a_i; o_j], row i * B + j.
__global__ void pairs_input_kernel(const float* __restrict__ S, const float* __restrict__ A,
                                   const float* __restrict__ Ob, int B, int d_s, int d_a, int d_o,
                                   float* __restrict__ X) {
  const int din = d_s + d_a + d_o;
  const long long n = (long long)B * B * din;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / din;
    const int c = (int)(e % din);
    const long long i = row / B, j = row % B;
    X[e] = c < d_s ? S[i * d_s + c] : c < d_s + d_a ? A[i * d_a + c - d_s] : Ob[j * d_o + c - d_s - d_a];
  }
}

// L[row] = l(pair row) on the CUDA cores, kSimtRows rows per tile.
template <typename TW>
__global__ void __launch_bounds__(kSimtThreads) pairs_simt_kernel(MlpDev m, const float* __restrict__ S,
                                                                  const float* __restrict__ A,
                                                                  const float* __restrict__ Ob, int B, int d_s,
                                                                  int d_a, int d_o, int ld, float* __restrict__ L) {
  extern __shared__ __align__(16) float sm[];
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  const int din = d_s + d_a + d_o;
  const long long rows = (long long)B * B;
  const long long ntiles = (rows + kSimtRows - 1) / kSimtRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kSimtRows;
    const int nr = (int)min((long long)kSimtRows, rows - row0);
    __syncthreads();
    for (int e = threadIdx.x; e < kSimtRows * din; e += blockDim.x) {
      const int r = e / din, c = e % din;
      float v = 0.0f;
      if (r < nr) {
        const long long i = (row0 + r) / B, j = (row0 + r) % B;
        v = c < d_s ? S[i * d_s + c] : c < d_s + d_a ? A[i * d_a + c - d_s] : Ob[j * d_o + c - d_s - d_a];
      }
      bufA[r * ld + c] = v;
    }
    const float* y = simt_mlp<TW>(m, bufA, bufB, ld, nr);
    for (int r = threadIdx.x; r < nr; r += blockDim.x) L[row0 + r] = y[r * ld];
  }
}

// Row i: lse_i, diag_i = L_ii - lse_i and (optionally) G_i. = (softmax - e_i) / B.
// One warp per row (eight rows per CTA): the maximum in FP32 (exact), the sum
// of exp(L_ij - max) (FP32 exponentials) in FP64 per lane, then a fixed-order
// warp reduction, so every row's sum has one order.
constexpr int kRowsPerCta = 8;
__global__ void __launch_bounds__(32 * kRowsPerCta) infonce_rows_kernel(const float* __restrict__ L, int B,
                                                                       double* __restrict__ lse_out,
                                                                       double* __restrict__ diag,
                                                                       float* __restrict__ G) {
  const int i = blockIdx.x * kRowsPerCta + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= B) return;
  const float* Li = L + (size_t)i * B;
  float mf = -INFINITY;
  for (int j = lane; j < B; j += 32) mf = fmaxf(mf, Li[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
  double z = 0.0;
  for (int j = lane; j < B; j += 32) z += (double)expf(Li[j] - mf);
  z = warp_sum(z);
  const double lse = (double)mf + log(z);
  if (lane == 0) {
    if (lse_out) lse_out[i] = lse;
    diag[i] = (double)Li[i] - lse;
  }
  if (G) {
    const float inv_b = 1.0f / (float)B, lf = (float)lse;
    float* Gi = G + (size_t)i * B;
    for (int j = lane; j < B; j += 32) Gi[j] = (expf(Li[j] - lf) - (j == i ? 1.0f : 0.0f)) * inv_b;
  }
}

__global__ void __launch_bounds__(1024) infonce_loss_kernel(const double* __restrict__ diag, int B,
                                                            double* __restrict__ loss) {
  __shared__ double red[33];
  double a = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) a += diag[i];
  a = block_sum(a, red);
  if (threadIdx.x == 0) *loss = -a / (double)B;
}

size_t a1024(size_t x) { return (x + 1023) & ~(size_t)1023; }

bool mlp_ok(const voila_mlp* m) { return m && m->n_layers >= 1 && m->n_layers <= VOILA_MAX_LAYERS; }

int widest_of(const voila_mlp* m) {
  int w = 0;
  for (int l = 0; l <= m->n_layers; ++l) w = m->dims[l] > w ? m->dims[l] : w;
  return w;
}

// Forward workspace: header | tensor-core scratch | L [B*B] f32 | diag [B] f64
struct FwdLayout {
  size_t tc, L, diag, total;
};

FwdLayout fwd_layout(const voila_mlp* ell, int B) {
  FwdLayout f;
  size_t o = 1024;
  f.tc = o;
  o += a1024(tc_pairs_scratch_bytes(ell));
  f.L = o;
  o += a1024((size_t)B * B * sizeof(float));
  f.diag = o;
  o += a1024((size_t)B * sizeof(double));
  f.total = o;
  return f;
}

voila_status check_infonce(const voila_mlp* ell, int B, int d_s, int d_a, int d_o) {
  if (!mlp_ok(ell) || B < 0 || B > 46340 || d_s < 0 || d_a < 0 || d_o < 0) return VOILA_ERR_ARG;
  if (ell->prec != VOILA_FP32 && ell->prec != VOILA_BF16) return VOILA_ERR_UNSUPPORTED;
  if (ell->dims[0] != d_s + d_a + d_o || ell->dims[ell->n_layers] != 1 || widest_of(ell) > VOILA_MAX_WIDTH)
    return VOILA_ERR_SHAPE;
  return VOILA_OK;
}

int grid_for(long long n, int per) {
  long long g = (n + per - 1) / per;
  if (g > 148 * 32) g = 148 * 32;
  return (int)(g < 1 ? 1 : g);
}

voila_status lse_and_loss(const float* L, int B, double* lse_out, double* diag, float* G, double* loss,
                          cudaStream_t s) {
  infonce_rows_kernel<<<(B + kRowsPerCta - 1) / kRowsPerCta, 32 * kRowsPerCta, 0, s>>>(L, B, lse_out, diag, G);
  infonce_loss_kernel<<<1, 1024, 0, s>>>(diag, B, loss);
  return cudaGetLastError() == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

}  // namespace
}  // namespace voila

using namespace voila;

extern "C" {

voila_status voila_preference_backup(const double* J, const double* log_pi0, int32_t K, double eta, double* V_out,
                                     double* pi_out, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (K < 1 || !J || !V_out || !(eta > 0.0) || !isfinite(eta)) return VOILA_ERR_ARG;
  backup_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(J, log_pi0, K, eta, V_out, pi_out);
  return cudaGetLastError() == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

voila_status voila_infonce_workspace_size(const voila_mlp* ell, int32_t B, size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!mlp_ok(ell) || !bytes || B < 0 || B > 46340) return VOILA_ERR_ARG;
  *bytes = fwd_layout(ell, B).total;
  return VOILA_OK;
}

voila_status voila_infonce_forward(const voila_mlp* ell, const float* S, const float* A, const float* Ob, int32_t B,
                                   int32_t d_s, int32_t d_a, int32_t d_o, float* L_out, double* lse_out,
                                   double* loss_out, float* G_out, void* workspace, size_t ws_bytes,
                                   voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  voila_status st = check_infonce(ell, B, d_s, d_a, d_o);
  if (st != VOILA_OK) return st;
  if (!loss_out) return VOILA_ERR_ARG;
  const FwdLayout F = fwd_layout(ell, B);
  if (!workspace || ws_bytes < F.total || ((uintptr_t)workspace & 1023)) return VOILA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  if (cudaMemsetAsync(ws, 0, sizeof(WsHeader), s) != cudaSuccess) return VOILA_ERR_CUDA;
  if (B == 0) return cudaMemsetAsync(loss_out, 0, sizeof(double), s) == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
  if (!S || !Ob || (d_a && !A)) return VOILA_ERR_ARG;
  float* L = L_out ? L_out : (float*)(ws + F.L);
  if (tc_pairs_supported(ell, d_s, d_a, d_o)) {
    st = tc_likelihood_pairs(ell, S, A, Ob, B, L, (WsHeader*)ws, ws + F.tc, s);
    if (st != VOILA_OK) return st;
  } else {
    MlpDev m;
    memset(&m, 0, sizeof(m));
    m.n_layers = ell->n_layers;
    m.act = ell->act;
    m.prec = ell->prec;
    for (int l = 0; l <= VOILA_MAX_LAYERS; ++l) m.dims[l] = ell->dims[l];
    for (int l = 0; l < ell->n_layers; ++l) {
      m.W[l] = ell->W[l];
      m.b[l] = ell->b[l];
    }
    const int wmax = widest_of(ell);
    const int ld = simt_ld(wmax);
    const size_t smem = (size_t)2 * kSimtRows * ld * sizeof(float);
    auto k = ell->prec == VOILA_BF16 ? pairs_simt_kernel<__nv_bfloat16> : pairs_simt_kernel<float>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return VOILA_ERR_CUDA;
    const long long ntiles = ((long long)B * B + kSimtRows - 1) / kSimtRows;
    k<<<(int)(ntiles < 148 * 4 ? ntiles : 148 * 4), kSimtThreads, smem, s>>>(m, S, A, Ob, B, d_s, d_a, d_o, ld, L);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  return lse_and_loss(L, B, lse_out, (double*)(ws + F.diag), G_out, loss_out, s);
}

// Training step workspace: header | X [B^2][din] | L [B^2] | saved [B^2][hidden] |
// G [B^2] | grads [n_params] | diag [B] | scratch (backward)
static size_t step_param_count(const voila_mlp* m) {
  size_t n = 0;
  for (int l = 0; l < m->n_layers; ++l) n += (size_t)m->dims[l + 1] * m->dims[l] + m->dims[l + 1];
  return n;
}

static size_t step_hidden(const voila_mlp* m) {
  size_t h = 0;
  for (int l = 0; l + 1 < m->n_layers; ++l) h += m->dims[l + 1];
  return h;
}

struct StepLayout {
  size_t x, L, saved, G, grads, diag, scratch, total;
  bool tc;  // BF16 likelihood: training forward/backward on the tensor cores
};

static StepLayout step_layout(const voila_mlp* ell, int B) {
  StepLayout S;
  const size_t rows = (size_t)B * B;
  size_t o = 1024;
  S.x = o;
  o += a1024(rows * ell->dims[0] * 4);
  S.L = o;
  o += a1024(rows * 4);
  S.tc = tc_train_supported(ell);
  S.saved = o;
  o += S.tc ? 0 : a1024(rows * step_hidden(ell) * 4);
  S.G = o;
  o += a1024(rows * 4);
  S.grads = o;
  o += a1024(step_param_count(ell) * 4);
  S.diag = o;
  o += a1024((size_t)B * 8);
  S.scratch = o;
  size_t bwd = 0;
  if (S.tc) bwd = tc_train_bytes(ell, (long long)rows);
  else voila_generator_bwd_workspace_size(ell, (int32_t)rows, &bwd);
  o += a1024(bwd);
  S.total = o;
  return S;
}

voila_status voila_infonce_step_workspace_size(const voila_mlp* ell, int32_t B, size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!mlp_ok(ell) || !bytes || B < 0 || B > 46340) return VOILA_ERR_ARG;
  *bytes = step_layout(ell, B).total;
  return VOILA_OK;
}

voila_status voila_infonce_step(const voila_mlp* ell, float* master, float* adam_m, float* adam_v,
                                const voila_adam* opt, const float* S, const float* A, const float* Ob, int32_t B,
                                int32_t d_s, int32_t d_a, int32_t d_o, double* loss_out, float* grad_out,
                                void* workspace, size_t ws_bytes, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  voila_status st = check_infonce(ell, B, d_s, d_a, d_o);
  if (st != VOILA_OK) return st;
  if (!master || !adam_m || !adam_v || !opt || !loss_out) return VOILA_ERR_ARG;
  if (B == 0) return VOILA_OK;
  if (!S || !Ob || (d_a && !A)) return VOILA_ERR_ARG;
  const StepLayout L = step_layout(ell, B);
  if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 1023)) return VOILA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  if (cudaMemsetAsync(ws, 0, sizeof(WsHeader), s) != cudaSuccess) return VOILA_ERR_CUDA;
  const int rows = B * B;
  float* X = (float*)(ws + L.x);
  float* Lm = (float*)(ws + L.L);
  float* saved = (float*)(ws + L.saved);
  float* G = (float*)(ws + L.G);
  float* grads = grad_out ? grad_out : (float*)(ws + L.grads);
  double* diag = (double*)(ws + L.diag);
  void* scratch = ws + L.scratch;
  const size_t scratch_bytes = L.total - L.scratch;
  pairs_input_kernel<<<grid_for((long long)rows * ell->dims[0], 256), 256, 0, s>>>(S, A, Ob, B, d_s, d_a, d_o, X);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  if (L.tc) st = tc_train_forward(ell, X, rows, Lm, scratch, (WsHeader*)ws, s);
  else st = voila_generator_fwd_train(ell, X, rows, Lm, saved, scratch, scratch_bytes, stream);
  if (st != VOILA_OK) return st;
  st = lse_and_loss(Lm, B, nullptr, diag, G, loss_out, s);
  if (st != VOILA_OK) return st;
  float* dW[VOILA_MAX_LAYERS];
  float* db[VOILA_MAX_LAYERS];
  size_t off = 0;
  for (int l = 0; l < ell->n_layers; ++l) {
    dW[l] = grads + off;
    off += (size_t)ell->dims[l + 1] * ell->dims[l];
    db[l] = grads + off;
    off += ell->dims[l + 1];
  }
  if (L.tc) st = tc_train_backward(ell, G, rows, grads, scratch, (WsHeader*)ws, s);
  else st = voila_generator_bwd(ell, X, saved, G, rows, nullptr, dW, db, scratch, scratch_bytes, stream);
  if (st != VOILA_OK) return st;
  st = voila_adam_step(master, grads, adam_m, adam_v, (int64_t)off, opt->lr, opt->beta1, opt->beta2, opt->eps,
                       opt->step, stream);
  if (st != VOILA_OK) return st;
  return voila_mlp_load_flat(ell, master, stream);
}

}  // extern "C"

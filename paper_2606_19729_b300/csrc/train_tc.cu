// MLP training forward and backward on the tensor cores (BF16 operands and
// activations, FP32 accumulation) for the distillation step (Eq. 3) and the
// likelihood's InfoNCE step (Eq. 6).
//
// With layers l = 1..L, W_l [d_l][d_{l-1}], z_l = h_{l-1} W_l^T + b_l,
// h_l = act(z_l) (h_0 = X), y = z_L:
//   forward   one GEMM per layer; hidden layers keep h_l (row-major, the next
//             GEMM's A operand), h_l^T (the dW GEMMs' B operand) and act'(z_l);
//   backward  delta_L = dY; delta_{l-1} = (delta_l W_l) * act'(z_{l-1}) with
//             the transposed weights as B operand; dW_l = delta_l^T h_{l-1} as
//             split-K GEMMs over the batch whose FP32 partials are summed in
//             split order; db_l = column sums of delta_l in a fixed order.
// Every sum runs in a fixed order, so a step is deterministic.
#include <math.h>
#include <string.h>

#include "../../include/voila.h"
#include "common.cuh"
#include "gemm.h"
#include "reduce.cuh"
#include "train_tc.h"

namespace voila {
namespace {

constexpr int kColsumBlocks = 148;  // row blocks of the output-bias gradient

int r16(int v) { return (v + 15) / 16 * 16; }
size_t a1k(size_t x) { return (x + 1023) & ~(size_t)1023; }

struct TrainLayout {
  int L, d[VOILA_MAX_LAYERS + 1], K0p, NLp;
  long long M, ldT;
  size_t xb, xt, h[VOILA_MAX_LAYERS], ht[VOILA_MAX_LAYERS], ad[VOILA_MAX_LAYERS], dl, dlt;
  size_t dd[VOILA_MAX_LAYERS], ddt[VOILA_MAX_LAYERS], w1p, wlp, wt[VOILA_MAX_LAYERS + 1], part, colpart, total;
  int splits_max;
};

TrainLayout train_layout(const voila_mlp* m, long long M) {
  TrainLayout T;
  memset(&T, 0, sizeof(T));
  T.L = m->n_layers;
  for (int l = 0; l <= T.L; ++l) T.d[l] = m->dims[l];
  T.K0p = r16(T.d[0]);
  T.NLp = r16(T.d[T.L]);
  T.M = M;
  T.ldT = (M + 127) / 128 * 128;
  const size_t bf = 2;
  size_t o = 0;
  T.xb = o; o += a1k((size_t)M * T.K0p * bf);
  T.xt = o; o += a1k((size_t)T.K0p * T.ldT * bf);
  for (int l = 1; l < T.L; ++l) {
    T.h[l] = o; o += a1k((size_t)M * T.d[l] * bf);
    T.ht[l] = o; o += a1k((size_t)T.d[l] * T.ldT * bf);
    T.ad[l] = o; o += a1k((size_t)M * T.d[l] * bf);
    T.dd[l] = o; o += a1k((size_t)M * T.d[l] * bf);
    T.ddt[l] = o; o += a1k((size_t)T.d[l] * T.ldT * bf);
  }
  T.dl = o; o += a1k((size_t)M * T.NLp * bf);
  T.dlt = o; o += a1k((size_t)T.NLp * T.ldT * bf);
  T.w1p = o; o += a1k((size_t)T.d[1] * T.K0p * bf);
  T.wlp = o; o += a1k((size_t)T.NLp * T.d[T.L - 1] * bf);
  for (int l = 2; l <= T.L; ++l) {
    const int kl = l == T.L ? T.NLp : T.d[l];
    T.wt[l] = o; o += a1k((size_t)T.d[l - 1] * kl * bf);
  }
  T.splits_max = 148;
  T.part = o; o += a1k((size_t)T.splits_max * 256 * 256 * sizeof(float));
  T.colpart = o; o += a1k((size_t)kColsumBlocks * 256 * sizeof(double));
  T.total = o;
  return T;
}

// X (FP32 [M][d]) -> Xb [M][Kp] and X^T [Kp][ldT], BF16, zero padded (Kp a
// multiple of 8). One row per thread: the row goes out in 16-byte stores, and
// a warp's transposed stores of one column are 32 consecutive rows.
__global__ void pad_rows_kernel(const float* __restrict__ X, long long M, int d, int Kp, long long ldT,
                                __nv_bfloat16* __restrict__ xb, __nv_bfloat16* __restrict__ xt) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
    const float* x = X + m * d;
    for (int c0 = 0; c0 < Kp; c0 += 8) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const int c = c0 + j;
        const __nv_bfloat16 lo = __float2bfloat16_rn(c < d ? x[c] : 0.0f);
        const __nv_bfloat16 hi = __float2bfloat16_rn(c + 1 < d ? x[c + 1] : 0.0f);
        xt[(size_t)c * ldT + m] = lo;
        xt[(size_t)(c + 1) * ldT + m] = hi;
        w[j >> 1] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      }
      *reinterpret_cast<uint4*>(xb + m * Kp + c0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// dst[r][c] = src[r][c] (r < R, c < C) else 0, for r < Rp, c < Cp.
__global__ void pad_copy_kernel(const __nv_bfloat16* __restrict__ src, int R, int C, int Rp, int Cp,
                                __nv_bfloat16* __restrict__ dst) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Rp * Cp; e += gridDim.x * blockDim.x) {
    const int r = e / Cp, c = e % Cp;
    dst[e] = (r < R && c < C) ? src[(size_t)r * C + c] : __float2bfloat16_rn(0.0f);
  }
}

// dst[c][r] = src[r][c] for r < R, c < C; dst is [C][Rp], zero for r >= R.
__global__ void pad_transpose_kernel(const __nv_bfloat16* __restrict__ src, int R, int C, int Rp,
                                     __nv_bfloat16* __restrict__ dst) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C * Rp; e += gridDim.x * blockDim.x) {
    const int c = e / Rp, r = e % Rp;
    dst[e] = r < R ? src[(size_t)r * C + c] : __float2bfloat16_rn(0.0f);
  }
}

// out[r][c] = sum_s P[s][r][c] (s in order), r < R, c < C; P is [S][Rg][Cg].
// Eight partials are loaded ahead of their (ordered) additions.
__global__ void reduce_partials_kernel(const float* __restrict__ P, int S, int Rg, int Cg, int R, int C,
                                       float* __restrict__ out) {
  const size_t step = (size_t)Rg * Cg;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * C; e += gridDim.x * blockDim.x) {
    const int r = e / C, c = e % C;
    const float* src = P + (size_t)r * Cg + c;
    float acc = 0.0f;
    int s = 0;
    for (; s + 8 <= S; s += 8) {
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldg(src + (size_t)(s + j) * step);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc += v[j];
    }
    for (; s < S; ++s) acc += __ldg(src + (size_t)s * step);
    out[e] = acc;
  }
}

// out[n] = sum_m DT[n][m], m < M (one CTA per n, eight values per 16-byte
// load and the tail of M element by element, in a fixed order).
__global__ void __launch_bounds__(256) rowsum_bf16_kernel(const __nv_bfloat16* __restrict__ DT, long long M,
                                                          long long ldT, float* __restrict__ out) {
  __shared__ double red[33];
  const __nv_bfloat16* row = DT + (size_t)blockIdx.x * ldT;
  const long long groups = M / 8;
  float a = 0.0f;
  long long gi = threadIdx.x;
  for (; gi + 3 * blockDim.x < groups; gi += 4 * blockDim.x) {  // four loads ahead, added in order
    uint4 w4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w4[u] = __ldg(reinterpret_cast<const uint4*>(row + 8 * (gi + u * blockDim.x)));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t ws[4] = {w4[u].x, w4[u].y, w4[u].z, w4[u].w};
#pragma unroll
      for (int j = 0; j < 4; ++j) a += __uint_as_float(ws[j] << 16) + __uint_as_float(ws[j] & 0xffff0000u);
    }
  }
  for (; gi < groups; gi += blockDim.x) {
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(row + 8 * gi));
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) a += __uint_as_float(ws[j] << 16) + __uint_as_float(ws[j] & 0xffff0000u);
  }
  for (long long m = 8 * groups + threadIdx.x; m < M; m += blockDim.x) a += __bfloat162float(row[m]);
  const double t = block_sum((double)a, red);
  if (threadIdx.x == 0) out[blockIdx.x] = (float)t;
}

// part[b][c] = sum over the rows of block b of dY[m][c] (contiguous row ranges,
// fixed order), then out[c] = sum_b part[b][c] in a fixed order. Thread t of a
// block (dL <= blockDim.x) adds column t mod dL of rows t / dL, + blockDim.x / dL,
// ... (consecutive threads read consecutive floats); the block then adds the
// threads of a column in thread order.
__global__ void __launch_bounds__(256) colsum_partial_kernel(const float* __restrict__ dY, long long M, int dL,
                                                             double* __restrict__ part) {
  __shared__ double red[256];
  const int rpi = blockDim.x / dL;  // rows per pass
  const int c = threadIdx.x % dL, r0 = threadIdx.x / dL;
  const long long per = (M + gridDim.x - 1) / gridDim.x;
  const long long m0 = blockIdx.x * per, m1 = m0 + per < M ? m0 + per : M;
  double a = 0.0;
  if (r0 < rpi)
    for (long long m = m0 + r0; m < m1; m += rpi) a += (double)__ldg(dY + m * dL + c);
  red[threadIdx.x] = a;
  __syncthreads();
  if ((int)threadIdx.x < dL) {
    double t = 0.0;
    for (int i = 0; i < rpi; ++i) t += red[i * dL + threadIdx.x];
    part[(size_t)blockIdx.x * dL + threadIdx.x] = t;
  }
}

// warp w sums columns w, w + 8, ...: lane j adds blocks j, j + 32, ..., then a
// fixed butterfly over the lanes
__global__ void colsum_final_kernel(const double* __restrict__ part, int nb, int dL, float* __restrict__ out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = w; c < dL; c += blockDim.x >> 5) {
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) a += part[(size_t)b * dL + c];
#pragma unroll
    for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[c] = (float)a;
  }
}

int grid_of(long long n) {
  long long g = (n + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

}  // namespace

bool tc_train_supported(const voila_mlp* m) {
  if (!m || m->prec != VOILA_BF16 || m->n_layers < 2 || m->n_layers > VOILA_MAX_LAYERS) return false;
  if (m->dims[0] < 1 || m->dims[0] > 256 || m->dims[m->n_layers] < 1 || m->dims[m->n_layers] > 256) return false;
  for (int l = 1; l < m->n_layers; ++l)
    if (m->dims[l] % 16 || m->dims[l] > 256) return false;
  if (m->act != VOILA_ACT_SILU && m->act != VOILA_ACT_TANH && m->act != VOILA_ACT_IDENTITY) return false;
  return true;
}

size_t tc_train_bytes(const voila_mlp* m, long long M) { return train_layout(m, M).total; }

voila_status tc_train_forward(const voila_mlp* m, const float* X, long long M, float* Y, void* scratch,
                              WsHeader* hdr, cudaStream_t s, bool spread) {
  if (!tc_train_supported(m) || ((uintptr_t)scratch & 1023)) return VOILA_ERR_UNSUPPORTED;
  const TrainLayout T = train_layout(m, M);
  const int L = T.L;
  typedef __nv_bfloat16 bf;
  // operands: padded input and first/last weights, transposed weights for the backward
  pad_rows_kernel<<<grid_of(M), 256, 0, s>>>(X, M, T.d[0], T.K0p, T.ldT, at<bf>(scratch, T.xb),
                                             at<bf>(scratch, T.xt));
  pad_copy_kernel<<<grid_of((long long)T.d[1] * T.K0p), 256, 0, s>>>((const bf*)m->W[0], T.d[1], T.d[0], T.d[1],
                                                                      T.K0p, at<bf>(scratch, T.w1p));
  pad_copy_kernel<<<grid_of((long long)T.NLp * T.d[L - 1]), 256, 0, s>>>(
      (const bf*)m->W[L - 1], T.d[L], T.d[L - 1], T.NLp, T.d[L - 1], at<bf>(scratch, T.wlp));
  for (int l = 2; l <= L; ++l) {
    const int kl = l == L ? T.NLp : T.d[l];
    pad_transpose_kernel<<<grid_of((long long)T.d[l - 1] * kl), 256, 0, s>>>((const bf*)m->W[l - 1], T.d[l],
                                                                             T.d[l - 1], kl, at<bf>(scratch, T.wt[l]));
  }
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  for (int l = 1; l <= L; ++l) {
    TcGemm g;
    memset(&g, 0, sizeof(g));
    g.A = l == 1 ? at<bf>(scratch, T.xb) : at<bf>(scratch, T.h[l - 1]);
    g.lda = l == 1 ? T.K0p : T.d[l - 1];
    g.K = g.lda;
    g.M = M;
    g.splits = 1;
    g.bias = m->b[l - 1];
    g.act = m->act;
    g.hdr = hdr;
    g.spread = spread;
    if (l < L) {
      g.B = l == 1 ? at<bf>(scratch, T.w1p) : (const bf*)m->W[l - 1];
      g.ldb = g.lda;
      g.N = T.d[l];
      g.mode = kGemmFwdHidden;
      g.H = at<bf>(scratch, T.h[l]);
      g.AD = at<bf>(scratch, T.ad[l]);
      g.HT = at<bf>(scratch, T.ht[l]);
      g.ldT = (int)T.ldT;
    } else {
      g.B = at<bf>(scratch, T.wlp);
      g.ldb = T.d[L - 1];
      g.N = T.NLp;
      g.mode = kGemmFwdOut;
      g.Y = Y;
      g.ldY = T.d[L];
      g.n_real = T.d[L];
    }
    if (tc_gemm(g, s) != cudaSuccess) return VOILA_ERR_CUDA;
  }
  return VOILA_OK;
}

voila_status tc_train_backward(const voila_mlp* m, const float* dY, long long M, float* grads, void* scratch,
                               WsHeader* hdr, cudaStream_t s, bool spread) {
  if (!tc_train_supported(m) || ((uintptr_t)scratch & 1023)) return VOILA_ERR_UNSUPPORTED;
  const TrainLayout T = train_layout(m, M);
  const int L = T.L;
  typedef __nv_bfloat16 bf;
  // flat gradient layout [W_0, b_0, W_1, b_1, ...]
  size_t goff[VOILA_MAX_LAYERS + 1][2];
  size_t o = 0;
  for (int l = 1; l <= L; ++l) {
    goff[l][0] = o;
    o += (size_t)T.d[l] * T.d[l - 1];
    goff[l][1] = o;
    o += T.d[l];
  }
  pad_rows_kernel<<<grid_of(M), 256, 0, s>>>(dY, M, T.d[L], T.NLp, T.ldT, at<bf>(scratch, T.dl),
                                             at<bf>(scratch, T.dlt));
  colsum_partial_kernel<<<kColsumBlocks, 256, 0, s>>>(dY, M, T.d[L], at<double>(scratch, T.colpart));
  colsum_final_kernel<<<1, 256, 0, s>>>(at<double>(scratch, T.colpart), kColsumBlocks, T.d[L], grads + goff[L][1]);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  // deltas of the hidden layers
  for (int l = L; l >= 2; --l) {
    TcGemm g;
    memset(&g, 0, sizeof(g));
    g.A = l == L ? at<bf>(scratch, T.dl) : at<bf>(scratch, T.dd[l]);
    g.lda = l == L ? T.NLp : T.d[l];
    g.K = g.lda;
    g.B = at<bf>(scratch, T.wt[l]);
    g.ldb = g.lda;
    g.M = M;
    g.N = T.d[l - 1];
    g.splits = 1;
    g.mode = kGemmBwd;
    g.AD_in = at<bf>(scratch, T.ad[l - 1]);
    g.H = at<bf>(scratch, T.dd[l - 1]);
    g.HT = at<bf>(scratch, T.ddt[l - 1]);
    g.ldT = (int)T.ldT;
    g.hdr = hdr;
    g.spread = spread;
    if (tc_gemm(g, s) != cudaSuccess) return VOILA_ERR_CUDA;
  }
  // weight gradients: split-K over the batch, partials summed in split order
  float* part = at<float>(scratch, T.part);
  const long long kchunks = (M + 63) / 64;
  for (int l = 1; l <= L; ++l) {
    const int Mg = l == L ? T.NLp : T.d[l];
    const int Ng = l == 1 ? T.K0p : T.d[l - 1];
    const int tiles = (Mg + 127) / 128;
    int splits = T.splits_max / tiles;
    if (splits < 1) splits = 1;
    if (splits > kchunks) splits = (int)kchunks;
    const long long per = (kchunks + splits - 1) / splits;  // as tc_gemm splits K
    splits = (int)((kchunks + per - 1) / per);
    TcGemm g;
    memset(&g, 0, sizeof(g));
    g.A = l == L ? at<bf>(scratch, T.dlt) : at<bf>(scratch, T.ddt[l]);
    g.lda = T.ldT;
    g.B = l == 1 ? at<bf>(scratch, T.xt) : at<bf>(scratch, T.ht[l - 1]);
    g.ldb = T.ldT;
    g.M = Mg;
    g.K = M;
    g.N = Ng;
    g.splits = splits;
    g.mode = kGemmPartial;
    g.P = part;
    g.hdr = hdr;
    g.spread = spread;
    if (tc_gemm(g, s) != cudaSuccess) return VOILA_ERR_CUDA;
    reduce_partials_kernel<<<grid_of((long long)T.d[l] * T.d[l - 1]), 256, 0, s>>>(
        part, splits, Mg, Ng, T.d[l], T.d[l - 1], grads + goff[l][0]);
    if (l < L) rowsum_bf16_kernel<<<T.d[l], 256, 0, s>>>(at<bf>(scratch, T.ddt[l]), M, T.ldT, grads + goff[l][1]);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  return VOILA_OK;
}

}  // namespace voila

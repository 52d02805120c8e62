// Training-side kernels: the generator forward that saves pre-activations,
// its hand-written backward (distillation, Eq. 3), and the teacher's DDIM
// sampler (Sec. 4.2.1). FP32 arithmetic on CUDA cores; weights FP32 or BF16.
//
// Backward of y = L_n(act(... act(L_1(x)))), L_l(h) = h W_l^T + b_l:
//   delta_n = dY;  dW_l = delta_l^T H_{l-1};  db_l = sum_b delta_l[b];
//   delta_{l-1} = (delta_l W_l) * act'(z_{l-1});  dX = delta_1 W_1,
// with H_{l-1} = act(z_{l-1}) (H_0 = X) recomputed from the saved z.
// Batch reductions (dW, db) are split over fixed batch chunks and summed in a
// fixed order, so results do not depend on scheduling.
#include <math.h>
#include <string.h>

#include "../../include/voila.h"
#include "trace.h"
#include "common.cuh"
#include "kernels.h"
#include "simt_mlp.cuh"
#include "tc.h"
#include "train_tc.h"

namespace voila {

namespace {

constexpr int kTile = 64;        // output tile of the GEMM kernels
constexpr int kKc = 16;          // reduction chunk staged in shared memory
constexpr int kBChunk = 1024;    // batch rows per partial dW / db

__device__ __forceinline__ float act_f(float z, int act) { return act_fp32(z, act); }

__device__ __forceinline__ float act_grad(float z, int act) {
  if (act == VOILA_ACT_TANH) {
    const float t = tanhf(z);
    return 1.0f - t * t;
  }
  if (act == VOILA_ACT_SILU) {
    const float sg = 1.0f / (1.0f + expf(-z));
    return sg * (1.0f + z * (1.0f - sg));
  }
  return 1.0f;
}

// Forward of one layer for training: z = h W^T + b written to `z_out` (if the
// layer is hidden) and act(z) (or z for the last layer) to `h_out`.
// One thread per output element; weights through the read-only cache.
template <typename TW>
__global__ void __launch_bounds__(256) layer_fwd_kernel(const float* __restrict__ h_in, int ld_in,
                                                        const TW* __restrict__ W, const float* __restrict__ b,
                                                        int B, int K, int N, int act, bool last,
                                                        float* __restrict__ z_out, int ld_z,
                                                        float* __restrict__ h_out, int ld_out) {
  __shared__ float hs[kTile][kKc + 1];
  __shared__ float ws[kKc][kTile + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 outputs each
  const int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kKc) {
    for (int i = threadIdx.x; i < kTile * kKc; i += blockDim.x) {
      const int r = i / kKc, k = i % kKc;
      const int row = row0 + r, kk = k0 + k;
      hs[r][k] = (row < B && kk < K) ? h_in[(size_t)row * ld_in + kk] : 0.0f;
      const int c = i / kKc;  // reuse the same index space for W^T tile
      const int col = col0 + c;
      ws[k][c] = (col < N && kk < K) ? ldw<TW>(W + (size_t)col * K + kk) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kKc; ++k) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = hs[ty * 4 + i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = ws[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = row0 + ty * 4 + i, col = col0 + tx * 4 + j;
      if (row < B && col < N) {
        const float z = acc[i][j] + b[col];
        if (!last && z_out) z_out[(size_t)row * ld_z + col] = z;
        h_out[(size_t)row * ld_out + col] = last ? z : act_f(z, act);
      }
    }
}

// delta_prev[b][k] = (sum_n delta[b][n] W[n][k]) * act'(z_prev[b][k])
// (act' skipped when z_prev is null: the gradient with respect to x).
template <typename TW>
__global__ void __launch_bounds__(256) delta_back_kernel(const float* __restrict__ delta, int ld_d,
                                                         const TW* __restrict__ W, int B, int N, int K,
                                                         const float* __restrict__ z_prev, int ld_z, int act,
                                                         float* __restrict__ out, int ld_out) {
  __shared__ float ds[kTile][kKc + 1];
  __shared__ float ws[kKc][kTile + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
  float acc[4][4] = {};
  for (int n0 = 0; n0 < N; n0 += kKc) {
    for (int i = threadIdx.x; i < kTile * kKc; i += blockDim.x) {
      const int r = i / kKc, n = i % kKc;
      const int row = row0 + r, nn = n0 + n;
      ds[r][n] = (row < B && nn < N) ? delta[(size_t)row * ld_d + nn] : 0.0f;
      const int c = i % kTile, n2 = i / kTile;
      const int col = col0 + c, nn2 = n0 + n2;
      ws[n2][c] = (col < K && nn2 < N) ? ldw<TW>(W + (size_t)nn2 * K + col) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int n = 0; n < kKc; ++n) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = ds[ty * 4 + i][n];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = ws[n][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int row = row0 + ty * 4 + i, col = col0 + tx * 4 + j;
      if (row < B && col < K) {
        float v = acc[i][j];
        if (z_prev) v *= act_grad(z_prev[(size_t)row * ld_z + col], act);
        out[(size_t)row * ld_out + col] = v;
      }
    }
}

// Partial weight and bias gradients of one batch chunk:
// part[chunk][n][k] = sum_{b in chunk} delta[b][n] * H[b][k], H = act(z_in) or X;
// bpart[chunk][n] = sum_{b in chunk} delta[b][n].
__global__ void __launch_bounds__(256) dw_partial_kernel(const float* __restrict__ delta, int ld_d,
                                                         const float* __restrict__ hin, int ld_h, bool apply_act,
                                                         int act, int B, int N, int K, float* __restrict__ part,
                                                         float* __restrict__ bpart) {
  __shared__ float dsm[kKc][kTile + 1];
  __shared__ float hsm[kKc][kTile + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int n0 = blockIdx.y * kTile, k0 = blockIdx.x * kTile;
  const int chunk = blockIdx.z;
  const int b_begin = chunk * kBChunk, b_end = min(B, b_begin + kBChunk);
  float acc[4][4] = {};
  float bacc[4] = {};
  for (int bb = b_begin; bb < b_end; bb += kKc) {
    for (int i = threadIdx.x; i < kKc * kTile; i += blockDim.x) {
      const int r = i / kTile, c = i % kTile;
      const int row = bb + r;
      const bool in = row < b_end;
      dsm[r][c] = (in && n0 + c < N) ? delta[(size_t)row * ld_d + n0 + c] : 0.0f;
      float h = (in && k0 + c < K) ? hin[(size_t)row * ld_h + k0 + c] : 0.0f;
      if (apply_act && in && k0 + c < K) h = act_f(h, act);
      hsm[r][c] = h;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kKc; ++r) {
      float d[4], h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) d[i] = dsm[r][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = hsm[r][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        bacc[i] += d[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(d[i], h[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  float* out = part + (size_t)chunk * N * K;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n = n0 + ty * 4 + i;
    if (n >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = k0 + tx * 4 + j;
      if (k < K) out[(size_t)n * K + k] = acc[i][j];
    }
    if (blockIdx.x == 0 && tx == 0) bpart[(size_t)chunk * N + n] = bacc[i];
  }
}

// dst[e] = sum_{c < chunks} part[c][e], fixed order.
__global__ void chunk_sum_kernel(const float* __restrict__ part, int chunks, long long elems, float* __restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < elems;
       e += (long long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < chunks; ++c) s += part[(size_t)c * elems + e];
    dst[e] = s;
  }
}

int grid_for(long long n, int per) {
  long long g = (n + per - 1) / per;
  if (g > 148 * 32) g = 148 * 32;
  return (int)(g < 1 ? 1 : g);
}

int hidden_total(const voila_mlp* m) {
  int t = 0;
  for (int l = 0; l + 1 < m->n_layers; ++l) t += m->dims[l + 1];
  return t;
}

int widest(const voila_mlp* m) {
  int w = 0;
  for (int l = 0; l <= m->n_layers; ++l) w = m->dims[l] > w ? m->dims[l] : w;
  return w;
}

template <typename TW>
cudaError_t fwd_train(const voila_mlp* m, const float* X, int B, float* Y, float* saved, float* tmp,
                      cudaStream_t s) {
  // hidden activations ping-pong in tmp ([2][B][widest]); z saved per layer
  const int ldz = hidden_total(m), wmax = widest(m);
  const float* h = X;
  int ld_h = m->dims[0];
  int zoff = 0;
  for (int l = 0; l < m->n_layers; ++l) {
    const int K = m->dims[l], N = m->dims[l + 1];
    const bool last = l == m->n_layers - 1;
    float* out = last ? Y : tmp + (size_t)(l & 1) * B * wmax;
    const int ld_out = last ? N : wmax;
    dim3 grid((N + kTile - 1) / kTile, (B + kTile - 1) / kTile);
    layer_fwd_kernel<TW><<<grid, 256, 0, s>>>(h, ld_h, (const TW*)m->W[l], m->b[l], B, K, N, m->act, last,
                                             saved ? saved + zoff : nullptr, ldz, out, ld_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    h = out;
    ld_h = ld_out;
    if (!last) zoff += N;
  }
  return cudaSuccess;
}

template <typename TW>
cudaError_t bwd(const voila_mlp* m, const float* X, const float* saved, const float* dY, int B, float* dX,
                float* const* dW, float* const* db, float* ws, cudaStream_t s) {
  const int ldz = hidden_total(m), wmax = widest(m);
  const int chunks = (B + kBChunk - 1) / kBChunk;
  float* dbuf[2] = {ws, ws + (size_t)B * wmax};
  float* part = dbuf[1] + (size_t)B * wmax;
  size_t pmax = 0;
  for (int l = 0; l < m->n_layers; ++l) {
    const size_t e = (size_t)m->dims[l + 1] * m->dims[l];
    pmax = e > pmax ? e : pmax;
  }
  float* bpart = part + (size_t)chunks * pmax;
  int zoff[VOILA_MAX_LAYERS + 1];
  zoff[0] = 0;
  for (int l = 0; l + 1 < m->n_layers; ++l) zoff[l + 1] = zoff[l] + m->dims[l + 1];
  const float* delta = dY;
  int ld_d = m->dims[m->n_layers];
  cudaError_t e;
  for (int l = m->n_layers - 1; l >= 0; --l) {
    const int K = m->dims[l], N = m->dims[l + 1];
    // input of layer l: X, or act(z_{l-1})
    const float* hin = l == 0 ? X : saved + zoff[l - 1];
    const int ld_h = l == 0 ? m->dims[0] : ldz;
    dim3 g1((K + kTile - 1) / kTile, (N + kTile - 1) / kTile, chunks);
    dw_partial_kernel<<<g1, 256, 0, s>>>(delta, ld_d, hin, ld_h, l > 0, m->act, B, N, K, part, bpart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    chunk_sum_kernel<<<grid_for((long long)N * K, 256), 256, 0, s>>>(part, chunks, (long long)N * K, dW[l]);
    chunk_sum_kernel<<<grid_for(N, 256), 256, 0, s>>>(bpart, chunks, N, db[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l > 0 || dX) {
      float* out = l > 0 ? dbuf[l & 1] : dX;
      const int ld_out = l > 0 ? wmax : K;
      dim3 g2((K + kTile - 1) / kTile, (B + kTile - 1) / kTile);
      delta_back_kernel<TW><<<g2, 256, 0, s>>>(delta, ld_d, (const TW*)m->W[l], B, N, K,
                                               l > 0 ? saved + zoff[l - 1] : nullptr, ldz, m->act, out, ld_out);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      delta = out;
      ld_d = ld_out;
    }
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// DDIM teacher sampling: one CTA owns 32 rows through all T steps; the
// denoiser runs as the shared-memory MLP tile of the CUDA-core path.
// ---------------------------------------------------------------------------
struct DdimArgs {
  MlpDev m;
  const float* S;
  const float* A;
  const float* omega;
  int B, d_s, d_a, d_x, T, emb;
  float sq_ab[64], sq_1mab[64];  // sqrt(abar_t), sqrt(1 - abar_t)
  float freq[32];                 // step-embedding frequencies 10000^(-i/half)
  float* Y;
  int ld;
};

template <typename TW>
__global__ void __launch_bounds__(kSimtThreads) ddim_kernel(DdimArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int ld = a.ld;
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  float* xs = bufB + kSimtRows * ld;   // [rows][d_x]
  const int din = a.d_s + a.d_a + a.d_x + a.emb;
  const long long ntiles = ((long long)a.B + kSimtRows - 1) / kSimtRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kSimtRows;
    const int nr = (int)min((long long)kSimtRows, (long long)a.B - row0);
    __syncthreads();
    for (int i = threadIdx.x; i < kSimtRows * a.d_x; i += blockDim.x) {
      const int r = i / a.d_x, d = i % a.d_x;
      xs[r * 16 + d] = r < nr ? a.omega[(size_t)(row0 + r) * a.d_x + d] : 0.0f;
    }
    for (int t = a.T - 1; t >= 0; --t) {
      __syncthreads();
      for (int i = threadIdx.x; i < kSimtRows * din; i += blockDim.x) {
        const int r = i / din, c = i % din;
        float v = 0.0f;
        if (r < nr) {
          if (c < a.d_s) v = a.S[(size_t)(row0 + r) * a.d_s + c];
          else if (c < a.d_s + a.d_a) v = a.A[(size_t)(row0 + r) * a.d_a + c - a.d_s];
          else if (c < a.d_s + a.d_a + a.d_x) v = xs[r * 16 + c - a.d_s - a.d_a];
          else {
            const int e = c - a.d_s - a.d_a - a.d_x, half = a.emb / 2;
            const float arg = (float)t * a.freq[e < half ? e : e - half];
            v = e < half ? sinf(arg) : cosf(arg);
          }
        }
        bufA[r * ld + c] = v;
      }
      const float* vhat = simt_mlp<TW>(a.m, bufA, bufB, ld, nr);
      const float sab = a.sq_ab[t], s1 = a.sq_1mab[t];
      const float sabp = t > 0 ? a.sq_ab[t - 1] : 1.0f, s1p = t > 0 ? a.sq_1mab[t - 1] : 0.0f;
      for (int i = threadIdx.x; i < nr * a.d_x; i += blockDim.x) {
        const int r = i / a.d_x, d = i % a.d_x;
        const float x = xs[r * 16 + d], v = vhat[r * ld + d];
        const float x0 = sab * x - s1 * v, eps = s1 * x + sab * v;
        xs[r * 16 + d] = sabp * x0 + s1p * eps;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr * a.d_x; i += blockDim.x) {
      const int r = i / a.d_x, d = i % a.d_x;
      a.Y[(size_t)(row0 + r) * a.d_x + d] = xs[r * 16 + d];
    }
  }
}


// X[b] = [S[b]; A[b]; omega[b]]: the generator input of Eq. 2.
__global__ void concat_input_kernel(const float* __restrict__ S, const float* __restrict__ A,
                                    const float* __restrict__ omega, int B, int d_s, int d_a, int d_x,
                                    float* __restrict__ X) {
  const int din = d_s + d_a + d_x;
  const long long n = (long long)B * din;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / din;
    const int c = (int)(i % din);
    X[i] = c < d_s ? S[b * d_s + c] : c < d_s + d_a ? A[b * d_a + c - d_s] : omega[b * d_x + c - d_s - d_a];
  }
}

constexpr int kLossBlocks = 296;  // fixed grid: the loss sum has one order

// r = Y - T;  dY = 2 r / B;  part[block] = sum of r^2 over the block's rows (FP64).
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                                  long long n, float inv_b2, float* __restrict__ dY,
                                                  double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = Y[i] - T[i];
    dY[i] = r * inv_b2;
    acc += (double)r * (double)r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_final_kernel(const double* __restrict__ part, int nparts, double inv_b, double* __restrict__ loss) {
  __shared__ double red[512];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += part[i];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] * inv_b;
}

// Adam (Kingma & Ba, 2015) on a flat FP32 parameter vector; c1 = 1 - beta1^t,
// c2 = 1 - beta2^t are the bias corrections of step t.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float beta1, float beta2, float eps,
                            float inv_c1, float inv_c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * inv_c1) / (sqrtf(vi * inv_c2) + eps);
  }
}

// Writes the forward copy of the student (W in its precision, b FP32) from the
// flat master vector [W_0, b_0, W_1, b_1, ...].
struct PublishArgs {
  int n_layers;
  long long off[2 * VOILA_MAX_LAYERS + 1];  // start of W_l at off[2l], b_l at off[2l+1]
  void* W[VOILA_MAX_LAYERS];
  float* b[VOILA_MAX_LAYERS];
};

template <typename TW>
__global__ void publish_kernel(const float* __restrict__ master, PublishArgs a) {
  const long long n = a.off[2 * a.n_layers];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int seg = 0;
    while (i >= a.off[seg + 1]) ++seg;
    const long long j = i - a.off[seg];
    const float x = master[i];
    if (seg & 1) a.b[seg >> 1][j] = x;
    else reinterpret_cast<TW*>(a.W[seg >> 1])[j] = (TW)x;
  }
}

long long param_layout(const voila_mlp* m, long long* off) {
  long long o = 0;
  for (int l = 0; l < m->n_layers; ++l) {
    off[2 * l] = o;
    o += (long long)m->dims[l + 1] * m->dims[l];
    off[2 * l + 1] = o;
    o += m->dims[l + 1];
  }
  off[2 * m->n_layers] = o;
  return o;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t bwd_ws_bytes(const voila_mlp* m, int B) {
  const int chunks = (B + kBChunk - 1) / kBChunk;
  size_t pmax = 0, nmax = 0;
  for (int l = 0; l < m->n_layers; ++l) {
    const size_t e = (size_t)m->dims[l + 1] * m->dims[l];
    pmax = e > pmax ? e : pmax;
    nmax = (size_t)m->dims[l + 1] > nmax ? (size_t)m->dims[l + 1] : nmax;
  }
  return ((size_t)2 * B * widest(m) + (size_t)chunks * (pmax + nmax)) * sizeof(float);
}

// Workspace of the teacher sampler: the status header (1024 bytes), then the
// tensor-core scratch (packed teacher, step embeddings) when that path runs.
constexpr size_t kDdimHeader = 1024;

size_t ddim_ws_bytes(const voila_mlp* teacher, int T) {
  const size_t tc = tc_ddim_scratch_bytes(teacher, T);
  return kDdimHeader + (tc + 1023) / 1024 * 1024;
}

// Workspace of the distillation step, in this order (each 256-byte aligned):
// teacher-sampler workspace, s_hat [B][d_x], X [B][din], Y [B][d_x],
// dY [B][d_x], saved [B][hidden], grads [n_params], loss partials
// [kLossBlocks] (FP64), scratch (bwd).
// The student's part of a distillation step (forward, loss, backward, Adam),
// offsets from the start of its region; the first kDdimHeader bytes are a
// status header when the region is a workspace of its own.
struct TrainRegion {
  size_t x, y, dy, saved, grads, part, scratch, total;
  bool tc;  // BF16 student: the training forward/backward run on the tensor cores (scratch)
};

TrainRegion train_region(const voila_mlp* st, int B, int d_x) {
  TrainRegion L;
  long long off[2 * VOILA_MAX_LAYERS + 1];
  const long long np = param_layout(st, off);
  size_t o = kDdimHeader;
  L.x = o;     o += align256((size_t)B * st->dims[0] * 4);
  L.y = o;     o += align256((size_t)B * d_x * 4);
  L.dy = o;    o += align256((size_t)B * d_x * 4);
  L.saved = o; o += tc_train_supported(st) ? 0 : align256((size_t)B * hidden_total(st) * 4);
  L.grads = o; o += align256((size_t)np * 4);
  L.part = o;  o += align256(kLossBlocks * 8);
  L.tc = tc_train_supported(st);
  o = (o + 1023) & ~(size_t)1023;
  L.scratch = o; o += L.tc ? tc_train_bytes(st, B) : align256(bwd_ws_bytes(st, B));
  L.total = o;
  return L;
}

struct DistillLayout {
  size_t ddim, s_hat, train, total;  // sampler workspace, targets, the student's region (1024-aligned)
  TrainRegion t;
};

DistillLayout distill_layout(const voila_mlp* teacher, const voila_mlp* st, int B, int d_x, int T) {
  DistillLayout L;
  size_t o = 0;
  L.ddim = o;  o += align256(ddim_ws_bytes(teacher, T));
  L.s_hat = o; o += align256((size_t)B * d_x * 4);
  o = (o + 1023) & ~(size_t)1023;
  L.train = o;
  L.t = train_region(st, B, d_x);
  L.total = o + L.t.total;
  return L;
}

bool student_ok(const voila_mlp* student, int d_s, int d_a, int d_x, voila_status* err) {
  if (student->n_layers < 1 || student->n_layers > VOILA_MAX_LAYERS) return *err = VOILA_ERR_ARG, false;
  if (student->prec != VOILA_FP32 && student->prec != VOILA_BF16) return *err = VOILA_ERR_UNSUPPORTED, false;
  if (student->dims[0] != d_s + d_a + d_x || student->dims[student->n_layers] != d_x)
    return *err = VOILA_ERR_SHAPE, false;
  for (int l = 0; l < student->n_layers; ++l)
    if (!student->W[l] || !student->b[l]) return *err = VOILA_ERR_ARG, false;
  return true;
}

// Steps 2-5 of a distillation step with the targets s_hat given; `base` is the
// student's region (TrainRegion offsets), `hdr` the status word the
// tensor-core kernels write.
voila_status distill_train(const voila_mlp* student, float* master, float* adam_m, float* adam_v,
                           const voila_adam* opt, const float* S, const float* A, const float* omega,
                           const float* s_hat, int32_t B, int32_t d_s, int32_t d_a, int32_t d_x, bool spread,
                           double* loss_out, float* grad_out, char* base, const TrainRegion& L, WsHeader* hdr,
                           cudaStream_t s);
}  // namespace
}  // namespace voila

using namespace voila;
namespace voila {
namespace {
voila_status distill_train(const voila_mlp* student, float* master, float* adam_m, float* adam_v,
                           const voila_adam* opt, const float* S, const float* A, const float* omega,
                           const float* s_hat, int32_t B, int32_t d_s, int32_t d_a, int32_t d_x, bool spread,
                           double* loss_out, float* grad_out, char* base, const TrainRegion& L, WsHeader* hdr,
                           cudaStream_t s) {
  float* X = (float*)(base + L.x);
  float* Y = (float*)(base + L.y);
  float* dY = (float*)(base + L.dy);
  float* saved = (float*)(base + L.saved);
  float* grads = grad_out ? grad_out : (float*)(base + L.grads);
  double* part = (double*)(base + L.part);
  float* scratch = (float*)(base + L.scratch);
  const size_t scratch_bytes = L.total - L.scratch;
  const voila_stream_t stream = (voila_stream_t)s;
  // 2. student forward f_T(s, a, omega), pre-activations saved
  concat_input_kernel<<<grid_for((long long)B * student->dims[0], 256), 256, 0, s>>>(S, A, omega, B, d_s, d_a,
                                                                                     d_x, X);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  voila_status st;
  if (L.tc) st = tc_train_forward(student, X, B, Y, scratch, hdr, s, spread);
  else st = voila_generator_fwd_train(student, X, B, Y, saved, scratch, scratch_bytes, stream);
  if (st != VOILA_OK) return st;
  // 3. loss (1/B) sum ||f - s_hat||^2 and dL/dY = 2 (f - s_hat) / B
  mse_kernel<<<kLossBlocks, 256, 0, s>>>(Y, s_hat, (long long)B * d_x, 2.0f / (float)B, dY, part);
  loss_final_kernel<<<1, 512, 0, s>>>(part, kLossBlocks, 1.0 / (double)B, loss_out);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  // 4. gradients into the flat layout of `master`
  long long off[2 * VOILA_MAX_LAYERS + 1];
  const long long np = param_layout(student, off);
  float* dW[VOILA_MAX_LAYERS];
  float* db[VOILA_MAX_LAYERS];
  for (int l = 0; l < student->n_layers; ++l) {
    dW[l] = grads + off[2 * l];
    db[l] = grads + off[2 * l + 1];
  }
  if (L.tc) st = tc_train_backward(student, dY, B, grads, scratch, hdr, s, spread);
  else st = voila_generator_bwd(student, X, saved, dY, B, nullptr, dW, db, scratch, scratch_bytes, stream);
  if (st != VOILA_OK) return st;
  // 5. Adam on the FP32 master weights, then the forward copy
  st = voila_adam_step(master, grads, adam_m, adam_v, np, opt->lr, opt->beta1, opt->beta2, opt->eps, opt->step,
                       stream);
  if (st != VOILA_OK) return st;
  return voila_mlp_load_flat(student, master, stream);
}
}  // namespace
}  // namespace voila


extern "C" {

voila_status voila_generator_fwd_train(const voila_mlp* mlp, const float* X, int32_t B, float* Y, float* saved,
                                       void* workspace, size_t ws_bytes, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!mlp || mlp->n_layers < 1 || mlp->n_layers > VOILA_MAX_LAYERS || B < 0) return VOILA_ERR_ARG;
  if (mlp->prec != VOILA_FP32 && mlp->prec != VOILA_BF16) return VOILA_ERR_UNSUPPORTED;
  if (B == 0) return VOILA_OK;
  if (!X || !Y) return VOILA_ERR_ARG;
  const size_t need = (size_t)2 * B * widest(mlp) * sizeof(float);
  if (!workspace || ws_bytes < need) return VOILA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = mlp->prec == VOILA_BF16 ? fwd_train<__nv_bfloat16>(mlp, X, B, Y, saved, (float*)workspace, s)
                                          : fwd_train<float>(mlp, X, B, Y, saved, (float*)workspace, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

voila_status voila_generator_bwd_workspace_size(const voila_mlp* mlp, int32_t B, size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!mlp || !bytes || mlp->n_layers < 1 || mlp->n_layers > VOILA_MAX_LAYERS || B < 0) return VOILA_ERR_ARG;
  *bytes = bwd_ws_bytes(mlp, B);
  return VOILA_OK;
}

voila_status voila_generator_bwd(const voila_mlp* mlp, const float* X, const float* saved, const float* dY,
                                 int32_t B, float* dX, float* const* dW, float* const* db, void* workspace,
                                 size_t ws_bytes, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!mlp || mlp->n_layers < 1 || mlp->n_layers > VOILA_MAX_LAYERS || B < 0 || !dW || !db) return VOILA_ERR_ARG;
  if (mlp->prec != VOILA_FP32 && mlp->prec != VOILA_BF16) return VOILA_ERR_UNSUPPORTED;
  for (int l = 0; l < mlp->n_layers; ++l)
    if (!dW[l] || !db[l]) return VOILA_ERR_ARG;
  if (B == 0) return VOILA_OK;
  if (!X || !dY || (mlp->n_layers > 1 && !saved)) return VOILA_ERR_ARG;
  size_t need = 0;
  voila_generator_bwd_workspace_size(mlp, B, &need);
  if (!workspace || ws_bytes < need) return VOILA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = mlp->prec == VOILA_BF16
                      ? bwd<__nv_bfloat16>(mlp, X, saved, dY, B, dX, dW, db, (float*)workspace, s)
                      : bwd<float>(mlp, X, saved, dY, B, dX, dW, db, (float*)workspace, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

voila_status voila_ddim_sample_workspace_size(const voila_mlp* teacher, int32_t T, size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!teacher || !bytes || teacher->n_layers < 1 || teacher->n_layers > VOILA_MAX_LAYERS || T < 1 || T > 64)
    return VOILA_ERR_ARG;
  *bytes = ddim_ws_bytes(teacher, T);
  return VOILA_OK;
}

voila_status voila_ddim_sample(const voila_mlp* teacher, const float* S, const float* A, const float* omega,
                               int32_t B, int32_t d_s, int32_t d_a, int32_t d_x, int32_t T, double beta0,
                               double beta1, int32_t emb_dim, float* Y, void* workspace, size_t ws_bytes,
                               voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!teacher || teacher->n_layers < 1 || teacher->n_layers > VOILA_MAX_LAYERS || B < 0) return VOILA_ERR_ARG;
  if (teacher->prec != VOILA_FP32 && teacher->prec != VOILA_BF16) return VOILA_ERR_UNSUPPORTED;
  if (T < 1 || T > 64 || d_x < 1 || d_x > 16 || emb_dim < 0 || emb_dim > 64 || (emb_dim & 1) || d_s < 0 ||
      d_a < 0)
    return VOILA_ERR_ARG;
  if (teacher->dims[0] != d_s + d_a + d_x + emb_dim || teacher->dims[teacher->n_layers] != d_x ||
      widest(teacher) > VOILA_MAX_WIDTH)
    return VOILA_ERR_SHAPE;
  if (!workspace || ws_bytes < ddim_ws_bytes(teacher, T) || ((uintptr_t)workspace & 1023))
    return VOILA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(workspace, 0, sizeof(WsHeader), s) != cudaSuccess) return VOILA_ERR_CUDA;
  if (B == 0) return VOILA_OK;
  if (!omega || !Y || (d_s && !S) || (d_a && !A)) return VOILA_ERR_ARG;
  if (tc_ddim_supported(teacher, d_s, d_a, d_x, emb_dim)) {
    // x_{tau-1} = cx x_tau + cv v with cx = sqrt(abar_{tau-1} abar_tau) + sqrt((1-abar_{tau-1})(1-abar_tau)),
    // cv = sqrt((1-abar_{tau-1}) abar_tau) - sqrt(abar_{tau-1} (1-abar_tau)), abar_{-1} = 1
    double abar[64], cx[64], cv[64], freq[32];
    double ab = 1.0;
    for (int u = 0; u < T; ++u) {
      ab *= 1.0 - (T > 1 ? beta0 + (beta1 - beta0) * u / (T - 1) : beta0);
      abar[u] = ab;
    }
    for (int t = 0; t < T; ++t) {
      const int tau = T - 1 - t;
      const double sab = sqrt(abar[tau]), s1 = sqrt(1.0 - abar[tau]);
      const double sabp = tau > 0 ? sqrt(abar[tau - 1]) : 1.0, s1p = tau > 0 ? sqrt(1.0 - abar[tau - 1]) : 0.0;
      cx[t] = sabp * sab + s1p * s1;
      cv[t] = s1p * sab - sabp * s1;
    }
    for (int i = 0; i < 32; ++i) freq[i] = pow(10000.0, -(double)i / 32.0);
    return tc_ddim_sample(teacher, S, A, omega, B, T, cx, cv, freq, Y, (WsHeader*)workspace,
                          (char*)workspace + kDdimHeader, s);
  }
  DdimArgs a;
  memset(&a, 0, sizeof(a));
  a.m.n_layers = teacher->n_layers;
  a.m.act = teacher->act;
  a.m.prec = teacher->prec;
  for (int l = 0; l <= VOILA_MAX_LAYERS; ++l) a.m.dims[l] = teacher->dims[l];
  for (int l = 0; l < VOILA_MAX_LAYERS; ++l) {
    a.m.W[l] = teacher->W[l];
    a.m.b[l] = teacher->b[l];
  }
  a.S = S;
  a.A = A;
  a.omega = omega;
  a.B = B;
  a.d_s = d_s;
  a.d_a = d_a;
  a.d_x = d_x;
  a.T = T;
  a.emb = emb_dim;
  double ab = 1.0;
  for (int t = 0; t < T; ++t) {  // linear beta, abar_t = prod (1 - beta)
    const double beta = T > 1 ? beta0 + (beta1 - beta0) * t / (T - 1) : beta0;
    ab *= 1.0 - beta;
    a.sq_ab[t] = (float)sqrt(ab);
    a.sq_1mab[t] = (float)sqrt(1.0 - ab);
  }
  for (int i = 0; i < emb_dim / 2; ++i) a.freq[i] = (float)pow(10000.0, -(double)i / (emb_dim / 2));
  a.Y = Y;
  const int wmax = widest(teacher);
  a.ld = simt_ld(wmax);
  const size_t smem = (size_t)2 * kSimtRows * a.ld * sizeof(float) + kSimtRows * 16 * sizeof(float);
  auto k = teacher->prec == VOILA_BF16 ? ddim_kernel<__nv_bfloat16> : ddim_kernel<float>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return VOILA_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kSimtThreads, smem) != cudaSuccess || per_sm < 1)
    return VOILA_ERR_CUDA;
  const long long ntiles = ((long long)B + kSimtRows - 1) / kSimtRows;
  const long long slots = (long long)sms * per_sm;
  k<<<(int)(ntiles < slots ? ntiles : slots), kSimtThreads, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

voila_status voila_adam_step(float* params, const float* grads, float* m, float* v, int64_t n, float lr,
                             float beta1, float beta2, float eps, int32_t step, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (n < 0 || step < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
      !(eps > 0.0f))
    return VOILA_ERR_ARG;
  if (n == 0) return VOILA_OK;
  if (!params || !grads || !m || !v) return VOILA_ERR_ARG;
  const double c1 = 1.0 - pow((double)beta1, step), c2 = 1.0 - pow((double)beta2, step);
  adam_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(params, grads, m, v, n, lr, beta1, beta2, eps,
                                                                   (float)(1.0 / c1), (float)(1.0 / c2));
  return cudaGetLastError() == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

voila_status voila_distill_step_workspace_size(const voila_mlp* teacher, const voila_mlp* student, int32_t B,
                                               int32_t d_x, int32_t T, size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!teacher || !student || !bytes || student->n_layers < 1 || student->n_layers > VOILA_MAX_LAYERS || B < 0 ||
      d_x < 1 || teacher->n_layers < 1 || teacher->n_layers > VOILA_MAX_LAYERS || T < 1 || T > 64)
    return VOILA_ERR_ARG;
  *bytes = distill_layout(teacher, student, B, d_x, T).total;
  return VOILA_OK;
}

voila_status voila_distill_step(const voila_mlp* teacher, const voila_mlp* student, const voila_ddim* ddim,
                                float* master, float* adam_m, float* adam_v, const voila_adam* opt,
                                const float* S, const float* A, const float* omega, int32_t B, int32_t d_s,
                                int32_t d_a, int32_t d_x, double* loss_out, float* grad_out, void* workspace,
                                size_t ws_bytes, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!teacher || !student || !ddim || !opt || !master || !adam_m || !adam_v || !loss_out || B < 0)
    return VOILA_ERR_ARG;
  voila_status err = VOILA_OK;
  if (!student_ok(student, d_s, d_a, d_x, &err)) return err;
  if (ddim->T < 1 || ddim->T > 64) return VOILA_ERR_ARG;
  if (B == 0) return VOILA_OK;
  const DistillLayout L = distill_layout(teacher, student, B, d_x, ddim->T);
  if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 1023)) return VOILA_ERR_WORKSPACE;
  char* ws = (char*)workspace;
  float* s_hat = (float*)(ws + L.s_hat);
  // 1. teacher targets s_hat' (the ODE sampler of Eq. 3)
  voila_status st = voila_ddim_sample(teacher, S, A, omega, B, d_s, d_a, d_x, ddim->T, ddim->beta0, ddim->beta1,
                                      ddim->emb_dim, s_hat, ws + L.ddim, L.s_hat - L.ddim, stream);
  if (st != VOILA_OK) return st;
  // 2-5. the student's step; its kernels report into the sampler's status word
  return distill_train(student, master, adam_m, adam_v, opt, S, A, omega, s_hat, B, d_s, d_a, d_x, false,
                       loss_out, grad_out, ws + L.train, L.t, (WsHeader*)ws, (cudaStream_t)stream);
}

voila_status voila_distill_train_step_workspace_size(const voila_mlp* student, int32_t B, int32_t d_x,
                                                     size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!student || !bytes || student->n_layers < 1 || student->n_layers > VOILA_MAX_LAYERS || B < 0 || d_x < 1)
    return VOILA_ERR_ARG;
  *bytes = train_region(student, B, d_x).total;
  return VOILA_OK;
}

voila_status voila_distill_train_step(const voila_mlp* student, float* master, float* adam_m, float* adam_v,
                                      const voila_adam* opt, const float* S, const float* A, const float* omega,
                                      const float* s_hat, int32_t B, int32_t d_s, int32_t d_a, int32_t d_x,
                                      int32_t flags, double* loss_out, float* grad_out, void* workspace,
                                      size_t ws_bytes, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!student || !opt || !master || !adam_m || !adam_v || !loss_out || B < 0 || (flags & ~VOILA_TRAIN_SPREAD))
    return VOILA_ERR_ARG;
  voila_status err = VOILA_OK;
  if (!student_ok(student, d_s, d_a, d_x, &err)) return err;
  if (B == 0) return VOILA_OK;
  if (!S || !A || !omega || !s_hat) return VOILA_ERR_ARG;
  const TrainRegion L = train_region(student, B, d_x);
  if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 1023)) return VOILA_ERR_WORKSPACE;
  WsHeader* hdr = (WsHeader*)workspace;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s) != cudaSuccess) return VOILA_ERR_CUDA;
  return distill_train(student, master, adam_m, adam_v, opt, S, A, omega, s_hat, B, d_s, d_a, d_x,
                       (flags & VOILA_TRAIN_SPREAD) != 0, loss_out, grad_out, (char*)workspace, L, hdr, s);
}

voila_status voila_mlp_load_flat(const voila_mlp* mlp, const float* flat, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!mlp || !flat || mlp->n_layers < 1 || mlp->n_layers > VOILA_MAX_LAYERS) return VOILA_ERR_ARG;
  if (mlp->prec != VOILA_FP32 && mlp->prec != VOILA_BF16) return VOILA_ERR_UNSUPPORTED;
  for (int l = 0; l < mlp->n_layers; ++l)
    if (!mlp->W[l] || !mlp->b[l]) return VOILA_ERR_ARG;
  long long off[2 * VOILA_MAX_LAYERS + 1];
  const long long np = param_layout(mlp, off);
  PublishArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.n_layers = mlp->n_layers;
  for (int i = 0; i <= 2 * mlp->n_layers; ++i) pa.off[i] = off[i];
  for (int l = 0; l < mlp->n_layers; ++l) {
    pa.W[l] = const_cast<void*>(mlp->W[l]);
    pa.b[l] = const_cast<float*>(mlp->b[l]);
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (mlp->prec == VOILA_BF16)
    publish_kernel<__nv_bfloat16><<<grid_for(np, 256), 256, 0, s>>>(flat, pa);
  else
    publish_kernel<float><<<grid_for(np, 256), 256, 0, s>>>(flat, pa);
  return cudaGetLastError() == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

}  // extern "C"

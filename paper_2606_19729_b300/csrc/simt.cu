// CUDA-core (FP32 FMA) kernels: the plain FP32 form of the rollout, the
// belief-update proposal/likelihood pass, the seeded and plain generator
// forward, and the noise fill kernels.
//
// A CTA owns a tile of kSimtRows rows (one row = one (particle, sequence)
// pair, or one batch row) and runs whole MLP chains on it in shared memory:
// activations ping-pong between two [rows][ld] FP32 buffers and every layer
// is y = act(x W^T + b) with the weights read through the read-only cache.
#include "common.cuh"
#include "kernels.h"
#include "simt_mlp.cuh"

namespace voila {

// Writes omega(c0_of_row, c1_of_row, c2) for rows [0, nrows) into columns
// [col0, col0 + dim) of buf. c0/c1 come from the row's (n, k) mapping.
__device__ __forceinline__ void put_noise(float* buf, int ld, int col0, int dim, int nrows,
                                          long long row0, int N, bool rollout_map, uint32_t c2,
                                          uint32_t stream, uint32_t planner, uint32_t k0,
                                          uint32_t k1, uint32_t n_off = 0, uint32_t k_off = 0) {
  const int nblk = (dim + 3) >> 2;
  for (int i = threadIdx.x; i < nrows * nblk; i += blockDim.x) {
    const int r = i / nblk, blk = i % nblk;
    const long long row = row0 + r;
    uint32_t c0, c1;
    if (rollout_map) {
      c0 = (uint32_t)(row % N) + n_off;
      c1 = (uint32_t)(row / N) + k_off;
    } else {
      c0 = (uint32_t)row;
      c1 = 0;
    }
    const float4 z = normal4(k0, k1, c0, c1, c2, stream, planner, (uint32_t)blk);
    const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (blk * 4 + q < dim) buf[r * ld + col0 + blk * 4 + q] = zz[q];
  }
}

// ---------------------------------------------------------------------------
// FP32 rollout: one CTA per tile of rows (row = k * N + n), all H steps.
// ---------------------------------------------------------------------------
template <typename TW, typename TR>
__global__ void __launch_bounds__(kSimtThreads)
rollout_simt_kernel(RolloutArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int ld = a.ld;
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  float* st = bufB + kSimtRows * ld;                      // [rows][d_s]
  double* Gs = reinterpret_cast<double*>(st + kSimtRows * 32);  // [rows]
  const long long rows = (long long)a.N * a.K;
  const long long ntiles = (rows + kSimtRows - 1) / kSimtRows;
  const int d_s = a.d_s, d_a = a.d_a, d_w = a.d_omega;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kSimtRows;
    const int nr = (int)min((long long)kSimtRows, rows - row0);
    __syncthreads();
    for (int i = threadIdx.x; i < kSimtRows * d_s; i += blockDim.x) {
      const int r = i / d_s, d = i % d_s;
      st[r * 32 + d] = (r < nr) ? a.particles[(size_t)((row0 + r) % a.N) * d_s + d] : 0.0f;
    }
    for (int r = threadIdx.x; r < kSimtRows; r += blockDim.x) Gs[r] = 0.0;
    double disc = 1.0;
    for (int t = 0; t < a.H; ++t) {
      __syncthreads();
      // x = [s_t ; a_{k,t} ; omega_T(n, k, t)]
      for (int i = threadIdx.x; i < kSimtRows * (d_s + d_a); i += blockDim.x) {
        const int r = i / (d_s + d_a), c = i % (d_s + d_a);
        float v = 0.0f;
        if (r < nr) {
          if (c < d_s) {
            v = st[r * 32 + c];
          } else {
            const long long k = (row0 + r) / a.N;
            v = a.actions[((size_t)k * a.H + t) * d_a + (c - d_s)];
          }
        }
        bufA[r * ld + c] = v;
      }
      if (d_w > 0)
        put_noise(bufA, ld, d_s + d_a, d_w, nr, row0, a.N, true, (uint32_t)t,
                  VOILA_STREAM_ROLLOUT_OMEGA, a.planner, a.key0, a.key1, a.n_off, a.k_off);
      const float* y = simt_mlp<TW>(a.g, bufA, bufB, ld, nr);
      for (int i = threadIdx.x; i < nr * d_s; i += blockDim.x) {
        const int r = i / d_s, d = i % d_s;
        st[r * 32 + d] = y[r * ld + d];
      }
      __syncthreads();
      if (a.reward_kind == VOILA_REWARD_GOAL) {
        for (int r = threadIdx.x; r < nr; r += blockDim.x) {
          float acc = 0.0f;
          for (int d = 0; d < a.goal_dims; ++d) {
            const float e = st[r * 32 + d] - a.goal[d];
            acc = fmaf(e, e, acc);
          }
          Gs[r] += disc * (double)(-acc);
        }
      } else {
        for (int i = threadIdx.x; i < kSimtRows * (d_s + d_a); i += blockDim.x) {
          const int r = i / (d_s + d_a), c = i % (d_s + d_a);
          float v = 0.0f;
          if (r < nr) {
            if (c < d_s) {
              v = st[r * 32 + c];
            } else {
              const long long k = (row0 + r) / a.N;
              v = a.actions[((size_t)k * a.H + t) * d_a + (c - d_s)];
            }
          }
          bufA[r * ld + c] = v;
        }
        const float* rv = simt_mlp<TR>(a.r, bufA, bufB, ld, nr);
        for (int r = threadIdx.x; r < nr; r += blockDim.x) Gs[r] += disc * (double)rv[r * ld];
      }
      disc *= a.gamma;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += blockDim.x) a.G[row0 + r] = Gs[r];
  }
}

// ---------------------------------------------------------------------------
// Belief-update proposal + likelihood: s'_i = g_T([s_i; a; omega_i]),
// l_i = ell([s'_i; a; o]) or the Gaussian test kind. Writes s' and l.
// ---------------------------------------------------------------------------
template <typename TW, typename TL>
__global__ void __launch_bounds__(kSimtThreads)
belief_propose_kernel(BeliefArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int ld = a.ld;
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  float* sp = bufB + kSimtRows * ld;  // [rows][32]
  const int d_s = a.d_s, d_a = a.d_a, d_o = a.d_o;
  const long long ntiles = ((long long)a.N + kSimtRows - 1) / kSimtRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kSimtRows;
    const int nr = (int)min((long long)kSimtRows, (long long)a.N - row0);
    __syncthreads();
    for (int i = threadIdx.x; i < kSimtRows * (d_s + d_a); i += blockDim.x) {
      const int r = i / (d_s + d_a), c = i % (d_s + d_a);
      float v = 0.0f;
      if (r < nr) v = (c < d_s) ? a.particles[(size_t)(row0 + r) * d_s + c] : a.action[c - d_s];
      bufA[r * ld + c] = v;
    }
    if (a.d_omega > 0)
      put_noise(bufA, ld, d_s + d_a, a.d_omega, nr, row0, 1, false, a.step,
                VOILA_STREAM_BELIEF_OMEGA, a.planner, a.key0, a.key1);
    const float* y = simt_mlp<TW>(a.g, bufA, bufB, ld, nr);
    for (int i = threadIdx.x; i < nr * d_s; i += blockDim.x) {
      const int r = i / d_s, d = i % d_s;
      const float v = y[r * ld + d];
      sp[r * 32 + d] = v;
      a.s_prop[(size_t)(row0 + r) * d_s + d] = v;
    }
    __syncthreads();
    if (a.lik_kind == VOILA_LIK_GAUSSIAN) {
      for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        double acc = 0.0;
        for (int d = 0; d < d_o; ++d) {
          const double e = (double)a.obs[d] - (double)sp[r * 32 + d];
          acc += e * e;
        }
        a.ell[row0 + r] = -acc / (2.0 * (double)a.sigma * (double)a.sigma);
      }
    } else {
      for (int i = threadIdx.x; i < kSimtRows * (d_s + d_a + d_o); i += blockDim.x) {
        const int r = i / (d_s + d_a + d_o), c = i % (d_s + d_a + d_o);
        float v = 0.0f;
        if (r < nr) {
          if (c < d_s) v = sp[r * 32 + c];
          else if (c < d_s + d_a) v = a.action[c - d_s];
          else v = a.obs[c - d_s - d_a];
        }
        bufA[r * ld + c] = v;
      }
      const float* lv = simt_mlp<TL>(a.l, bufA, bufB, ld, nr);
      for (int r = threadIdx.x; r < nr; r += blockDim.x) a.ell[row0 + r] = (double)lv[r * ld];
    }
  }
}

// ---------------------------------------------------------------------------
// Generator forward: plain (X given) or seeded (X = [S; A; omega]).
// ---------------------------------------------------------------------------
template <typename TW>
__global__ void __launch_bounds__(kSimtThreads)
mlp_fwd_kernel(FwdArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int ld = a.ld;
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  const int d_in = a.m.dims[0], d_out = a.m.dims[a.m.n_layers];
  const long long ntiles = ((long long)a.B + kSimtRows - 1) / kSimtRows;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kSimtRows;
    const int nr = (int)min((long long)kSimtRows, (long long)a.B - row0);
    __syncthreads();
    if (a.X) {
      for (int i = threadIdx.x; i < kSimtRows * d_in; i += blockDim.x) {
        const int r = i / d_in, c = i % d_in;
        bufA[r * ld + c] = (r < nr) ? a.X[(size_t)(row0 + r) * d_in + c] : 0.0f;
      }
    } else {
      const int ds = a.d_s, da = a.d_a;
      for (int i = threadIdx.x; i < kSimtRows * (ds + da); i += blockDim.x) {
        const int r = i / (ds + da), c = i % (ds + da);
        float v = 0.0f;
        if (r < nr)
          v = (c < ds) ? a.S[(size_t)(row0 + r) * ds + c]
                       : a.A[(size_t)(row0 + r) * a.a_stride + (c - ds)];
        bufA[r * ld + c] = v;
      }
      if (a.d_omega > 0)
        put_noise(bufA, ld, ds + da, a.d_omega, nr, row0, 1, false, a.step, a.stream_id,
                  a.planner, a.key0, a.key1);
    }
    const float* y = simt_mlp<TW>(a.m, bufA, bufB, ld, nr);
    for (int i = threadIdx.x; i < nr * d_out; i += blockDim.x) {
      const int r = i / d_out, c = i % d_out;
      a.Y[(size_t)(row0 + r) * d_out + c] = y[r * ld + c];
    }
  }
}

// ---------------------------------------------------------------------------
// Noise checks.
// ---------------------------------------------------------------------------
__global__ void philox_fill_kernel(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2,
                                   uint32_t c3, uint32_t* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint4 w = philox(make_uint4((uint32_t)i, c1, c2, c3), k0, k1);
    reinterpret_cast<uint4*>(out)[i] = w;
  }
}

__global__ void normal_fill_kernel(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2,
                                   uint32_t stream, uint32_t planner, int dim, float* out,
                                   long long n) {
  const int nblk = (dim + 3) >> 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * nblk;
       i += (long long)gridDim.x * blockDim.x) {
    const long long row = i / nblk;
    const int blk = (int)(i % nblk);
    const float4 z = normal4(k0, k1, (uint32_t)row, c1, c2, stream, planner, (uint32_t)blk);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    for (int q = 0; q < 4; ++q)
      if (blk * 4 + q < dim) out[row * dim + blk * 4 + q] = zz[q];
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static int simt_grid(long long ntiles, size_t smem) {
  int per_sm = (int)(200 * 1024 / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  long long g = 148LL * per_sm;
  if (g > ntiles) g = ntiles;
  return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// FP32 rollout for small MLPs (generator and reward of two hidden layers at
// most 64 wide, inputs at most 16 wide): a group of TPR = 4 or 8 threads of
// one warp per row (particle, sequence) through all H steps, thread `sub` of
// the group computing hidden units j = TPR i + sub of both hidden layers; the
// units the next layer needs from the other threads arrive by warp shuffles,
// in input order. The weights of both MLPs sit in shared memory, zero padded
// to 64 hidden units and 16 inputs (padding adds exact zero products), rows
// strided so that the group's rows fall in different banks. Every layer
// accumulates in input order from its bias, like the tiled kernel, so both
// group sizes and the tiled kernel give the same bits.
// ---------------------------------------------------------------------------
constexpr int kRowHid = 64, kRowIn = 16, kRowOut = 8;
// Rows a launch of the row kernel holds at once: 4 CTAs of 32 rows per SM (the
// two MLPs' 50 KB of shared memory per CTA allow four).
constexpr long long kRowsOneWave = 148LL * 4 * 32;
constexpr int kRowW0Ld = kRowIn + 4;   // 80-byte rows: a group's rows j = TPR i + sub in distinct banks
constexpr int kRowW1Ld = kRowHid + 4;  // 272-byte rows, likewise
// one MLP in shared memory: W0 [64][20], b0 [64], W1 [64][68], b1 [64], W2 [8][64], b2 [8]
constexpr int kRowMlpFloats =
    kRowHid * kRowW0Ld + kRowHid + kRowHid * kRowW1Ld + kRowHid + kRowOut * kRowHid + kRowOut;

__device__ void load_row_mlp(float* dst, const MlpDev& m) {
  float* W0 = dst;
  float* b0 = W0 + kRowHid * kRowW0Ld;
  float* W1 = b0 + kRowHid;
  float* b1 = W1 + kRowHid * kRowW1Ld;
  float* W2 = b1 + kRowHid;
  float* b2 = W2 + kRowOut * kRowHid;
  const float* w0 = static_cast<const float*>(m.W[0]);
  const float* w1 = static_cast<const float*>(m.W[1]);
  const float* w2 = static_cast<const float*>(m.W[2]);
  const int d0 = m.dims[0], d1 = m.dims[1], d2 = m.dims[2], d3 = m.dims[3];
  for (int i = threadIdx.x; i < kRowHid * kRowW0Ld; i += blockDim.x) {
    const int j = i / kRowW0Ld, k = i % kRowW0Ld;
    W0[i] = (j < d1 && k < d0) ? w0[j * d0 + k] : 0.0f;
  }
  for (int i = threadIdx.x; i < kRowHid * kRowW1Ld; i += blockDim.x) {
    const int j = i / kRowW1Ld, k = i % kRowW1Ld;
    W1[i] = (j < d2 && k < d1) ? w1[j * d1 + k] : 0.0f;
  }
  for (int i = threadIdx.x; i < kRowOut * kRowHid; i += blockDim.x) {
    const int j = i / kRowHid, k = i % kRowHid;
    W2[i] = (j < d3 && k < d2) ? w2[j * d2 + k] : 0.0f;
  }
  for (int i = threadIdx.x; i < kRowHid; i += blockDim.x) {
    b0[i] = i < d1 ? m.b[0][i] : 0.0f;
    b1[i] = i < d2 ? m.b[1][i] : 0.0f;
  }
  for (int i = threadIdx.x; i < kRowOut; i += blockDim.x) b2[i] = i < d3 ? m.b[2][i] : 0.0f;
}

// y[NOUT] = mlp(x) for one row, computed by its group of TPR threads (every
// thread of the group passes the same x and gets the same y); the MLP's
// padded weights at `w`. Thread `sub` of the group computes hidden units
// TPR i + sub; every unit and output accumulates from its bias in input order.
template <int NOUT, int TPR>
__device__ __forceinline__ void group_mlp(const float* __restrict__ w, const float* x, float* y, int act,
                                          unsigned gmask, int gbase, int sub) {
  const float* W0 = w;
  const float* b0 = W0 + kRowHid * kRowW0Ld;
  const float* W1 = b0 + kRowHid;
  const float* b1 = W1 + kRowHid * kRowW1Ld;
  const float* W2 = b1 + kRowHid;
  const float* b2 = W2 + kRowOut * kRowHid;
  constexpr int kPer = kRowHid / TPR;  // hidden units per thread
  float h[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) {  // first hidden layer: units TPR i + sub
    const int j = TPR * i + sub;
    float acc = b0[j];
#pragma unroll
    for (int k = 0; k < kRowIn; k += 4) {
      const float4 wv = *reinterpret_cast<const float4*>(W0 + j * kRowW0Ld + k);
      acc = fmaf(x[k], wv.x, acc);
      acc = fmaf(x[k + 1], wv.y, acc);
      acc = fmaf(x[k + 2], wv.z, acc);
      acc = fmaf(x[k + 3], wv.w, acc);
    }
    h[i] = act_fp32(acc, act);
  }
  float a[kPer];  // second hidden layer, units TPR i + sub
#pragma unroll
  for (int i = 0; i < kPer; ++i) a[i] = b1[TPR * i + sub];
#pragma unroll
  for (int i2 = 0; i2 < kPer; ++i2) {  // inputs TPR i2 .. TPR i2 + TPR - 1, one from each thread of the group
    float hv[TPR];
#pragma unroll
    for (int q = 0; q < TPR; ++q) hv[q] = __shfl_sync(gmask, h[i2], gbase + q);
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
#pragma unroll
      for (int q = 0; q < TPR; q += 4) {
        const float4 wv = *reinterpret_cast<const float4*>(W1 + (TPR * i + sub) * kRowW1Ld + TPR * i2 + q);
        a[i] = fmaf(hv[q], wv.x, a[i]);
        a[i] = fmaf(hv[q + 1], wv.y, a[i]);
        a[i] = fmaf(hv[q + 2], wv.z, a[i]);
        a[i] = fmaf(hv[q + 3], wv.w, a[i]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) a[i] = act_fp32(a[i], act);
#pragma unroll
  for (int m = 0; m < NOUT; ++m) y[m] = b2[m];
#pragma unroll
  for (int i2 = 0; i2 < kPer; ++i2) {  // output layer over all 64 units, in order
    float gv[TPR];
#pragma unroll
    for (int q = 0; q < TPR; ++q) gv[q] = __shfl_sync(gmask, a[i2], gbase + q);
#pragma unroll
    for (int m = 0; m < NOUT; ++m) {
#pragma unroll
      for (int q = 0; q < TPR; q += 4) {
        const float4 wv = *reinterpret_cast<const float4*>(W2 + m * kRowHid + TPR * i2 + q);
        y[m] = fmaf(gv[q], wv.x, y[m]);
        y[m] = fmaf(gv[q + 1], wv.y, y[m]);
        y[m] = fmaf(gv[q + 2], wv.z, y[m]);
        y[m] = fmaf(gv[q + 3], wv.w, y[m]);
      }
    }
  }
}

// TPR threads per row (4 or 8), 32 rows per CTA. Eight threads per row (four
// CTAs per SM, 64 registers) double the warps of a launch whose rows fit in one
// wave; with more rows four threads per row do less work in total (each thread
// of a group computes the output layer in full).
template <int DS, bool RMLP, int TPR>
__global__ void __launch_bounds__(32 * TPR, TPR == 8 ? 4 : 1) rollout_rows_kernel(RolloutArgs a) {
  extern __shared__ __align__(16) float sw[];
  float* gw = sw;
  float* rw = sw + kRowMlpFloats;
  load_row_mlp(gw, a.g);
  if (RMLP) load_row_mlp(rw, a.r);
  __syncthreads();
  const long long rows = (long long)a.N * a.K;
  const int d_a = a.d_a, d_w = a.d_omega;
  const int lane = threadIdx.x & 31, sub = lane & (TPR - 1), gbase = lane & ~(TPR - 1);
  const unsigned gmask = (TPR == 8 ? 0xFFu : 0xFu) << gbase;
  for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TPR; row < rows;
       row += ((long long)gridDim.x * blockDim.x) / TPR) {
    const int n = (int)(row % a.N), k = (int)(row / a.N);
    float s[DS];
#pragma unroll
    for (int i = 0; i < DS; ++i) s[i] = a.particles[(size_t)n * DS + i];
    double G = 0.0, disc = 1.0;
    for (int t = 0; t < a.H; ++t) {
      const float* at = a.actions + ((size_t)k * a.H + t) * d_a;
      float x[kRowIn];
#pragma unroll
      for (int i = 0; i < kRowIn; ++i) x[i] = 0.0f;
#pragma unroll
      for (int i = 0; i < DS; ++i) x[i] = s[i];
#pragma unroll
      for (int i = 0; i < kRowIn - DS; ++i)
        if (i < d_a) x[DS + i] = __ldg(at + i);
#pragma unroll
      for (int b = 0; b < (kRowIn + 3) / 4; ++b)
        if (4 * b < d_w) {
          const float4 z = normal4(a.key0, a.key1, (uint32_t)n + a.n_off, (uint32_t)k + a.k_off, (uint32_t)t,
                                   VOILA_STREAM_ROLLOUT_OMEGA, a.planner, (uint32_t)b);
          const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = DS + d_a + 4 * b + q;  // d_s + d_a + d_omega <= kRowIn
            if (4 * b + q < d_w) {
#pragma unroll
              for (int cc = DS; cc < kRowIn; ++cc)
                if (cc == c) x[cc] = zz[q];
            }
          }
        }
      group_mlp<DS, TPR>(gw, x, s, a.g.act, gmask, gbase, sub);
      float r;
      if (RMLP) {
        float xr[kRowIn];
#pragma unroll
        for (int i = 0; i < kRowIn; ++i) xr[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < DS; ++i) xr[i] = s[i];
#pragma unroll
        for (int i = 0; i < kRowIn - DS; ++i)
          if (i < d_a) xr[DS + i] = __ldg(at + i);
        float rv[1];
        group_mlp<1, TPR>(rw, xr, rv, a.r.act, gmask, gbase, sub);
        r = rv[0];
      } else {
        float acc = 0.0f;
#pragma unroll
        for (int d = 0; d < DS; ++d)
          if (d < a.goal_dims) {
            const float e = s[d] - a.goal[d];
            acc = fmaf(e, e, acc);
          }
        r = -acc;
      }
      G += disc * (double)r;
      disc *= a.gamma;
    }
    if (sub == 0) a.G[row] = G;
  }
}

// The row kernel takes FP32 generators (and reward MLPs) of two hidden layers
// of at most 64 units, inputs of at most 16 and a state of 4 or 8.
static bool rows_kernel_fits(const MlpDev& m, int out) {
  return m.prec == VOILA_FP32 && m.n_layers == 3 && m.dims[0] <= kRowIn && m.dims[1] <= kRowHid &&
         m.dims[2] <= kRowHid && m.dims[3] == out;
}

size_t rollout_simt_smem(int ld) {
  return (size_t)2 * kSimtRows * ld * sizeof(float) + kSimtRows * 32 * sizeof(float) +
         kSimtRows * sizeof(double);
}

cudaError_t launch_rollout_simt(const RolloutArgs& a, cudaStream_t s) {
  const bool rmlp = a.reward_kind == VOILA_REWARD_MLP;
  if ((a.d_s == 4 || a.d_s == 8) && rows_kernel_fits(a.g, a.d_s) && (!rmlp || rows_kernel_fits(a.r, 1)) &&
      (rmlp || a.goal_dims <= a.d_s)) {
    const size_t smem = (size_t)(rmlp ? 2 : 1) * kRowMlpFloats * sizeof(float);
    void (*k)(RolloutArgs);
    const long long rows = (long long)a.N * a.K;
    const int tpr = rows <= kRowsOneWave ? 8 : 4;
    if (tpr == 8) {
      if (a.d_s == 4) k = rmlp ? rollout_rows_kernel<4, true, 8> : rollout_rows_kernel<4, false, 8>;
      else k = rmlp ? rollout_rows_kernel<8, true, 8> : rollout_rows_kernel<8, false, 8>;
    } else {
      if (a.d_s == 4) k = rmlp ? rollout_rows_kernel<4, true, 4> : rollout_rows_kernel<4, false, 4>;
      else k = rmlp ? rollout_rows_kernel<8, true, 4> : rollout_rows_kernel<8, false, 4>;
    }
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    long long grid = (rows + 31) / 32;  // 32 rows per CTA
    if (grid > 148LL * 8) grid = 148LL * 8;
    k<<<(int)grid, 32 * tpr, smem, s>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = rollout_simt_smem(a.ld);
  const long long ntiles = ((long long)a.N * a.K + kSimtRows - 1) / kSimtRows;
  const int grid = simt_grid(ntiles, smem);
  const bool gb = a.g.prec == VOILA_BF16;
  const bool rb = a.reward_kind == VOILA_REWARD_MLP && a.r.prec == VOILA_BF16;
  void (*k)(RolloutArgs);
  if (gb) k = rb ? rollout_simt_kernel<__nv_bfloat16, __nv_bfloat16> : rollout_simt_kernel<__nv_bfloat16, float>;
  else k = rb ? rollout_simt_kernel<float, __nv_bfloat16> : rollout_simt_kernel<float, float>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kSimtThreads, smem, s>>>(a);
  return cudaGetLastError();
}

size_t belief_propose_smem(int ld) {
  return (size_t)2 * kSimtRows * ld * sizeof(float) + kSimtRows * 32 * sizeof(float);
}

cudaError_t launch_belief_propose(const BeliefArgs& a, cudaStream_t s) {
  const size_t smem = belief_propose_smem(a.ld);
  const long long ntiles = ((long long)a.N + kSimtRows - 1) / kSimtRows;
  const int grid = simt_grid(ntiles, smem);
  const bool gb = a.g.prec == VOILA_BF16;
  const bool lb = a.lik_kind == VOILA_LIK_MLP && a.l.prec == VOILA_BF16;
  void (*k)(BeliefArgs);
  if (gb) k = lb ? belief_propose_kernel<__nv_bfloat16, __nv_bfloat16> : belief_propose_kernel<__nv_bfloat16, float>;
  else k = lb ? belief_propose_kernel<float, __nv_bfloat16> : belief_propose_kernel<float, float>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kSimtThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mlp_fwd(const FwdArgs& a, cudaStream_t s) {
  const size_t smem = (size_t)2 * kSimtRows * a.ld * sizeof(float);
  const long long ntiles = ((long long)a.B + kSimtRows - 1) / kSimtRows;
  const int grid = simt_grid(ntiles, smem);
  void (*k)(FwdArgs) = a.m.prec == VOILA_BF16 ? mlp_fwd_kernel<__nv_bfloat16> : mlp_fwd_kernel<float>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kSimtThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_philox_fill(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3,
                               uint32_t* out, long long n, cudaStream_t s) {
  long long g = (n + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  if (g < 1) g = 1;
  philox_fill_kernel<<<(int)g, 256, 0, s>>>(k0, k1, c1, c2, c3, out, n);
  return cudaGetLastError();
}

cudaError_t launch_normal_fill(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2,
                               uint32_t stream, uint32_t planner, int dim, float* out,
                               long long n, cudaStream_t s) {
  long long g = (n * ((dim + 3) / 4) + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  if (g < 1) g = 1;
  normal_fill_kernel<<<(int)g, 256, 0, s>>>(k0, k1, c1, c2, stream, planner, dim, out, n);
  return cudaGetLastError();
}

}  // namespace voila

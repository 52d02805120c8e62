// Log-weight normalisation, exact FP64 prefix sum, systematic resampling and
// gather (SIR step of Sec. 3; weights exp(l / lambda), Sec. 4.2.3), plus the
// deterministic per-sequence return reduction J_k = sum_n w_n G_{n,k}.
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace voila {

constexpr int kResampleThreads = 1024;

// Exclusive scan of one double per thread. The inputs are multiples of 2^-52
// whose partial sums stay below 2, so every addition is exact and the result
// does not depend on the order.
__device__ double block_exclusive_scan(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  __syncthreads();
  if (lane == 31) red[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < nw) red[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const double warp_off = (wid > 0) ? red[wid - 1] : 0.0;
  return warp_off + inc - v;
}

// Tempered log-weight lw_i = l_i / lambda + logw_i (Sec. 4.2.3) in FP32: the
// weights' arithmetic runs in FP32; FP64 holds only their sum, the normalised
// quantised weights and the exact prefix sum that drives the resampling.
__device__ __forceinline__ float log_weight(const ResampleArgs& a, int i) {
  float lw = __fdiv_rn((float)a.ell[i], (float)a.lambda);
  if (a.logw) lw = __fadd_rn(lw, (float)a.logw[i]);
  return lw;
}

__global__ void __launch_bounds__(kResampleThreads) belief_resample_kernel(ResampleArgs a) {
  __shared__ double red[33];
  __shared__ int bad_s;
  const int N = a.N, nt = blockDim.x, tid = threadIdx.x;
  const int chunk = (N + nt - 1) / nt;
  const int i0 = min(N, tid * chunk), i1 = min(N, i0 + chunk);
  if (tid == 0) bad_s = 0;
  __syncthreads();
  // lw_i = l_i / lambda + logw_i (FP32)
  float lmax = -INFINITY;
  int bad = 0;
  for (int i = i0; i < i1; ++i) {
    const float lw = log_weight(a, i);
    a.C[i] = (double)lw;
    if (isnan(lw) || lw == INFINITY) bad = 1;
    lmax = fmaxf(lmax, lw);
  }
  if (bad) atomicOr(&bad_s, 1);
  const double m = block_max((double)lmax, red);  // an FP32 value
  if (bad_s) {
    if (tid == 0) set_status(a.hdr, VOILA_ERR_NONFINITE, 1);
    return;
  }
  if (m == -INFINITY) {
    if (tid == 0) set_status(a.hdr, VOILA_ERR_DEGENERATE, 1);
    return;
  }
  // e_i = exp(lw_i - m) in FP32, Z = sum e_i in FP64
  double zl = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double e = (double)expf((float)a.C[i] - (float)m);
    a.C[i] = e;
    zl += e;
  }
  const double Z = block_sum(zl, red);
  // q_i = rn(w_i 2^52) 2^-52 and the local inclusive prefix
  double acc = 0.0, q2 = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double w = __ddiv_rn(a.C[i], Z);
    const double q = rint(w * 4503599627370496.0) * 2.220446049250313e-16;
    if (a.w_out) a.w_out[i] = q;
    acc += q;
    q2 += q * q;
    a.C[i] = acc;
  }
  const double off = block_exclusive_scan(acc, red);
  for (int i = i0; i < i1; ++i) a.C[i] += off;
  const double sq = block_sum(q2, red);  // ends with __syncthreads: C is complete
  const double total = a.C[N - 1];
  const uint4 wd = philox(make_uint4(0u, 0u, a.step, ctr_word3(VOILA_STREAM_RESAMPLE, a.planner, 0)),
                          a.key0, a.key1);
  const double u0 = uniform53(wd.x, wd.y);
  const double dN = (double)N;
  for (int j = i0; j < i1; ++j) {
    const double p = __ddiv_rn(__dmul_rn(__dadd_rn(u0, (double)j), total), dN);
    int lo = 0, hi = N;  // first i with C_i > p
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a.C[mid] > p) hi = mid;
      else lo = mid + 1;
    }
    const int idx = lo < N ? lo : N - 1;
    if (a.idx_out) a.idx_out[j] = idx;
    for (int d = 0; d < a.d_s; ++d)
      a.particles_out[(size_t)j * a.d_s + d] = a.s_prop[(size_t)idx * a.d_s + d];
  }
  if (tid == 0) {
    if (a.logZ_out) *a.logZ_out = m + log(Z);
    if (a.ess_out) *a.ess_out = 1.0 / sq;
  }
}

// ---------------------------------------------------------------------------
// Many-CTA form (N > kResampleSingleCta; measured faster from 4096 particles
// up, mostly from the parallel search and gather): segment b = particles
// [b S, (b + 1) S), S = kResampleSegElems, one CTA each; thread t of a
// segment owns four consecutive particles. The segment partials (maximum,
// non-finite flag, sum of exponentials, total of the quantised weights, sum
// of their squares) go to a.part, and every CTA of a later launch combines
// them in segment order, so all CTAs see the same m and Z and the result does
// not depend on scheduling. The prefix sums stay segment-local: the quantised
// weights are multiples of 2^-52 with partial sums below 2, so
// C_i = (exclusive segment offset) + (local prefix) is exact, and the search
// first finds the segment, then the index inside it.
// ---------------------------------------------------------------------------
constexpr int kSegThreads = kResampleSegElems / 4;
enum { kPartMax = 0, kPartBad = 1, kPartZ = 2, kPartTotal = 3, kPartSq = 4 };

__device__ __forceinline__ double part_at(const ResampleArgs& a, int which, int seg) {
  return a.part[which * kResampleMaxSegs + seg];
}

// Global maximum and non-finite flag from the segment partials, in segment order.
__device__ __forceinline__ void combine_max(const ResampleArgs& a, int G, double& m, bool& bad) {
  m = -INFINITY;
  bad = false;
  for (int b = 0; b < G; ++b) {
    m = fmax(m, part_at(a, kPartMax, b));
    bad = bad || part_at(a, kPartBad, b) != 0.0;
  }
}

__global__ void __launch_bounds__(kSegThreads) resample_seg_max_kernel(ResampleArgs a) {
  __shared__ double red[33];
  const int b = blockIdx.x;
  const int s1 = min(a.N, (b + 1) * kResampleSegElems);
  const int i0 = min(s1, b * kResampleSegElems + 4 * (int)threadIdx.x), i1 = min(s1, i0 + 4);
  float lmax = -INFINITY;
  double bad = 0.0;
  for (int i = i0; i < i1; ++i) {
    const float lw = log_weight(a, i);
    a.C[i] = (double)lw;
    if (isnan(lw) || lw == INFINITY) bad = 1.0;
    lmax = fmaxf(lmax, lw);
  }
  const double m = block_max((double)lmax, red);
  const double f = block_max(bad, red);
  if (threadIdx.x == 0) {
    a.part[kPartMax * kResampleMaxSegs + b] = m;
    a.part[kPartBad * kResampleMaxSegs + b] = f;
  }
}

__global__ void __launch_bounds__(kSegThreads) resample_seg_exp_kernel(ResampleArgs a) {
  __shared__ double red[33];
  double m;
  bool bad;
  combine_max(a, gridDim.x, m, bad);
  if (bad || m == -INFINITY) {
    if (blockIdx.x == 0 && threadIdx.x == 0)
      set_status(a.hdr, bad ? VOILA_ERR_NONFINITE : VOILA_ERR_DEGENERATE, 1);
    return;
  }
  const int b = blockIdx.x;
  const int s1 = min(a.N, (b + 1) * kResampleSegElems);
  const int i0 = min(s1, b * kResampleSegElems + 4 * (int)threadIdx.x), i1 = min(s1, i0 + 4);
  double zl = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double e = (double)expf((float)a.C[i] - (float)m);
    a.C[i] = e;
    zl += e;
  }
  const double z = block_sum(zl, red);
  if (threadIdx.x == 0) a.part[kPartZ * kResampleMaxSegs + b] = z;
}

__global__ void __launch_bounds__(kSegThreads) resample_seg_scan_kernel(ResampleArgs a) {
  __shared__ double red[33];
  double m;
  bool bad;
  combine_max(a, gridDim.x, m, bad);
  if (bad || m == -INFINITY) return;
  double Z = 0.0;
  for (int s = 0; s < (int)gridDim.x; ++s) Z += part_at(a, kPartZ, s);
  const int b = blockIdx.x;
  const int s1 = min(a.N, (b + 1) * kResampleSegElems);
  const int i0 = min(s1, b * kResampleSegElems + 4 * (int)threadIdx.x), i1 = min(s1, i0 + 4);
  double acc = 0.0, q2 = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double w = __ddiv_rn(a.C[i], Z);
    const double q = rint(w * 4503599627370496.0) * 2.220446049250313e-16;
    if (a.w_out) a.w_out[i] = q;
    acc += q;
    q2 += q * q;
    a.C[i] = acc;
  }
  const double off = block_exclusive_scan(acc, red);
  for (int i = i0; i < i1; ++i) a.C[i] += off;  // segment-local inclusive prefix
  const double tot = block_sum(acc, red);       // exact: every partial sum is representable
  const double sq = block_sum(q2, red);
  if (threadIdx.x == 0) {
    a.part[kPartTotal * kResampleMaxSegs + b] = tot;
    a.part[kPartSq * kResampleMaxSegs + b] = sq;
  }
}

constexpr int kSearchThreads = 256;

__global__ void __launch_bounds__(kSearchThreads) resample_seg_search_kernel(ResampleArgs a, int G) {
  __shared__ double segoff[kResampleMaxSegs + 1];  // exclusive offsets; segoff[G] = C_{N-1}
  __shared__ int stop_s;
  if (threadIdx.x == 0) {
    double m;
    bool bad;
    combine_max(a, G, m, bad);
    stop_s = bad || m == -INFINITY;
    if (!stop_s) {
      double acc = 0.0;
      for (int s = 0; s < G; ++s) {
        segoff[s] = acc;
        acc += part_at(a, kPartTotal, s);
      }
      segoff[G] = acc;
      if (blockIdx.x == 0) {
        double Z = 0.0, sq = 0.0;
        for (int s = 0; s < G; ++s) {
          Z += part_at(a, kPartZ, s);
          sq += part_at(a, kPartSq, s);
        }
        if (a.logZ_out) *a.logZ_out = m + log(Z);
        if (a.ess_out) *a.ess_out = 1.0 / sq;
      }
    }
  }
  __syncthreads();
  if (stop_s) return;
  const int N = a.N;
  const int j = blockIdx.x * kSearchThreads + threadIdx.x;
  if (j >= N) return;
  const double total = segoff[G];
  const uint4 wd = philox(make_uint4(0u, 0u, a.step, ctr_word3(VOILA_STREAM_RESAMPLE, a.planner, 0)),
                          a.key0, a.key1);
  const double u0 = uniform53(wd.x, wd.y);
  const double p = __ddiv_rn(__dmul_rn(__dadd_rn(u0, (double)j), total), (double)N);
  int lo = 0, hi = G;  // first segment whose end prefix exceeds p
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (segoff[mid + 1] > p) hi = mid;
    else lo = mid + 1;
  }
  int idx = N - 1;
  if (lo < G) {
    const double base = segoff[lo];
    int l2 = lo * kResampleSegElems, h2 = min(N, (lo + 1) * kResampleSegElems);
    const int end = h2;
    while (l2 < h2) {  // first i of the segment with base + C_i > p
      const int mid = (l2 + h2) >> 1;
      if (base + a.C[mid] > p) h2 = mid;
      else l2 = mid + 1;
    }
    idx = l2 < end ? l2 : N - 1;
  }
  if (a.idx_out) a.idx_out[j] = idx;
  for (int d = 0; d < a.d_s; ++d) a.particles_out[(size_t)j * a.d_s + d] = a.s_prop[(size_t)idx * a.d_s + d];
}

cudaError_t launch_belief_resample(const ResampleArgs& a, cudaStream_t s) {
  if (a.N <= kResampleSingleCta) {
    belief_resample_kernel<<<1, kResampleThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  const int G = (a.N + kResampleSegElems - 1) / kResampleSegElems;
  if (G > kResampleMaxSegs || !a.part) return cudaErrorInvalidValue;
  resample_seg_max_kernel<<<G, kSegThreads, 0, s>>>(a);
  resample_seg_exp_kernel<<<G, kSegThreads, 0, s>>>(a);
  resample_seg_scan_kernel<<<G, kSegThreads, 0, s>>>(a);
  resample_seg_search_kernel<<<(a.N + kSearchThreads - 1) / kSearchThreads, kSearchThreads, 0, s>>>(a, G);
  return cudaGetLastError();
}

// J_k = sum_n w_n G[k][n]: one CTA per sequence, fixed summation order;
// without w every particle weighs 1 / N_total (N_total = N unless the call is
// one particle shard of a larger problem). A J_k that is NaN or infinite (a
// non-finite weight, particle, action or model output reached it) latches
// VOILA_ERR_NONFINITE in the workspace status word.
__global__ void __launch_bounds__(256) reduce_returns_kernel(const double* __restrict__ G,
                                                             const double* __restrict__ w, int N,
                                                             int N_total, int K, double* __restrict__ J,
                                                             WsHeader* hdr) {
  __shared__ double red[33];
  const int k = blockIdx.x;
  const double invN = 1.0 / (double)N_total;
  double acc = 0.0;
  const double* g = G + (size_t)k * N;
  for (int n = threadIdx.x; n < N; n += blockDim.x) acc += g[n] * (w ? w[n] : invN);
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) {
    J[k] = tot;
    if (!isfinite(tot)) set_status(hdr, VOILA_ERR_NONFINITE, kWhereReturns);
  }
}

// argmax_k J_k, lowest index on ties (NaN never wins).
__global__ void __launch_bounds__(1024) argmax_kernel(const double* __restrict__ J, int K,
                                                      int32_t* best) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  double v = -INFINITY;
  int i = K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double x = J[k];
    if (!isnan(x) && (i == K || x > v)) {  // k rises: ties keep the lower index
      v = x;
      i = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    bv[wid] = v;
    bi[wid] = i;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? bv[lane] : -INFINITY;
    i = lane < nw ? bi[lane] : K;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
      }
    }
    if (lane == 0) *best = (i < K) ? i : 0;
  }
}

// All planners of a batched rollout in one launch: block b is sequence
// b - k_start(q) of planner q (fixed summation order, as above).
__global__ void __launch_bounds__(256) reduce_returns_batched_kernel(const __grid_constant__ BatchedReduceArgs a) {
  __shared__ double red[33];
  const long long b = blockIdx.x;
  int q = 0;
  while (q < a.P - 1 && b >= a.k_end[q]) ++q;
  const int k = (int)(b - (q ? a.k_end[q - 1] : 0));
  const int N = a.N[q];
  const double invN = 1.0 / (double)N;
  const double* g = a.G[q] + (size_t)k * N;
  const double* w = a.w[q];
  double acc = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x) acc += g[n] * (w ? w[n] : invN);
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) {
    a.J[q][k] = tot;
    if (!isfinite(tot)) set_status(a.hdr, VOILA_ERR_NONFINITE, kWhereReturns);
  }
}

__global__ void __launch_bounds__(1024) argmax_batched_kernel(const __grid_constant__ BatchedReduceArgs a) {
  const int q = blockIdx.x;
  if (a.best[q] == nullptr) return;
  __shared__ double bv[32];
  __shared__ int bi[32];
  const int K = a.K[q];
  const double* J = a.J[q];
  double v = -INFINITY;
  int i = K;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double x = J[k];
    if (!isnan(x) && (i == K || x > v)) {
      v = x;
      i = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    bv[wid] = v;
    bi[wid] = i;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? bv[lane] : -INFINITY;
    i = lane < nw ? bi[lane] : K;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, i, o);
      if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
      }
    }
    if (lane == 0) *a.best[q] = (i < K) ? i : 0;
  }
}

cudaError_t launch_reduce_returns_batched(const BatchedReduceArgs& a, cudaStream_t s) {
  const long long blocks = a.k_end[a.P - 1];
  if (blocks <= 0) return cudaSuccess;
  reduce_returns_batched_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  argmax_batched_kernel<<<a.P, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce_returns(const double* G, const double* w, int N, int N_total, int K, double* J,
                                  int32_t* best_k, WsHeader* hdr, cudaStream_t s) {
  reduce_returns_kernel<<<K, 256, 0, s>>>(G, w, N, N_total, K, J, hdr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !best_k) return e;
  argmax_kernel<<<1, 1024, 0, s>>>(J, K, best_k);
  return cudaGetLastError();
}

}  // namespace voila

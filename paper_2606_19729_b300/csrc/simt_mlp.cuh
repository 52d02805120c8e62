// The shared-memory MLP tile of the CUDA-core kernels: a CTA holds
// kSimtRows rows in two [rows][ld] FP32 buffers and runs y = act(x W^T + b)
// layer by layer, weights through the read-only cache.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace voila {

// One layer on a tile held in shared memory. Threads are split into
// `ng` row groups x `cpp` columns; a thread owns column j (stride cpp) and
// rows rg, rg+ng, ... so narrow layers still keep most threads busy.
template <typename TW>
__device__ void simt_layer(const float* __restrict__ in, float* __restrict__ out, int ld,
                           int nrows, int K, int Nout, const TW* __restrict__ W,
                           const float* __restrict__ b, int act, bool last) {
  const int nt = blockDim.x, tid = threadIdx.x;
  int ng = nt / Nout;
  if (ng < 1) ng = 1;
  if (ng > kSimtRows) ng = kSimtRows;
  const int cpp = nt / ng;
  const int j0 = tid % cpp, rg = tid / cpp;
  if (rg >= ng) return;
  const int nr = (nrows - rg + ng - 1) / ng;  // rows this thread owns
  for (int j = j0; j < Nout; j += cpp) {
    float acc[kSimtRows];
    const float bj = __ldg(b + j);
#pragma unroll
    for (int i = 0; i < kSimtRows; ++i) acc[i] = bj;
    const TW* wj = W + (size_t)j * K;
    for (int k = 0; k < K; ++k) {
      const float wv = ldw<TW>(wj + k);
#pragma unroll
      for (int i = 0; i < kSimtRows; ++i)
        if (i < nr) acc[i] = fmaf(in[(rg + i * ng) * ld + k], wv, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < kSimtRows; ++i)
      if (i < nr) out[(rg + i * ng) * ld + j] = last ? acc[i] : act_fp32(acc[i], act);
  }
}

// Runs all layers; returns the buffer holding the output.
template <typename TW>
__device__ float* simt_mlp(const MlpDev& m, float* bufA, float* bufB, int ld, int nrows) {
  float* cur = bufA;
  float* nxt = bufB;
  for (int l = 0; l < m.n_layers; ++l) {
    __syncthreads();
    simt_layer<TW>(cur, nxt, ld, nrows, m.dims[l], m.dims[l + 1],
                   reinterpret_cast<const TW*>(m.W[l]), m.b[l], m.act, l == m.n_layers - 1);
    float* t = cur;
    cur = nxt;
    nxt = t;
  }
  __syncthreads();
  return cur;
}

}  // namespace voila

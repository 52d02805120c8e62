// The shared-memory MLP tile of the CUDA-core kernels: a CTA holds
// kSimtRows rows in two [rows][ld] FP32 buffers and runs y = act(x W^T + b)
// layer by layer, weights through the read-only cache.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace voila {

// Row stride of the [rows][ld] activation buffers for layers up to maxw wide:
// a multiple of 4 (16-byte rows for float4 loads) that is 4 mod 32, so the
// rows that different threads of a warp read start in different banks.
inline int simt_ld(int maxw) { return (maxw + 31) / 32 * 32 + 4; }

// Four consecutive weights W[k .. k + 3] (16 or 8 bytes, aligned when K % 4 == 0).
template <typename TW>
__device__ __forceinline__ void ldw4(const TW* p, float* w);
template <>
__device__ __forceinline__ void ldw4<float>(const float* p, float* w) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  w[0] = v.x;
  w[1] = v.y;
  w[2] = v.z;
  w[3] = v.w;
}
template <>
__device__ __forceinline__ void ldw4<__nv_bfloat16>(const __nv_bfloat16* p, float* w) {
  const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
  w[0] = __uint_as_float(v.x << 16);
  w[1] = __uint_as_float(v.x & 0xffff0000u);
  w[2] = __uint_as_float(v.y << 16);
  w[3] = __uint_as_float(v.y & 0xffff0000u);
}

// One layer on a tile held in shared memory. Threads are split into
// `ng` row groups x `cpp` columns; a thread owns column j (stride cpp) and
// rows rg, rg+ng, ... so narrow layers still keep most threads busy. When K
// is a multiple of 4, four K values are read per 16-byte shared load and
// four weights per global load (four FMAs per row and load).
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
    int k = 0;
    if ((K & 3) == 0) {
      for (; k < K; k += 4) {
        float w[4];
        ldw4<TW>(wj + k, w);
#pragma unroll
        for (int i = 0; i < kSimtRows; ++i)
          if (i < nr) {
            const float4 x = *reinterpret_cast<const float4*>(in + (rg + i * ng) * ld + k);
            acc[i] = fmaf(x.x, w[0], acc[i]);
            acc[i] = fmaf(x.y, w[1], acc[i]);
            acc[i] = fmaf(x.z, w[2], acc[i]);
            acc[i] = fmaf(x.w, w[3], acc[i]);
          }
      }
    }
    for (; k < K; ++k) {
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

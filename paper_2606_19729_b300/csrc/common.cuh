// Device helpers shared by the VOiLA kernels: Philox4x32-10, uniforms,
// Box-Muller normals, activations and the device-side model descriptors.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/voila.h"

namespace voila {

// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11): one round maps
// (c0, c1, c2, c3) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)); the key is bumped by the Weyl constants between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

__host__ __device__ __forceinline__ uint32_t ctr_word3(uint32_t stream, uint32_t planner,
                                                       uint32_t block) {
  return (stream << 28) | (planner << 12) | block;
}

// (2 * (x >> 9) + 1) * 2^-24: a 24-bit odd integer times a power of two,
// exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float uniform24(uint32_t x) {
  return (float)((x >> 9) * 2u + 1u) * 5.9604644775390625e-8f;
}

// 53-bit uniform in [0, 1) from two words: ((x0 << 21) | (x1 >> 11)) * 2^-53.
__device__ __forceinline__ double uniform53(uint32_t x0, uint32_t x1) {
  const unsigned long long m = ((unsigned long long)x0 << 21) | (unsigned long long)(x1 >> 11);
  return (double)m * 1.1102230246251565e-16;
}

// Box-Muller (1958): (r cos 2 pi ub, r sin 2 pi ub), r = sqrt(-2 ln ua).
__device__ __forceinline__ void box_muller(float ua, float ub, float& z0, float& z1) {
  const float r = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Four normals of block `block` at counter (c0, c1, c2) of `stream`.
__device__ __forceinline__ float4 normal4(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                          uint32_t c2, uint32_t stream, uint32_t planner,
                                          uint32_t block) {
  const uint4 w = philox(make_uint4(c0, c1, c2, ctr_word3(stream, planner, block)), k0, k1);
  float4 z;
  box_muller(uniform24(w.x), uniform24(w.y), z.x, z.y);
  box_muller(uniform24(w.z), uniform24(w.w), z.z, z.w);
  return z;
}

// Activations in FP32 (accurate library forms; the last layer is linear).
__device__ __forceinline__ float act_fp32(float h, int act) {
  if (act == VOILA_ACT_TANH) return tanhf(h);
  if (act == VOILA_ACT_SILU) return h / (1.0f + expf(-h));
  return h;
}

// Device copy of a voila_mlp (passed by value as a kernel argument).
struct MlpDev {
  int n_layers;
  int act;
  int prec;
  int dims[VOILA_MAX_LAYERS + 1];
  const void* W[VOILA_MAX_LAYERS];
  const float* b[VOILA_MAX_LAYERS];
};

template <typename TW>
__device__ __forceinline__ float ldw(const TW* p);
template <>
__device__ __forceinline__ float ldw<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ldw<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// Status word in the first 16 bytes of every workspace.
struct WsHeader {
  int32_t status;
  int32_t where;
  int32_t pad[2];
};

__device__ __forceinline__ void set_status(WsHeader* h, int32_t code, int32_t where) {
  if (h) {
    atomicCAS(&h->status, 0, code);
    h->where = where;
  }
}

}  // namespace voila

// BF16 tensor-core GEMM with the epilogues of MLP training (tcgen05, TMA).
//
// D[M][N] = A[M][K] . B[N][K]^T, A and B BF16 K-major (row-major [rows][K]),
// FP32 accumulation in TMEM; a work unit is a 128-row tile over all N <= 256
// columns and a range of K (split-K), persistent CTAs (one per SM) take units
// in turn with two accumulators in TMEM. Warp 0 streams A and B
// K-chunks of 64 (128-byte rows, 128B swizzle) into a 3-stage ring with TMA,
// warp 1 issues the MMAs (M = 128, N, K = 16) from one thread, warps 2-17 read
// the accumulator (warp w owns TMEM lanes 32 (w mod 4) .. +31, one row per
// thread; the four warps of a lane quadrant split the columns) and run one of
// the epilogues:
//   kFwdHidden  z = acc + b;  H = act(z), AD = act'(z) row-major, H^T via
//               a shared-memory transpose (BF16);
//   kFwdOut     Y = acc + b (FP32, the first n_real columns);
//   kBwd        delta = acc * AD_in;  D row-major and D^T (BF16);
//   kPartial    P[split][m][n] = acc (FP32), summed later in split order.
// Every wait is bounded; on expiry the kernel records VOILA_ERR_TIMEOUT,
// waits (bounded) for its copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include "../../include/voila.h"
#include "common.cuh"
#include "gemm.h"
#include "tc_ptx.cuh"

namespace voila {
namespace {

constexpr int kGThreads = 576;  // producer warp, MMA warp, 16 epilogue warps
constexpr int kGEpiThreads = 512;
constexpr int kGStages = 3;
constexpr int kGABytes = 128 * 128;  // 128 rows x 64 BF16
constexpr int kGBBytes = 256 * 128;  // up to 256 rows x 64 BF16
constexpr int kGStageBytes = 256 * 128 * 2;  // transposed staging: [N <= 256][128 rows] BF16
constexpr long long kGSpin = 4000000000LL;

struct GemmParams {
  CUtensorMap ta, tb;
  int M, N;           // rows of A (valid rows), columns of D (MMA N, multiple of 16, <= 256)
  int n_real;         // columns stored by kFwdOut / kPartial-transposed users
  int kchunks;        // K chunks of 64 per unit (K split)
  int splits;         // K splits
  int mode, act;
  uint32_t bbytes;    // bytes of one B chunk (N rows x 128 B)
  const float* bias;
  __nv_bfloat16* H;   // [M][N]
  __nv_bfloat16* AD;  // [M][N]
  __nv_bfloat16* HT;  // [N][ldT]
  const __nv_bfloat16* AD_in;
  float* Y;
  int ldY;
  float* P;           // [splits][M][N]
  int ldT;
  WsHeader* hdr;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool gwait(uint32_t bar, uint32_t parity, volatile int* abort_flag, WsHeader* hdr,
                                      int where) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kGSpin) {
      *abort_flag = 1;
      set_status(hdr, VOILA_ERR_TIMEOUT, where);
      return false;
    }
  }
}

__device__ __forceinline__ void act_and_grad(float z, int act, float& h, float& d) {
  if (act == VOILA_ACT_SILU) {
    const float sg = __fdividef(1.0f, 1.0f + __expf(-z));
    h = z * sg;
    d = sg * (1.0f + z * (1.0f - sg));
  } else if (act == VOILA_ACT_TANH) {
    h = tanhf(z);
    d = 1.0f - h * h;
  } else {
    h = z;
    d = 1.0f;
  }
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi) { return ptx::pack_bf16x2(lo, hi); }

// Persistent: each CTA takes work units u = blockIdx.x, + gridDim.x, ... (unit =
// 128-row tile x K split). Two FP32 accumulators in TMEM (columns [0, 256) and
// [256, 512)) let the MMAs of a CTA's next unit run while the epilogue warps
// drain the previous one; the producer streams the next unit's chunks into the
// ring meanwhile. The transposed outputs go through their own staging buffer.
__global__ void __launch_bounds__(kGThreads, 1) gemm_tc_kernel(const __grid_constant__ GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* ringA = smem;
  uint8_t* ringB = smem + kGStages * kGABytes;
  __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(ringB + kGStages * kGBBytes);  // [N][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(stage) + kGStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + kGStages;
  uint64_t* accf = bars + 2 * kGStages;      // [2] accumulator b holds a finished unit
  uint64_t* acce = bars + 2 * kGStages + 2;  // [2] accumulator b has been read out
  uint64_t* drain = bars + 2 * kGStages + 4;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kGStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  float* bias_s = reinterpret_cast<float*>(bars + 2 * kGStages + 6);  // [256]: the epilogue's bias reads
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = (p.M + 127) / 128;
  const long long units = (long long)tiles * p.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGStages; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_u32(&accf[b]), 1);
      ptx::mbar_init(ptx::smem_u32(&acce[b]), kGEpiThreads / 32);  // every epilogue warp
    }
    ptx::mbar_init(ptx::smem_u32(drain), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (p.bias)
    for (int i = threadIdx.x; i < p.N; i += blockDim.x) bias_s[i] = p.bias[i];
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      ptx::prefetch_tmap(&p.ta);
      ptx::prefetch_tmap(&p.tb);
      int last[kGStages];
      for (int s = 0; s < kGStages; ++s) last[s] = -1;
      bool ok = true;
      long long c = 0;  // chunks loaded by this CTA
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int m0 = (int)(u % tiles) * 128, kc0 = (int)(u / tiles) * p.kchunks;
        for (int j = 0; j < p.kchunks && ok; ++j, ++c) {
          const int slot = (int)(c % kGStages);
          const uint32_t phase = (uint32_t)(c / kGStages) & 1u;
          if (!gwait(ptx::smem_u32(&empty[slot]), phase ^ 1u, abort_flag, p.hdr, 70)) {
            ok = false;
            break;
          }
          const uint32_t fb = ptx::smem_u32(&full[slot]);
          ptx::mbar_arrive_expect_tx(fb, (uint32_t)kGABytes + p.bbytes);
          tma_load_2d(ptx::smem_u32(ringA + slot * kGABytes), &p.ta, (kc0 + j) * 64, m0, fb);
          tma_load_2d(ptx::smem_u32(ringB + slot * kGBBytes), &p.tb, (kc0 + j) * 64, 0, fb);
          last[slot] = (int)phase;
        }
      }
      if (!ok) {  // loads still in flight complete before shared memory goes away
        for (int s = 0; s < kGStages; ++s)
          if (last[s] >= 0) {
            const long long t0 = clock64();
            while (!ptx::mbar_try_wait(ptx::smem_u32(&full[s]), (uint32_t)last[s]) && clock64() - t0 < kGSpin) {
            }
          }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = ptx::idesc_bf16(128, p.N);
      bool ok = true;
      long long c = 0;
      int k = 0;  // units of this CTA
      for (long long u = blockIdx.x; u < units && ok; u += gridDim.x, ++k) {
        const int b = k & 1;
        // the epilogue has read this accumulator's previous unit (two units ago)
        if (k >= 2 && !gwait(ptx::smem_u32(&acce[b]), (uint32_t)((k - 2) >> 1) & 1u, abort_flag, p.hdr, 73)) {
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * 256);
        for (int j = 0; j < p.kchunks && ok; ++j, ++c) {
          const int slot = (int)(c % kGStages);
          const uint32_t phase = (uint32_t)(c / kGStages) & 1u;
          if (!gwait(ptx::smem_u32(&full[slot]), phase, abort_flag, p.hdr, 71)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint64_t ad = ptx::smem_desc(ptx::smem_u32(ringA + slot * kGABytes), 1024, ptx::kSwizzle128B);
          const uint64_t bd = ptx::smem_desc(ptx::smem_u32(ringB + slot * kGBBytes), 1024, ptx::kSwizzle128B);
          const uint32_t ahi = (uint32_t)(ad >> 32), alo = (uint32_t)ad;
          const uint32_t bhi = (uint32_t)(bd >> 32), blo = (uint32_t)bd;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)  // K = 16 per MMA: +32 bytes (+2 in the address field)
            ptx::mma_bf16(d, ptx::desc_with_lo(ahi, alo + 2 * kk), ptx::desc_with_lo(bhi, blo + 2 * kk), idesc,
                          (j | kk) ? 1u : 0u);
          ptx::mma_commit(ptx::smem_u32(&empty[slot]));
        }
        ptx::mma_commit(ptx::smem_u32(&accf[b]));  // this unit's MMAs (or none) have completed
      }
      // every MMA issued (also after an abort) completes before TMEM is freed
      ptx::mma_commit(ptx::smem_u32(drain));
      const long long t0 = clock64();
      while (!ptx::mbar_try_wait(ptx::smem_u32(drain), 0) && clock64() - t0 < kGSpin) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int slice = (warp - 2) >> 2;  // column quarter of this warp
    const int r = 32 * q + lane;
    const int cps = p.N >= 64 ? p.N / 4 : 16;  // columns per slice (multiples of 16)
    const int c_lo = slice * cps, c_hi = c_lo + cps < p.N ? c_lo + cps : p.N;
    const bool transpose = p.mode == kGemmFwdHidden || p.mode == kGemmBwd;
    bool ok = true;
    int k = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++k) {
      const int b = k & 1;
      const int m0 = (int)(u % tiles) * 128, split = (int)(u / tiles);
      const int m = m0 + r;
      const bool valid = m < p.M;
      if (ok) ok = gwait(ptx::smem_u32(&accf[b]), (uint32_t)(k >> 1) & 1u, abort_flag, p.hdr, 72);
      ptx::tc_fence_after();
      const uint32_t tq = tmem + (uint32_t)(b * 256) + ((uint32_t)(32 * q) << 16);
      bool released = false;  // this warp has arrived on acce[b] for this unit
      if (ok) {
        for (int cb = c_lo; cb < c_hi; cb += 16) {
          float v[16];
          ptx::tmem_ld16(tq + cb, v);
          ptx::tmem_wait_ld();
          if (cb + 16 >= c_hi) {  // this warp's last read of the accumulator
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&acce[b]));
            released = true;
          }
          if (transpose) {
            float h[16], d[16];
            if (p.mode == kGemmFwdHidden) {
#pragma unroll
              for (int j = 0; j < 16; ++j) act_and_grad(v[j] + bias_s[cb + j], p.act, h[j], d[j]);
            } else {
              float a[16];
              if (valid) {
                const uint4* src = reinterpret_cast<const uint4*>(p.AD_in + (size_t)m * p.N + cb);
                const uint4 w0 = src[0], w1 = src[1];
                const uint32_t ws[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  a[2 * j] = __uint_as_float(ws[j] << 16);
                  a[2 * j + 1] = __uint_as_float(ws[j] & 0xffff0000u);
                }
              } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) a[j] = 0.0f;
              }
#pragma unroll
              for (int j = 0; j < 16; ++j) h[j] = v[j] * a[j];
            }
            if (valid) {
              uint4* dst = reinterpret_cast<uint4*>(p.H + (size_t)m * p.N + cb);
              dst[0] = make_uint4(bf2(h[0], h[1]), bf2(h[2], h[3]), bf2(h[4], h[5]), bf2(h[6], h[7]));
              dst[1] = make_uint4(bf2(h[8], h[9]), bf2(h[10], h[11]), bf2(h[12], h[13]), bf2(h[14], h[15]));
              if (p.mode == kGemmFwdHidden) {
                uint4* dd = reinterpret_cast<uint4*>(p.AD + (size_t)m * p.N + cb);
                dd[0] = make_uint4(bf2(d[0], d[1]), bf2(d[2], d[3]), bf2(d[4], d[5]), bf2(d[6], d[7]));
                dd[1] = make_uint4(bf2(d[8], d[9]), bf2(d[10], d[11]), bf2(d[12], d[13]), bf2(d[14], d[15]));
              }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) stage[(cb + j) * 128 + r] = __float2bfloat16_rn(valid ? h[j] : 0.0f);
          } else if (p.mode == kGemmFwdOut) {
            if (valid)
              for (int j = 0; j < 16; ++j)
                if (cb + j < p.n_real) p.Y[(size_t)m * p.ldY + cb + j] = v[j] + bias_s[cb + j];
          } else {  // kGemmPartial
            if (valid) {
              float4* dst = reinterpret_cast<float4*>(p.P + ((size_t)split * p.M + m) * p.N + cb);
#pragma unroll
              for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
          }
        }
      }
      if (!released) {  // no columns for this warp, or aborted: release all the same
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&acce[b]));
      }
      if (transpose) {
        // transposed copy: stage [N][128] -> HT[n][m0 .. m0 + 127], 16 bytes per store
        asm volatile("bar.sync 1, 512;" ::: "memory");
        if (ok) {
          const int per_row = 16;  // 128 BF16 = 16 x 16 bytes
          for (int e = threadIdx.x - 64; e < p.N * per_row; e += kGEpiThreads) {
            const int n = e / per_row, j = e % per_row;
            const int mm = m0 + 8 * j;
            if (mm + 8 <= p.ldT)
              *reinterpret_cast<uint4*>(p.HT + (size_t)n * p.ldT + mm) =
                  *reinterpret_cast<const uint4*>(stage + n * 128 + 8 * j);
          }
        }
        asm volatile("bar.sync 1, 512;" ::: "memory");  // the stage is free for the next unit
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem, 512);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// [rows][K] BF16 with row stride ld elements; box = 64 K x box_rows rows, 128B swizzle, zero fill.
bool make_map(CUtensorMap* map, const __nv_bfloat16* base, long long K, long long rows, long long ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc || ((uintptr_t)base & 15) || (ld * 2) % 16 || K < 1 || rows < 1) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gemm_smem_bytes() {
  return 1024 + kGStages * (kGABytes + kGBBytes) + kGStageBytes + (2 * kGStages + 6) * 8 + 256 * 4;
}

cudaError_t tc_gemm(const TcGemm& g, cudaStream_t s) {
  if (g.N < 16 || g.N > 256 || g.N % 16 || g.M < 1 || g.K < 1 || g.splits < 1) return cudaErrorInvalidValue;
  GemmParams p;
  memset(&p, 0, sizeof(p));
  if (!make_map(&p.ta, g.A, g.K, g.M, g.lda, 128)) return cudaErrorInvalidValue;
  if (!make_map(&p.tb, g.B, g.K, g.N, g.ldb, g.N)) return cudaErrorInvalidValue;
  const int kchunks_total = (int)((g.K + 63) / 64);
  p.M = g.M;
  p.N = g.N;
  p.n_real = g.n_real;
  p.kchunks = (kchunks_total + g.splits - 1) / g.splits;
  p.mode = g.mode;
  p.act = g.act;
  p.bbytes = (uint32_t)g.N * 128u;
  p.bias = g.bias;
  p.H = g.H;
  p.AD = g.AD;
  p.HT = g.HT;
  p.AD_in = g.AD_in;
  p.Y = g.Y;
  p.ldY = g.ldY;
  p.P = g.P;
  p.ldT = g.ldT;
  p.hdr = g.hdr;
  const size_t smem = tc_gemm_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int splits = (kchunks_total + p.kchunks - 1) / p.kchunks;
  p.splits = splits;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long units = (long long)((g.M + 127) / 128) * splits;
  const int grid = (int)(units < nsm ? units : nsm);  // persistent: one CTA per SM
  gemm_tc_kernel<<<grid, kGThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace voila

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
//   kFwdHidden  z = acc + b;  H = act(z), AD = act'(z) row-major and H^T (BF16);
//   kFwdOut     Y = acc + b (FP32, the first n_real columns);
//   kBwd        delta = acc * AD_in;  D row-major and D^T (BF16);
//   kPartial    P[split][m][n] = acc (FP32), summed later in split order.
// The BF16 outputs leave by TMA: each warp stages its 32 rows x 16 columns
// (row-major, and transposed) in its own shared-memory slots and one lane
// stores them as tensor tiles, so no store instruction scatters over 32
// rows and no warp waits for another.
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
constexpr int kGWarpStage = 3 * 32 * 16;   // BF16 per epilogue warp: [32][16] row-major x2, [16][32] transposed
constexpr long long kGSpin = 4000000000LL;

struct GemmParams {
  CUtensorMap ta, tb;
  CUtensorMap tH, tAD, tHT;  // store maps: H / AD [M][N] (box 16 x 32), HT [N][M] (box 32 x 16)
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

__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// act(z) and act'(z) of a pair z = (z0, z1) in packed FP32x2 arithmetic, one
// MUFU op per value. SiLU: s = sigmoid(z) = (1 + tanh(z/2)) / 2, act = z s,
// act' = s (1 + z (1 - s)) = s + act (1 - s); tanh: t = tanh z, act' = 1 - t^2.
// (tanh.approx.f32: relative error about 2^-11, below the BF16 rounding of
// the stored values.)
__device__ __forceinline__ void act_and_grad2(uint64_t z, int act, uint32_t& hp, uint32_t& dp) {
  using ptx::f2_fma;
  using ptx::f2_pack;
  using ptx::f2_unpack;
  using ptx::tanh_approx;
  float h0, h1, d0, d1;
  if (act == VOILA_ACT_SILU) {
    const uint64_t half = f2_pack(0.5f, 0.5f), nhalf = f2_pack(-0.5f, -0.5f);
    float a0, a1;
    f2_unpack(f2_mul(z, half), a0, a1);
    const uint64_t t = f2_pack(tanh_approx(a0), tanh_approx(a1));
    const uint64_t s = f2_fma(t, half, half), om = f2_fma(t, nhalf, half);
    const uint64_t h = f2_mul(z, s);
    f2_unpack(h, h0, h1);
    f2_unpack(f2_fma(h, om, s), d0, d1);
  } else if (act == VOILA_ACT_TANH) {
    float z0, z1;
    f2_unpack(z, z0, z1);
    const uint64_t t = f2_pack(tanh_approx(z0), tanh_approx(z1));
    f2_unpack(t, h0, h1);
    f2_unpack(f2_fma(t, f2_pack(-h0, -h1), f2_pack(1.0f, 1.0f)), d0, d1);
  } else {
    f2_unpack(z, h0, h1);
    d0 = d1 = 1.0f;
  }
  hp = ptx::pack_bf16x2(h0, h1);
  dp = ptx::pack_bf16x2(d0, d1);
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi) { return ptx::pack_bf16x2(lo, hi); }

// Persistent: each CTA takes work units u = blockIdx.x, + gridDim.x, ... (unit =
// 128-row tile x K split). Two FP32 accumulators in TMEM (columns [0, 256) and
// [256, 512)) let the MMAs of a CTA's next unit run while the epilogue warps
// drain the previous one; the producer streams the next unit's chunks into the
// ring meanwhile.
__global__ void __launch_bounds__(kGThreads, 1) gemm_tc_kernel(const __grid_constant__ GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* ringA = smem;
  uint8_t* ringB = smem + kGStages * kGABytes;
  __nv_bfloat16* stage = reinterpret_cast<__nv_bfloat16*>(ringB + kGStages * kGBBytes);  // per epilogue warp
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + 16 * kGWarpStage);
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
    const bool tstore = p.mode == kGemmFwdHidden || p.mode == kGemmBwd;
    __nv_bfloat16* stH = stage + (warp - 2) * kGWarpStage;  // [32 rows][16] : H (or D)
    __nv_bfloat16* stA = stH + 512;                          // [32 rows][16] : AD
    __nv_bfloat16* stT = stH + 1024;                         // [16][32 rows] : H^T (or D^T)
    bool pending = false;  // lane 0: bulk stores of this warp whose reads may be in flight
    bool ok = true;
    int k = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++k) {
      const int b = k & 1;
      const int m0 = (int)(u % tiles) * 128, split = (int)(u / tiles);
      const int m = m0 + r;
      const bool valid = m < p.M;
      const int mq = m0 + 32 * q;  // first row of this warp's lane quadrant
      if (ok) ok = gwait(ptx::smem_u32(&accf[b]), (uint32_t)(k >> 1) & 1u, abort_flag, p.hdr, 72);
      ptx::tc_fence_after();
      const uint32_t tq = tmem + (uint32_t)(b * 256) + ((uint32_t)(32 * q) << 16);
      bool released = false;  // this warp has arrived on acce[b] for this unit
      if (ok) {
        // backward: the activation derivatives of the next 16 columns are
        // loaded one batch ahead of their use
        uint4 an0 = make_uint4(0u, 0u, 0u, 0u), an1 = an0;
        if (p.mode == kGemmBwd && valid && c_lo < c_hi) {
          const uint4* src = reinterpret_cast<const uint4*>(p.AD_in + (size_t)m * p.N + c_lo);
          an0 = __ldg(src);
          an1 = __ldg(src + 1);
        }
        for (int cb = c_lo; cb < c_hi; cb += 16) {
          float v[16];
          ptx::tmem_ld16(tq + cb, v);
          const uint4 a0 = an0, a1 = an1;
          if (p.mode == kGemmBwd && valid && cb + 16 < c_hi) {
            const uint4* src = reinterpret_cast<const uint4*>(p.AD_in + (size_t)m * p.N + cb + 16);
            an0 = __ldg(src);
            an1 = __ldg(src + 1);
          }
          ptx::tmem_wait_ld();
          ptx::tie8(v);  // no use of v is scheduled before the wait
          ptx::tie8(v + 8);
          if (cb + 16 >= c_hi) {  // this warp's last read of the accumulator
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ptx::smem_u32(&acce[b]));
            released = true;
          }
          if (tstore) {
            uint32_t hp[8], dp[8];
            if (p.mode == kGemmFwdHidden) {
              const float4* b4 = reinterpret_cast<const float4*>(bias_s + cb);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float4 bb = b4[j];
                act_and_grad2(ptx::f2_add(ptx::f2_pack(v[4 * j], v[4 * j + 1]), ptx::f2_pack(bb.x, bb.y)), p.act,
                              hp[2 * j], dp[2 * j]);
                act_and_grad2(ptx::f2_add(ptx::f2_pack(v[4 * j + 2], v[4 * j + 3]), ptx::f2_pack(bb.z, bb.w)), p.act,
                              hp[2 * j + 1], dp[2 * j + 1]);
              }
            } else {
              const uint32_t ws[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float d0, d1;
                ptx::f2_unpack(f2_mul(ptx::f2_pack(v[2 * j], v[2 * j + 1]),
                                      ptx::f2_pack(__uint_as_float(ws[j] << 16), __uint_as_float(ws[j] & 0xffff0000u))),
                               d0, d1);
                hp[j] = bf2(d0, d1);
              }
            }
            // the slots are free once the previous batch's stores have read them
            if (lane == 0 && pending) ptx::bulk_wait_read_all();
            __syncwarp();
            uint4* rowH = reinterpret_cast<uint4*>(stH + lane * 16);
            rowH[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
            rowH[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
            if (p.mode == kGemmFwdHidden) {
              uint4* rowA = reinterpret_cast<uint4*>(stA + lane * 16);
              rowA[0] = make_uint4(dp[0], dp[1], dp[2], dp[3]);
              rowA[1] = make_uint4(dp[4], dp[5], dp[6], dp[7]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              stT[(2 * j) * 32 + lane] = __ushort_as_bfloat16((unsigned short)(hp[j] & 0xffffu));
              stT[(2 * j + 1) * 32 + lane] = __ushort_as_bfloat16((unsigned short)(hp[j] >> 16));
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            // rows from M on (a ragged last tile) fall outside the tensors and are not written
            if (lane == 0 && mq < p.M) {
              ptx::tma_store_2d(&p.tH, cb, mq, ptx::smem_u32(stH));
              if (p.mode == kGemmFwdHidden) ptx::tma_store_2d(&p.tAD, cb, mq, ptx::smem_u32(stA));
              ptx::tma_store_2d(&p.tHT, mq, cb, ptx::smem_u32(stT));
              ptx::bulk_commit();
              pending = true;
            }
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
    }
    // the bulk stores complete (their shared-memory reads and global writes)
    // before the kernel ends
    if (lane == 0 && pending) ptx::bulk_wait_all();
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

// Store map of a row-major [rows][cols] BF16 tensor (row stride ld elements), box
// box_c columns x box_r rows, no swizzle: the shared-memory tile is dense row-major.
bool make_store_map(CUtensorMap* map, const __nv_bfloat16* base, long long cols, long long rows, long long ld,
                    int box_c, int box_r) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc || ((uintptr_t)base & 15) || (ld * 2) % 16 || cols < 1 || rows < 1) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)box_c, (cuuint32_t)box_r};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t tc_gemm_smem_bytes() {
  return 1024 + kGStages * (kGABytes + kGBBytes) + 16 * kGWarpStage * 2 + (2 * kGStages + 6) * 8 + 256 * 4;
}

cudaError_t tc_gemm(const TcGemm& g, cudaStream_t s) {
  if (g.N < 16 || g.N > 256 || g.N % 16 || g.M < 1 || g.K < 1 || g.splits < 1) return cudaErrorInvalidValue;
  GemmParams p;
  memset(&p, 0, sizeof(p));
  if (!make_map(&p.ta, g.A, g.K, g.M, g.lda, 128)) return cudaErrorInvalidValue;
  if (!make_map(&p.tb, g.B, g.K, g.N, g.ldb, g.N)) return cudaErrorInvalidValue;
  if (g.mode == kGemmFwdHidden || g.mode == kGemmBwd) {
    if (!g.H || !g.HT || (g.mode == kGemmFwdHidden && !g.AD) || (g.mode == kGemmBwd && !g.AD_in) || g.ldT < g.M)
      return cudaErrorInvalidValue;
    if (!make_store_map(&p.tH, g.H, g.N, g.M, g.N, 16, 32)) return cudaErrorInvalidValue;
    if (g.mode == kGemmFwdHidden && !make_store_map(&p.tAD, g.AD, g.N, g.M, g.N, 16, 32)) return cudaErrorInvalidValue;
    if (!make_store_map(&p.tHT, g.HT, g.M, g.N, g.ldT, 32, 16)) return cudaErrorInvalidValue;
  }
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
  // persistent: one CTA per SM; spread: one CTA per unit
  const int grid = (int)(g.spread || units < nsm ? units : nsm);
  gemm_tc_kernel<<<grid, kGThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace voila

// BF16 tensor-core rollout on sm_103a (tcgen05 + TMEM).
//
// One persistent CTA per SM runs pairs of 128-row tiles (row = k * N + n, one
// (particle, action-sequence) pair per row) through all H steps of the
// generator s' = g_T([s; a; omega]) (Eq. 2) and the reward head, and
// accumulates G = sum_t gamma^t r_t in FP64 (value definition, Sec. 2.1).
//
// Warp roles (576 threads):
//   warp 0      producer: streams the packed, pre-swizzled BF16 weight chunks
//               of every layer through a ring of shared-memory slots with
//               cp.async.bulk (the whole weight set, 560 KB for the 3x256
//               generator + reward, does not fit in 227 KB of shared memory);
//   warp 1      MMA issuer: allocates the 512 TMEM columns and issues the
//               tcgen05.mma of the two tiles alternately, one layer at a time,
//               so one tile's MMAs run while the other tile's epilogue runs
//               (each tile streams its own pass over the weights; L2 has the
//               bandwidth for it);
//   warps 2-17  epilogue, eight warps per tile (two per TMEM lane quadrant,
//               splitting the columns), one thread per row: TMEM ->
//               registers, bias + SiLU (1/2 folded into W, b; one tanh.approx per value), BF16 into the next
//               layer's A operand (128B-swizzled K-major), plus the row's
//               state s_t, Philox noise, reward and FP64 return.
// Accumulators: tile 0 in TMEM columns [0, 256), tile 1 in [256, 512).
// Every wait on an mbarrier is bounded; on expiry the kernel records
// VOILA_ERR_TIMEOUT in the workspace status word, drains its own copies and
// MMAs, frees TMEM and returns.
#include <string.h>

#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"

namespace voila {

namespace {

constexpr int kTcThreads = 576;   // producer warp, MMA warp, 16 epilogue warps
constexpr int kEpiWarpsPerTile = 8;
constexpr int kTileRows = 128;
constexpr int kStages = 5;
constexpr int kSlotBytes = 256 * 64;      // N <= 256 rows x 32 BF16 of K
constexpr int kABytes = 4 * 128 * 128;    // 128 rows x 256 BF16, four 64-wide K slabs
constexpr int kMaxTcLayers = 16;
constexpr long long kSpinLimit = 4000000000LL;  // ~2 s of SM clock per wait

struct TcLayer {
  int Kp;           // input width rounded up to 16 (MMA K steps of 16)
  int Npad;         // output width (hidden: multiple of 64; output layer: rounded up to 16)
  int nchunks;      // ceil(Kp / 32) weight chunks of [Npad][32]
  int chunk_bytes;  // Npad * 64
  int bias_off;     // offset into the concatenated bias vector
  int act;          // activation after this layer (-1: linear output layer)
  uint32_t idesc;
  long long wofs;   // byte offset of chunk 0 in the packed weight stream
};

struct TcParams {
  TcLayer layers[kMaxTcLayers];
  int n_gen, n_total;
  const uint8_t* wstream;
  const float* bias_all;
  int bias_total;  // floats, multiple of 4
  const float* particles;
  const float* actions;
  int N, K, H;
  long long rows, pairs;
  double gamma;
  uint32_t key0, key1, planner;
  int reward_kind, goal_dims;
  float goal[VOILA_MAX_GOAL];
  double* G;
  WsHeader* hdr;
};

__device__ __forceinline__ bool bounded_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                             WsHeader* hdr, int where) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kSpinLimit) {
      *abort_flag = 1;
      set_status(hdr, VOILA_ERR_TIMEOUT, where);
      return false;
    }
  }
}

// Activation of two accumulator values, packed to BF16x2 for the next layer.
// SiLU: the weights and bias of a SiLU layer are packed pre-scaled by 1/2
// (exact in BF16/FP32), so the accumulator holds u = x/2 and
// silu(x) = x sigmoid(x) = u (1 + tanh u) = fma(u, tanh u, u): one MUFU op
// (tanh.approx.f32; the packed BF16x2/FP16x2 forms measured slower on this
// part) and one FMA per value.
__device__ __forceinline__ uint32_t act_pair(float u0, float u1, int act) {
  if (act == VOILA_ACT_SILU)
    return ptx::pack_bf16x2(fmaf(u0, ptx::tanh_approx(u0), u0), fmaf(u1, ptx::tanh_approx(u1), u1));
  if (act == VOILA_ACT_TANH) return ptx::pack_bf16x2(ptx::tanh_approx(u0), ptx::tanh_approx(u1));
  return ptx::pack_bf16x2(u0, u1);
}

// 32 accumulator columns [32c, 32c + 32) of row r -> bias + activation ->
// four 16-byte chunks of the next layer's A operand.
__device__ __forceinline__ void epi_cols32(const float* v, const float* bl, int c, int act, uint8_t* A,
                                           int r) {
  uint8_t* slab = A + (c >> 1) * (128 * 128);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 b0 = *reinterpret_cast<const float4*>(bl + 32 * c + 8 * j);
    const float4 b1 = *reinterpret_cast<const float4*>(bl + 32 * c + 8 * j + 4);
    uint4 o;
    o.x = act_pair(v[8 * j + 0] + b0.x, v[8 * j + 1] + b0.y, act);
    o.y = act_pair(v[8 * j + 2] + b0.z, v[8 * j + 3] + b0.w, act);
    o.z = act_pair(v[8 * j + 4] + b1.x, v[8 * j + 5] + b1.y, act);
    o.w = act_pair(v[8 * j + 6] + b1.z, v[8 * j + 7] + b1.w, act);
    *reinterpret_cast<uint4*>(slab + r * 128 + ((((c & 1) * 4 + j) ^ (r & 7)) << 4)) = o;
  }
}

// Byte address of 16-byte chunk j (8 BF16 columns) of row r in a 128B-swizzled
// K-major slab: the chunk index is XORed with r mod 8.
__device__ __forceinline__ uint8_t* a_chunk(uint8_t* slab, int r, int j) {
  return slab + r * 128 + ((j ^ (r & 7)) << 4);
}

template <int KP>
__device__ __forceinline__ void store_row(uint8_t* A, int r, const float* x) {
#pragma unroll
  for (int j = 0; j < KP / 8; ++j) {
    uint4 v;
    v.x = ptx::pack_bf16x2(x[8 * j + 0], x[8 * j + 1]);
    v.y = ptx::pack_bf16x2(x[8 * j + 2], x[8 * j + 3]);
    v.z = ptx::pack_bf16x2(x[8 * j + 4], x[8 * j + 5]);
    v.w = ptx::pack_bf16x2(x[8 * j + 6], x[8 * j + 7]);
    *reinterpret_cast<uint4*>(a_chunk(A, r, j)) = v;
  }
}

// x = [s; a; omega_T(n, k, t)] zero-padded to a multiple of 16, as BF16.
template <int DS, int DA, int DW>
__device__ __forceinline__ void write_gen_input(uint8_t* A, int r, const float* s, const float* a,
                                                uint32_t k0, uint32_t k1, uint32_t n, uint32_t k,
                                                uint32_t t, uint32_t planner) {
  constexpr int KP = (DS + DA + DW + 15) / 16 * 16;
  float x[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) x[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < DS; ++i) x[i] = s[i];
#pragma unroll
  for (int i = 0; i < DA; ++i) x[DS + i] = a[i];
#pragma unroll
  for (int b = 0; b < (DW + 3) / 4; ++b) {
    const float4 z = normal4(k0, k1, n, k, t, VOILA_STREAM_ROLLOUT_OMEGA, planner, (uint32_t)b);
    if (4 * b + 0 < DW) x[DS + DA + 4 * b + 0] = z.x;
    if (4 * b + 1 < DW) x[DS + DA + 4 * b + 1] = z.y;
    if (4 * b + 2 < DW) x[DS + DA + 4 * b + 2] = z.z;
    if (4 * b + 3 < DW) x[DS + DA + 4 * b + 3] = z.w;
  }
  store_row<KP>(A, r, x);
}

// x = [s_{t+1}; a_t] zero-padded, as BF16 (reward-head input).
template <int DS, int DA>
__device__ __forceinline__ void write_rew_input(uint8_t* A, int r, const float* s, const float* a) {
  constexpr int KP = (DS + DA + 15) / 16 * 16;
  float x[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) x[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < DS; ++i) x[i] = s[i];
#pragma unroll
  for (int i = 0; i < DA; ++i) x[DS + i] = a[i];
  store_row<KP>(A, r, x);
}

template <int DS, int DA, int DW>
__global__ void __launch_bounds__(kTcThreads, 1) rollout_tc_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* Abuf[2] = {smem, smem + kABytes};
  uint8_t* ring = smem + 2 * kABytes;
  float* bias_s = reinterpret_cast<float*>(ring + kStages * kSlotBytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(bias_s + p.bias_total);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* accf = bars + 2 * kStages;      // [2]
  uint64_t* ready = bars + 2 * kStages + 2;  // [2]
  uint64_t* drain = bars + 2 * kStages + 4;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
    }
    for (int g = 0; g < 2; ++g) {
      ptx::mbar_init(ptx::smem_u32(&accf[g]), 1);
      ptx::mbar_init(ptx::smem_u32(&ready[g]), kEpiWarpsPerTile);  // one arrival per epilogue warp
    }
    ptx::mbar_init(ptx::smem_u32(drain), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  for (int i = threadIdx.x; i < p.bias_total; i += blockDim.x) bias_s[i] = p.bias_all[i];
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_u32(tmem_holder), 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const uint32_t ring_addr = ptx::smem_u32(ring);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      int last_round[kStages];
      for (int s = 0; s < kStages; ++s) last_round[s] = -1;
      for (long long pr = blockIdx.x; pr < p.pairs && ok; pr += gridDim.x)
        for (int t = 0; t < p.H && ok; ++t)
          for (int l = 0; l < p.n_total && ok; ++l)
            for (int g = 0; g < 2 && ok; ++g) {
              const TcLayer& L = p.layers[l];
              for (int c = 0; c < L.nchunks; ++c, ++it) {
                const int slot = (int)(it % kStages);
                const uint32_t round = (uint32_t)(it / kStages);
                if (!bounded_wait(ptx::smem_u32(&empty[slot]), (round & 1) ^ 1, abort_flag, p.hdr, 10)) {
                  ok = false;
                  break;
                }
                ptx::mbar_arrive_expect_tx(ptx::smem_u32(&full[slot]), (uint32_t)L.chunk_bytes);
                ptx::bulk_g2s(ring_addr + slot * kSlotBytes, p.wstream + L.wofs + (long long)c * L.chunk_bytes,
                              (uint32_t)L.chunk_bytes, ptx::smem_u32(&full[slot]));
                last_round[slot] = (int)round;
              }
            }
      if (!ok) {  // drain copies still in flight before the CTA's shared memory goes away
        for (int s = 0; s < kStages; ++s)
          if (last_round[s] >= 0) {
            const long long t0 = clock64();
            while (!ptx::mbar_try_wait(ptx::smem_u32(&full[s]), (uint32_t)last_round[s] & 1) &&
                   clock64() - t0 < kSpinLimit) {
            }
          }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      long long it = 0;
      uint32_t nready0 = 0, nready1 = 0;
      bool ok = true;
      const uint32_t a_addr0 = ptx::smem_u32(Abuf[0]), a_addr1 = ptx::smem_u32(Abuf[1]);
      for (long long pr = blockIdx.x; pr < p.pairs && ok; pr += gridDim.x)
        for (int t = 0; t < p.H && ok; ++t)
          for (int l = 0; l < p.n_total && ok; ++l)
            for (int g = 0; g < 2 && ok; ++g) {
              // tile g's A operand for layer l is ready and its accumulator is free
              const uint32_t nr = g ? nready1 : nready0;
              if (!bounded_wait(ptx::smem_u32(&ready[g]), nr & 1, abort_flag, p.hdr, 21 + g)) {
                ok = false;
                break;
              }
              if (g) ++nready1;
              else ++nready0;
              ptx::tc_fence_after();
              const TcLayer& L = p.layers[l];
              const uint32_t a_addr = g ? a_addr1 : a_addr0;
              for (int c = 0; c < L.nchunks; ++c, ++it) {
                const int slot = (int)(it % kStages);
                const uint32_t round = (uint32_t)(it / kStages);
                if (!bounded_wait(ptx::smem_u32(&full[slot]), round & 1, abort_flag, p.hdr, 20)) {
                  ok = false;
                  break;
                }
                ptx::tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                  const int kidx = 32 * c + 16 * kk;
                  if (kidx < L.Kp) {
                    const uint64_t ad = ptx::smem_desc(a_addr + (kidx >> 6) * (128 * 128) + (kidx & 63) * 2,
                                                       1024, ptx::kSwizzle128B);
                    const uint64_t bd = ptx::smem_desc(ring_addr + slot * kSlotBytes + kk * 32, 512,
                                                       ptx::kSwizzle64B);
                    ptx::mma_bf16(tmem_base + g * 256, ad, bd, L.idesc, (c > 0 || kk > 0) ? 1u : 0u);
                  }
                }
                ptx::mma_commit(ptx::smem_u32(&empty[slot]));
                if (c == L.nchunks - 1) ptx::mma_commit(ptx::smem_u32(&accf[g]));
              }
            }
      // wait for every MMA this thread issued (normal exit and abort alike)
      ptx::mma_commit(ptx::smem_u32(drain));
      const long long t0 = clock64();
      while (!ptx::mbar_try_wait(ptx::smem_u32(drain), 0) && clock64() - t0 < kSpinLimit) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // Eight warps per tile: warp w may read TMEM lanes 32*(w % 4) .. +31 (its
    // rows); the two warps of a lane quadrant split the hidden columns. The
    // "sub 0" warps also own the row state (s_t, omega, reward, G).
    const int e = warp - 2;
    const int g = e >> 3;                   // tile of this warp
    const int sub = (e >> 2) & 1;           // column half of the hidden layers
    const int q = warp & 3;                 // TMEM lane quadrant this warp may access
    const int r = 32 * q + lane;            // row within the tile
    uint8_t* A = Abuf[g];
    const uint32_t tm = tmem_base + (uint32_t)(g * 256) + ((uint32_t)(32 * q) << 16);
    const uint32_t ready_bar = ptx::smem_u32(&ready[g]);
    const uint32_t acc_bar = ptx::smem_u32(&accf[g]);
    uint32_t nacc = 0;
    bool ok = true;
    for (long long pr = blockIdx.x; pr < p.pairs && ok; pr += gridDim.x) {
      const long long row = pr * (2 * kTileRows) + g * kTileRows + r;
      const bool valid = row < p.rows;
      const uint32_t n = valid ? (uint32_t)(row % p.N) : 0u;
      const uint32_t k = valid ? (uint32_t)(row / p.N) : 0u;
      const float* act_row = p.actions + (size_t)k * p.H * DA;
      float s[DS], a[DA];
      if (sub == 0) {
#pragma unroll
        for (int i = 0; i < DS; ++i) s[i] = valid ? __ldg(p.particles + (size_t)n * DS + i) : 0.0f;
#pragma unroll
        for (int i = 0; i < DA; ++i) a[i] = __ldg(act_row + i);
        write_gen_input<DS, DA, DW>(A, r, s, a, p.key0, p.key1, n, k, 0, p.planner);
      }
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ready_bar);
      double Gacc = 0.0, disc = 1.0;
      for (int t = 0; t < p.H && ok; ++t) {
        for (int l = 0; l < p.n_total; ++l) {
          const TcLayer& L = p.layers[l];
          if (!bounded_wait(acc_bar, nacc & 1, abort_flag, p.hdr, 30 + g)) {
            ok = false;
            break;
          }
          ++nacc;
          ptx::tc_fence_after();
          const float* bl = bias_s + L.bias_off;
          // no A operand follows the final layer of the final step
          const bool arrive = !(t == p.H - 1 && l == p.n_total - 1);
          if (L.act >= 0) {
            // hidden layer: bias + activation -> BF16 A operand of the next layer,
            // 32 columns per TMEM load (measured faster than larger batches)
            const int nc = L.Npad >> 6;  // 32-column batches per warp (half the columns)
            for (int c = sub * nc; c < (sub + 1) * nc; ++c) {
              float v[32];
              ptx::tmem_ld32(tm + 32 * c, v);
              ptx::tmem_wait_ld32(v);
              epi_cols32(v, bl, c, L.act, A, r);
            }
          } else if (sub == 0 && l == p.n_gen - 1) {
            // generator output: s_{t+1} (FP32, kept in registers)
            float v[32];
            ptx::tmem_ld16(tm, v);
            if (DS > 16) ptx::tmem_ld16(tm + 16, v + 16);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < DS; ++i) s[i] = v[i] + bl[i];
            if (p.reward_kind == VOILA_REWARD_GOAL) {
              float acc = 0.0f;
#pragma unroll
              for (int i = 0; i < VOILA_MAX_GOAL; ++i)
                if (i < p.goal_dims && i < DS) {
                  const float d = s[i] - p.goal[i];
                  acc = fmaf(d, d, acc);
                }
              Gacc += disc * (double)(-acc);
              disc *= p.gamma;
              if (t + 1 < p.H) {
#pragma unroll
                for (int i = 0; i < DA; ++i) a[i] = __ldg(act_row + (t + 1) * DA + i);
                write_gen_input<DS, DA, DW>(A, r, s, a, p.key0, p.key1, n, k, (uint32_t)(t + 1), p.planner);
              }
            } else {
              write_rew_input<DS, DA>(A, r, s, a);
            }
          } else if (sub == 0) {
            // reward output r_t: G += gamma^t r_t in FP64
            float v[16];
            ptx::tmem_ld16(tm, v);
            ptx::tmem_wait_ld();
            Gacc += disc * (double)(v[0] + bl[0]);
            disc *= p.gamma;
            if (t + 1 < p.H) {
#pragma unroll
              for (int i = 0; i < DA; ++i) a[i] = __ldg(act_row + (t + 1) * DA + i);
              write_gen_input<DS, DA, DW>(A, r, s, a, p.key0, p.key1, n, k, (uint32_t)(t + 1), p.planner);
            }
          }
          ptx::tc_fence_before();
          if (arrive) {
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(ready_bar);
          }
        }
      }
      if (sub == 0 && valid && ok) p.G[row] = Gacc;
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, 512);
}

// One launch packs every layer: W[l] ([N][K] BF16 row-major) becomes chunks
// of [Npad][32] with the 64B swizzle (16-byte chunk j of row n lands at
// j ^ ((n >> 1) & 3)), zero padded; biases are copied zero padded.
struct PackTable {
  const __nv_bfloat16* W[kMaxTcLayers];
  const float* b[kMaxTcLayers];
  int N[kMaxTcLayers], K[kMaxTcLayers], Npad[kMaxTcLayers], nchunks[kMaxTcLayers];
  long long wofs[kMaxTcLayers], welems_end[kMaxTcLayers];
  int bias_off[kMaxTcLayers];
  int half[kMaxTcLayers];  // 1: SiLU layer, pack W and b scaled by 1/2
  int n;
  uint8_t* wout;
  float* bout;
};

__global__ void pack_kernel(const __grid_constant__ PackTable t) {
  const long long total = t.welems_end[t.n - 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (e >= t.welems_end[l]) ++l;
    const long long e0 = e - (l ? t.welems_end[l - 1] : 0);
    const int Npad = t.Npad[l];
    const int c = (int)(e0 / (Npad * 32));
    const int rem = (int)(e0 % (Npad * 32));
    const int nrow = rem / 32, kk = rem % 32;
    const int kg = 32 * c + kk;
    __nv_bfloat16 v =
        (nrow < t.N[l] && kg < t.K[l]) ? t.W[l][(size_t)nrow * t.K[l] + kg] : __float2bfloat16(0.0f);
    if (t.half[l]) v = __hmul(v, __float2bfloat16(0.5f));  // exact: power-of-two scaling
    const int j = kk >> 3;
    const size_t byte =
        (size_t)t.wofs[l] + (size_t)c * Npad * 64 + (size_t)nrow * 64 + (((j ^ ((nrow >> 1) & 3)) << 4)) + (kk & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(t.wout + byte) = v;
    if (c == 0 && kk == 0) {
      const int np4 = (Npad + 3) / 4 * 4;
      if (nrow < np4)
        t.bout[t.bias_off[l] + nrow] = nrow < t.N[l] ? (t.half[l] ? 0.5f : 1.0f) * t.b[l][nrow] : 0.0f;
      if (nrow == Npad - 1)
        for (int i = Npad; i < np4; ++i) t.bout[t.bias_off[l] + i] = 0.0f;
    }
  }
}

struct Plan {
  TcParams p;
  PackTable pack;
  size_t wbytes, bias_bytes, total;
  bool ok;
};

int round_up(int v, int m) { return (v + m - 1) / m * m; }

Plan make_plan(const voila_mlp* g, const voila_reward* R) {
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  pl.ok = false;
  const voila_mlp* mlps[2] = {g, R && R->kind == VOILA_REWARD_MLP ? R->mlp : nullptr};
  int nl = 0, boff = 0;
  long long wofs = 0, welems = 0;
  for (int m = 0; m < 2; ++m) {
    const voila_mlp* M = mlps[m];
    if (!M) continue;
    if (M->prec != VOILA_BF16 || M->n_layers < 2) return pl;
    for (int l = 0; l < M->n_layers; ++l) {
      if (nl >= kMaxTcLayers) return pl;
      const int K = M->dims[l], N = M->dims[l + 1];
      const bool last = l == M->n_layers - 1;
      if (l == 0 && K > 64) return pl;
      if (l > 0 && (K % 64 != 0 || K > 256)) return pl;
      if (!last && (N % 64 != 0 || N > 256)) return pl;
      if (last && N > 32) return pl;
      TcLayer& L = pl.p.layers[nl];
      L.Kp = round_up(K, 16);
      L.Npad = last ? round_up(N, 16) : N;
      L.nchunks = (L.Kp + 31) / 32;
      L.chunk_bytes = L.Npad * 64;
      L.bias_off = boff;
      L.act = last ? -1 : M->act;
      L.idesc = ptx::idesc_bf16(128, L.Npad);
      L.wofs = wofs;
      PackTable& T = pl.pack;
      T.W[nl] = (const __nv_bfloat16*)M->W[l];
      T.b[nl] = M->b[l];
      T.N[nl] = N;
      T.K[nl] = K;
      T.Npad[nl] = L.Npad;
      T.nchunks[nl] = L.nchunks;
      T.wofs[nl] = wofs;
      T.bias_off[nl] = boff;
      T.half[nl] = (!last && M->act == VOILA_ACT_SILU) ? 1 : 0;
      welems += (long long)L.nchunks * L.Npad * 32;
      T.welems_end[nl] = welems;
      wofs += (long long)L.nchunks * L.chunk_bytes;
      boff += round_up(L.Npad, 4);
      ++nl;
    }
    if (m == 0) pl.p.n_gen = nl;
  }
  pl.p.n_total = nl;
  pl.pack.n = nl;
  pl.p.bias_total = boff;
  pl.wbytes = (size_t)wofs;
  pl.bias_bytes = (size_t)boff * sizeof(float);
  pl.total = (pl.wbytes + 255) / 256 * 256 + (pl.bias_bytes + 255) / 256 * 256;
  pl.ok = true;
  return pl;
}

size_t tc_smem_bytes(int bias_total) {
  return 1024 + 2 * kABytes + kStages * kSlotBytes + (size_t)bias_total * 4 + (2 * kStages + 5) * 8 + 16;
}

template <int DS, int DA, int DW>
cudaError_t launch_tc(const TcParams& p, size_t smem, int grid, cudaStream_t s) {
  auto k = rollout_tc_kernel<DS, DA, DW>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kTcThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t tc_rollout_scratch_bytes(const voila_mlp* g_T, const voila_reward* R) {
  Plan pl = make_plan(g_T, R);
  return pl.ok ? pl.total : 0;
}

voila_status tc_rollout(const voila_mlp* g_T, const voila_reward* R, const RolloutArgs& a,
                        WsHeader* hdr, void* scratch, cudaStream_t s) {
  Plan pl = make_plan(g_T, R);
  if (!pl.ok) return VOILA_ERR_UNSUPPORTED;
  const bool dims_a = a.d_s == 8 && a.d_a == 2 && a.d_omega == 8;
  const bool dims_b = a.d_s == 12 && a.d_a == 3 && a.d_omega == 16;
  if (!dims_a && !dims_b) return VOILA_ERR_UNSUPPORTED;
  if (a.H == 0) {
    return cudaMemsetAsync(a.G, 0, (size_t)a.N * a.K * sizeof(double), s) == cudaSuccess ? VOILA_OK
                                                                                       : VOILA_ERR_CUDA;
  }
  uint8_t* wst = (uint8_t*)scratch;
  float* bias_all = (float*)(wst + (pl.wbytes + 255) / 256 * 256);
  pl.pack.wout = wst;
  pl.pack.bout = bias_all;
  {
    const long long total = pl.pack.welems_end[pl.pack.n - 1];
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    pack_kernel<<<(int)blocks, 256, 0, s>>>(pl.pack);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  TcParams& p = pl.p;
  p.wstream = wst;
  p.bias_all = bias_all;
  p.particles = a.particles;
  p.actions = a.actions;
  p.N = a.N;
  p.K = a.K;
  p.H = a.H;
  p.rows = (long long)a.N * a.K;
  p.pairs = (p.rows + 2 * kTileRows - 1) / (2 * kTileRows);
  p.gamma = a.gamma;
  p.key0 = a.key0;
  p.key1 = a.key1;
  p.planner = a.planner;
  p.reward_kind = a.reward_kind;
  p.goal_dims = a.goal_dims;
  for (int i = 0; i < VOILA_MAX_GOAL; ++i) p.goal[i] = a.goal[i];
  p.G = a.G;
  p.hdr = hdr;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(p.pairs < nsm ? p.pairs : nsm);
  const size_t smem = tc_smem_bytes(p.bias_total);
  cudaError_t e = dims_a ? launch_tc<8, 2, 8>(p, smem, grid, s) : launch_tc<12, 3, 16>(p, smem, grid, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

}  // namespace voila

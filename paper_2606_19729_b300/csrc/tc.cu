// BF16 tensor-core rollout on sm_103a (tcgen05 + TMEM, CTA-pair MMA).
//
// Clusters of two CTAs on two SMs run "super-pairs" of 512 rows (row =
// k * N + n, one (particle, action-sequence) pair per row): each CTA owns two
// 128-row tiles, and the pair's matching tiles form one M = 256 tcgen05.mma
// (cta_group::2). Every row goes through all H steps of the generator
// s' = g_T([s; a; omega]) (Eq. 2) and the reward head, accumulating
// G = sum_t gamma^t r_t in FP64 (value definition, Sec. 2.1).
//
// The pair MMA is what makes the contraction fit this part: an M = 128 MMA
// reads A (4 KB) and B (8 KB) from one SM's shared memory per K = 16 step,
// and with the weight stream on top that exceeds the shared-memory bandwidth
// the tensor core gets; in the pair each SM reads its A and only half of B,
// and loads only half of every weight chunk.
//
// Warp roles (576 threads per CTA):
//   warp 0      producer: TMA-loads this CTA's half (N/2 rows) of every
//               [N][64] weight chunk into a ring of shared-memory slots; the
//               loads of both CTAs complete on the even CTA's barrier;
//   warp 1      allocates the 512 TMEM columns (both CTAs); in the even CTA
//               it issues the pair MMAs of the two tiles alternately, one
//               layer at a time, so one tile's MMAs run while the other
//               tile's epilogue runs, and commits to both CTAs' barriers;
//   warps 2-17  epilogue, eight warps per tile (two per TMEM lane quadrant,
//               splitting the columns), one thread per row: TMEM ->
//               registers, bias + SiLU (1/2 folded into W and b; one
//               tanh.approx per value), BF16 into the next layer's A operand
//               (128B-swizzled K-major), plus the row's state s_t, Philox
//               noise, reward and FP64 return.
// Accumulators: tile 0 in TMEM columns [0, 256), tile 1 in [256, 512).
// Every wait on an mbarrier is bounded; on expiry the kernel records
// VOILA_ERR_TIMEOUT in the workspace status word, drains its copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <cuda_fp8.h>

#include "common.cuh"
#include "tc.h"
#include "tc_ptx.cuh"

namespace voila {

namespace {

constexpr int kTcThreads = 576;   // producer warp, MMA warp, 16 epilogue warps
constexpr int kEpiWarpsPerTile = 8;
constexpr int kTileRows = 128;
constexpr int kStages = 5;
constexpr int kSlotBytes = 128 * 128;     // half of a [256][64] BF16 weight chunk
constexpr int kABytes = 4 * 128 * 128;    // 128 rows x 256 BF16, four 64-wide K slabs
constexpr int kMaxTcLayers = 16;
constexpr int kSuperRows = 4 * kTileRows;  // rows of one work item (two tiles on each CTA of the pair)
constexpr long long kSpinLimit = 4000000000LL;  // ~2 s of SM clock per wait
// What the rows of a launch are: rollout rows (n, k) over H planning steps;
// DDIM teacher samples over the sampler's steps; likelihood pairs (i, j) of
// the InfoNCE objective (one evaluation, H = 1).
// ... and the observation sampler of progressive widening (rows = the listed
// widened simulations, one evaluation of f_Z, outputs scattered to the tree).
// ... and the proposal of the belief update (rows = particles: one generator
// step, then the likelihood of the proposal, its scalar output fused).
constexpr int kModeRollout = 0, kModeDdim = 1, kModePairs = 2, kModeObserve = 3, kModePropose = 4;

struct TcLayer {
  int Kp;           // input width rounded up to 16 (MMA K steps of 16)
  int Npad;         // output width (hidden: multiple of 64; output layer: rounded up to 32)
  int nslabs;       // ceil(Kp / 64) K-slabs of [Npad][64]
  int slab_bytes;   // one CTA's half of a slab: Npad / 2 rows x 128 B
  int spc;          // slabs per ring chunk (several for narrow layers)
  int nchunks;      // ceil(nslabs / spc)
  int bias_off;     // offset into the concatenated bias vector
  int act;          // activation after this layer (-1: linear output layer)
  int fp8;          // 1: E4M3 operands (kind::f8f6f4, 128 K per slab), else BF16 (64 K per slab)
  int out_fp8;      // 1: this layer's epilogue writes the next layer's A operand as E4M3
  int ksteps;       // MMA K steps (32 K each for FP8, 16 for BF16)
  int scale_off;    // per-output-channel weight scales (FP8 layers), offset into the scale vector
  int ngroups;      // 256-column groups of the output (2 for a 512-wide layer in the wide kernel)
  int box_rows;     // rows of one CTA's TMA box: min(Npad, 256) / 2
  uint32_t idesc;
  int row0;         // first row of chunk 0 in the [rows][64] weight tensor
  int fuse_out;     // 1: a scalar output layer follows, computed in this layer's epilogue on CUDA cores
  int fuse_off;     // its weights (fuse_K floats) and bias in the fused-output vector
  int fuse_K;
  int rot;          // wide kernel: 1 when this layer's K < 256 sits in the upper A half (see make_plan)
};

// One independent planning problem of a (batched) launch.
struct TcPlanner {
  const float* particles;  // [N][d_s]
  const float* actions;    // [K][H][d_a]
  double* G;               // [K][N]
  long long rows;          // N * K
  int N, H;
  uint32_t planner;        // noise stream id
  uint32_t n_off, k_off;   // the rows' particle and sequence indices in the unsharded problem
                           // (noise counters (n + n_off, k + k_off, t))
};

struct TcParams {
  CUtensorMap tmap[kMaxTcLayers];  // per layer: box of [Npad / 2][64], 128B swizzle
  TcLayer layers[kMaxTcLayers];
  int n_gen, n_total;
  const float* bias_all;
  int bias_total;   // floats, multiple of 4
  int scale_total;  // floats after the biases in the same vector (FP8 channel scales)
  int fuse_total;   // floats after the scales: fused scalar-output weights and biases
  double gamma;
  uint32_t key0, key1;
  int reward_kind, goal_dims;
  float goal[VOILA_MAX_GOAL];
  WsHeader* hdr;
  // Work items are 512-row super-pairs, numbered planner by planner in table
  // order; cluster c takes items c, c + clusters, ... (with the table sorted
  // by descending horizon this approximates longest-processing-time first),
  // or, in the queue instantiation, whichever item is next on the global
  // counter `queue` (zeroed before the launch) when the cluster is ready.
  unsigned long long* queue;
  int P;
  long long total_items;
  long long item_end[kMaxPlanners];  // inclusive prefix sum of items per planner
  TcPlanner pl[kMaxPlanners];
  // DDIM teacher sampling (the sampler's step t of the launch is diffusion step
  // T-1-t): x_{next} = cx[t] x + cv[t] v, conditioning rows s [B][8], a [B][2],
  // step embeddings as BF16 rows of 64 ([T][8] uint4), samples out [B][8].
  const float* ddim_s;
  const float* ddim_a;
  const uint4* ddim_emb;
  float* ddim_y;
  float ddim_cx[64];
  float ddim_cv[64];
  // likelihood pairs: row i * B + j evaluates l([s'_i (8); a_i (2); o_j (6)]) -> out[row];
  // gather form (gather_node != null): row m evaluates
  // l([s'_m; act[node_m]; obs[node_m][branch_m]]) for rows m < pair_B
  const float* pair_s;
  const float* pair_a;
  const float* pair_o;
  long long pair_B;
  float* pair_out;
  const int32_t* gather_node;
  const int32_t* gather_branch;
  int gather_n_nodes, gather_C_max;
  // observation sampler (Eq. 5) of progressive widening: row i (i < *obs_count)
  // is simulation m = obs_list[i], input [s'_m (pair_s); act[node_m] (pair_a);
  // omega_Z] with omega_Z the normals of stream VOILA_STREAM_OBS_OMEGA at
  // counter (m, 0, obs_step); f_Z's output goes to obs_out[node_m][branch_m]
  // (obs_d values). Simulation indices are < pair_B.
  const int32_t* obs_list;
  const int32_t* obs_count;
  float* obs_out;
  int obs_d;
  uint32_t obs_step, obs_planner;
  // belief proposal (Sec. 3 SIR step): row i = particle i, s'_i = g_T([s_i; a;
  // omega_T]) with the noise of stream VOILA_STREAM_BELIEF_OMEGA at counter
  // (i, 0, prop_step), s'_i to prop_s, l([s'_i; a; o]) to prop_ell (the
  // likelihood is the second MLP, in the reward head's place); o has 6 values
  const float* prop_obs;
  float* prop_s;
  double* prop_ell;
  uint32_t prop_step;
};

__device__ __forceinline__ int item_planner(const TcParams& p, long long it) {
  int q = 0;
  while (q < p.P - 1 && it >= p.item_end[q]) ++q;
  return q;
}

__device__ __forceinline__ bool bounded_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                             WsHeader* hdr, int where, long long limit = kSpinLimit) {
  if (ptx::mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      set_status(hdr, VOILA_ERR_TIMEOUT, where);
      return false;
    }
  }
}

// ---- work-item queue (QUEUE instantiations) -------------------------------
// The even CTA's producer thread claims items from the global counter and
// posts each in slot j mod kItemRing of both CTAs' item rings (j = the
// cluster's item number); every other role of the pair (the MMA thread, the
// odd CTA's producer, each epilogue warp of both CTAs) takes item j from its
// own ring and frees the slot on the even CTA's item_empty barrier, so all
// roles walk the same items in the same order. -1 marks the end.
constexpr int kItemRing = 4;
constexpr int kItemTakers = 2 + 2 * (kTcThreads / 32 - 2);

// Static order: cluster c of n takes item j n + c in even rounds j and
// j n + (n - 1 - c) in odd ones when `serp` is set (a serpentine deal: with the
// items sorted by decreasing horizon, no cluster takes the largest item of
// every round), else j n + c.
__device__ __forceinline__ long long static_item(long long j, long long c, long long n, bool serp) {
  return j * n + ((serp && (j & 1)) ? n - 1 - c : c);
}

// bounded_wait with acquire semantics at cluster scope (the phase is completed
// by release arrivals of the other CTA of the pair as well).
__device__ __forceinline__ bool bounded_wait_cluster(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                                     WsHeader* hdr, int where) {
  if (ptx::mbar_try_wait_acq_cluster(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (ptx::mbar_try_wait_acq_cluster(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kSpinLimit) {
      *abort_flag = 1;
      set_status(hdr, VOILA_ERR_TIMEOUT, where);
      return false;
    }
  }
}

__device__ __forceinline__ long long claim_item(uint64_t* item_full, uint64_t* item_empty, long long* ring,
                                                long long j, unsigned long long* counter, long long total,
                                                volatile int* abort_flag, WsHeader* hdr) {
  const int sl = (int)(j % kItemRing);
  const uint32_t par = (uint32_t)((j / kItemRing) & 1);
  if (!bounded_wait_cluster(ptx::smem_u32(&item_empty[sl]), par ^ 1, abort_flag, hdr, 13)) return -2;
  const long long c = (long long)atomicAdd(counter, 1ull);
  const long long it = c < total ? c : -1;
  for (uint32_t r = 0; r < 2; ++r) {
    ptx::st_shared_cluster_s64(ptx::mapa_shared(ptx::smem_u32(&ring[sl]), r), it);
    ptx::mbar_arrive_release_cluster(ptx::mapa_shared(ptx::smem_u32(&item_full[sl]), r));
  }
  return it;
}

// Takes item j (-1: no more, -2: a wait expired). warp_wide: called by all 32
// lanes of a warp, which then agree on the result, and lane 0 frees the slot.
__device__ __forceinline__ long long take_item(uint64_t* item_full, uint64_t* item_empty, long long* ring,
                                               long long j, bool warp_wide, volatile int* abort_flag,
                                               WsHeader* hdr) {
  const int sl = (int)(j % kItemRing);
  const uint32_t par = (uint32_t)((j / kItemRing) & 1);
  const bool got = bounded_wait_cluster(ptx::smem_u32(&item_full[sl]), par, abort_flag, hdr, 14);
  long long it = got ? *reinterpret_cast<volatile long long*>(&ring[sl]) : -2;
  if (warp_wide) {
    if (!__all_sync(0xffffffffu, got)) return -2;
    it = __shfl_sync(0xffffffffu, it, 0);
  }
  if (!got) return -2;
  if (!warp_wide || (threadIdx.x & 31) == 0)
    ptx::mbar_arrive_release_cluster(ptx::mapa_shared(ptx::smem_u32(&item_empty[sl]), 0));
  return it;
}

// Activation of two accumulator values, packed to BF16x2 for the next layer.
// SiLU: the weights and bias of a SiLU layer are packed pre-scaled by 1/2
// (exact in BF16/FP32), so the accumulator holds u = x/2 and
// silu(x) = x sigmoid(x) = u (1 + tanh u) = fma(u, tanh u, u): one MUFU op
// (tanh.approx.f32; the packed BF16x2/FP16x2 forms measured slower on this
// part) and one FMA per value.
__device__ __forceinline__ float act_value(float u, int act) {
  if (act == VOILA_ACT_SILU) return fmaf(u, ptx::tanh_approx(u), u);
  if (act == VOILA_ACT_TANH) return ptx::tanh_approx(u);
  return u;
}

// SiLU (folded form above) of the pair (x0, x1) = z + b, or = z * sc + b for
// an E4M3 layer's channel scale, in packed FP32x2 arithmetic; returns the
// activations as a packed pair.
__device__ __forceinline__ uint64_t silu2(uint64_t x) {
  float u0, u1;
  ptx::f2_unpack(x, u0, u1);
  return ptx::f2_fma(x, ptx::f2_pack(ptx::tanh_approx(u0), ptx::tanh_approx(u1)), x);
}

__device__ __forceinline__ uint32_t silu2_bf16(uint64_t x) {
  float y0, y1;
  ptx::f2_unpack(silu2(x), y0, y1);
  return ptx::pack_bf16x2(y0, y1);
}

__device__ __forceinline__ uint32_t act_pair(float u0, float u1, int act) {
  if (act == VOILA_ACT_SILU)
    return ptx::pack_bf16x2(fmaf(u0, ptx::tanh_approx(u0), u0), fmaf(u1, ptx::tanh_approx(u1), u1));
  if (act == VOILA_ACT_TANH) return ptx::pack_bf16x2(ptx::tanh_approx(u0), ptx::tanh_approx(u1));
  return ptx::pack_bf16x2(u0, u1);
}

// 32 accumulator columns [32c, 32c + 32) of row r -> (channel scale) + bias +
// activation -> the next layer's A operand: BF16 (four 16-byte chunks, 64 K
// per 128-byte swizzled row) or E4M3 (two chunks, 128 K per row).
template <bool SCALE, bool OUT_FP8>
__device__ __forceinline__ void epi_cols32(float* u, const float* bl, const float* sl, int c, int act,
                                           uint8_t* A, int r) {
  if (!SCALE && !OUT_FP8) {  // BF16 -> BF16: bias, activation and store, eight columns at a time
    uint8_t* slab = A + (c >> 1) * (128 * 128);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 b0 = *reinterpret_cast<const float4*>(bl + 32 * c + 8 * j);
      const float4 b1 = *reinterpret_cast<const float4*>(bl + 32 * c + 8 * j + 4);
      uint4 o;
      if (act == VOILA_ACT_SILU) {
        using ptx::f2_add;
        using ptx::f2_pack;
        o.x = silu2_bf16(f2_add(f2_pack(u[8 * j + 0], u[8 * j + 1]), f2_pack(b0.x, b0.y)));
        o.y = silu2_bf16(f2_add(f2_pack(u[8 * j + 2], u[8 * j + 3]), f2_pack(b0.z, b0.w)));
        o.z = silu2_bf16(f2_add(f2_pack(u[8 * j + 4], u[8 * j + 5]), f2_pack(b1.x, b1.y)));
        o.w = silu2_bf16(f2_add(f2_pack(u[8 * j + 6], u[8 * j + 7]), f2_pack(b1.z, b1.w)));
      } else {
        o.x = act_pair(u[8 * j + 0] + b0.x, u[8 * j + 1] + b0.y, act);
        o.y = act_pair(u[8 * j + 2] + b0.z, u[8 * j + 3] + b0.w, act);
        o.z = act_pair(u[8 * j + 4] + b1.x, u[8 * j + 5] + b1.y, act);
        o.w = act_pair(u[8 * j + 6] + b1.z, u[8 * j + 7] + b1.w, act);
      }
      *reinterpret_cast<uint4*>(slab + r * 128 + ((((c & 1) * 4 + j) ^ (r & 7)) << 4)) = o;
    }
    return;
  }
  using ptx::f2_pack;
  // The E4M3 paths serve SiLU MLPs only (the FP8 form is refused for other activations).
  if (SCALE && !OUT_FP8) {  // E4M3 layer, BF16 output: one pass
    uint8_t* slab = A + (c >> 1) * (128 * 128);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t wv[4];
#pragma unroll
      for (int k2 = 0; k2 < 2; ++k2) {
        const int i = 8 * j + 4 * k2;
        const float4 b = *reinterpret_cast<const float4*>(bl + 32 * c + i);
        const float4 sc = *reinterpret_cast<const float4*>(sl + 32 * c + i);
        wv[2 * k2] = silu2_bf16(ptx::f2_fma(f2_pack(u[i], u[i + 1]), f2_pack(sc.x, sc.y), f2_pack(b.x, b.y)));
        wv[2 * k2 + 1] =
            silu2_bf16(ptx::f2_fma(f2_pack(u[i + 2], u[i + 3]), f2_pack(sc.z, sc.w), f2_pack(b.z, b.w)));
      }
      *reinterpret_cast<uint4*>(slab + r * 128 + ((((c & 1) * 4 + j) ^ (r & 7)) << 4)) =
          make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    return;
  }
  if (OUT_FP8) {
    // E4M3 output in one pass: (channel scale and) bias, SiLU, four values per
    // 32-bit word, sixteen per 16-byte chunk (128 K per 128-byte swizzled row)
    uint8_t* slab = A + (c >> 2) * (128 * 128);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t wv[4];
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) {
        const int i = 16 * j + 4 * k4;
        const float4 b = *reinterpret_cast<const float4*>(bl + 32 * c + i);
        uint64_t x01, x23;
        if (SCALE) {
          const float4 sc = *reinterpret_cast<const float4*>(sl + 32 * c + i);
          x01 = ptx::f2_fma(f2_pack(u[i], u[i + 1]), f2_pack(sc.x, sc.y), f2_pack(b.x, b.y));
          x23 = ptx::f2_fma(f2_pack(u[i + 2], u[i + 3]), f2_pack(sc.z, sc.w), f2_pack(b.z, b.w));
        } else {
          x01 = ptx::f2_add(f2_pack(u[i], u[i + 1]), f2_pack(b.x, b.y));
          x23 = ptx::f2_add(f2_pack(u[i + 2], u[i + 3]), f2_pack(b.z, b.w));
        }
        float y0, y1, y2, y3;
        ptx::f2_unpack(silu2(x01), y0, y1);
        ptx::f2_unpack(silu2(x23), y2, y3);
        wv[k4] = ptx::pack_e4m3x4(y0, y1, y2, y3);
      }
      *reinterpret_cast<uint4*>(slab + r * 128 + ((((c & 3) * 2 + j) ^ (r & 7)) << 4)) =
          make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
    return;
  }
}

// 16 accumulator columns [16b, 16b + 16) of row r, as epi_cols32 (layers whose
// quarter of the columns is 16 wide).
template <bool SCALE, bool OUT_FP8>
__device__ __forceinline__ void epi_cols16(float* u, const float* bl, const float* sl, int b, int act,
                                           uint8_t* A, int r) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 bb = *reinterpret_cast<const float4*>(bl + 16 * b + 4 * j);
    if (SCALE) {
      const float4 sc = *reinterpret_cast<const float4*>(sl + 16 * b + 4 * j);
      u[4 * j + 0] = fmaf(u[4 * j + 0], sc.x, bb.x);
      u[4 * j + 1] = fmaf(u[4 * j + 1], sc.y, bb.y);
      u[4 * j + 2] = fmaf(u[4 * j + 2], sc.z, bb.z);
      u[4 * j + 3] = fmaf(u[4 * j + 3], sc.w, bb.w);
    } else {
      u[4 * j + 0] += bb.x;
      u[4 * j + 1] += bb.y;
      u[4 * j + 2] += bb.z;
      u[4 * j + 3] += bb.w;
    }
  }
  if (!OUT_FP8) {
    uint8_t* slab = A + (b >> 2) * (128 * 128);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint4 o;
      o.x = act_pair(u[8 * j + 0], u[8 * j + 1], act);
      o.y = act_pair(u[8 * j + 2], u[8 * j + 3], act);
      o.z = act_pair(u[8 * j + 4], u[8 * j + 5], act);
      o.w = act_pair(u[8 * j + 6], u[8 * j + 7], act);
      *reinterpret_cast<uint4*>(slab + r * 128 + ((((b & 3) * 2 + j) ^ (r & 7)) << 4)) = o;
    }
  } else {
    uint8_t* slab = A + (b >> 3) * (128 * 128);
    uint4 o;
    o.x = ptx::pack_e4m3x4(act_value(u[0], act), act_value(u[1], act), act_value(u[2], act), act_value(u[3], act));
    o.y = ptx::pack_e4m3x4(act_value(u[4], act), act_value(u[5], act), act_value(u[6], act), act_value(u[7], act));
    o.z = ptx::pack_e4m3x4(act_value(u[8], act), act_value(u[9], act), act_value(u[10], act), act_value(u[11], act));
    o.w = ptx::pack_e4m3x4(act_value(u[12], act), act_value(u[13], act), act_value(u[14], act), act_value(u[15], act));
    *reinterpret_cast<uint4*>(slab + r * 128 + (((b & 7) ^ (r & 7)) << 4)) = o;
  }
}

// The columns [W c, W c + W) of row r of a layer followed by a fused scalar
// output: (channel scale) + bias + activation, dotted in FP32 with the output
// weights wf (the activations are not rounded to BF16). The dot product runs
// as two interleaved partial sums (even and odd columns) in one FP32x2
// register; the caller adds the two halves.
template <bool SCALE, int W>
__device__ __forceinline__ uint64_t fuse_cols(const float* u, const float* bl, const float* sl, int c, int act,
                                              const float* wf, uint64_t part) {
  using ptx::f2_pack;
#pragma unroll
  for (int j = 0; j < W; j += 4) {
    const float4 b = *reinterpret_cast<const float4*>(bl + W * c + j);
    const float4 w = *reinterpret_cast<const float4*>(wf + W * c + j);
    uint64_t x01, x23;
    if (SCALE) {
      const float4 sc = *reinterpret_cast<const float4*>(sl + W * c + j);
      x01 = ptx::f2_fma(f2_pack(u[j], u[j + 1]), f2_pack(sc.x, sc.y), f2_pack(b.x, b.y));
      x23 = ptx::f2_fma(f2_pack(u[j + 2], u[j + 3]), f2_pack(sc.z, sc.w), f2_pack(b.z, b.w));
    } else {
      x01 = ptx::f2_add(f2_pack(u[j], u[j + 1]), f2_pack(b.x, b.y));
      x23 = ptx::f2_add(f2_pack(u[j + 2], u[j + 3]), f2_pack(b.z, b.w));
    }
    if (SCALE || act == VOILA_ACT_SILU) {  // E4M3 layers: SiLU MLPs only
      x01 = silu2(x01);
      x23 = silu2(x23);
    } else {
      float y0, y1, y2, y3;
      ptx::f2_unpack(x01, y0, y1);
      ptx::f2_unpack(x23, y2, y3);
      x01 = f2_pack(act_value(y0, act), act_value(y1, act));
      x23 = f2_pack(act_value(y2, act), act_value(y3, act));
    }
    part = ptx::f2_fma(x01, f2_pack(w.x, w.y), part);
    part = ptx::f2_fma(x23, f2_pack(w.z, w.w), part);
  }
  return part;
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

// The rollout epilogues keep a row's generator inputs as packed BF16 words
// (every one of them is rounded to BF16 where it enters an MMA): the state
// s_t as DS / 2 words and the tail [a_t; omega_T(n, k, t)] as
// (DA + DW + 1) / 2 words (an odd last word has a zero high half).
template <int KP>
__device__ __forceinline__ void store_words(uint8_t* A, int r, const uint32_t* x) {
#pragma unroll
  for (int j = 0; j < KP / 8; ++j)
    *reinterpret_cast<uint4*>(a_chunk(A, r, j)) = make_uint4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
}

template <int DS>
__device__ __forceinline__ void pack_state(uint32_t* s_pk, const float* s) {
#pragma unroll
  for (int i = 0; i < DS / 2; ++i) s_pk[i] = ptx::pack_bf16x2(s[2 * i], s[2 * i + 1]);
}

// [a_t; omega_T(n, k, t)] of one row, packed: a_t = act[0 .. DA), the noise
// from stream VOILA_STREAM_ROLLOUT_OMEGA at counter (n, k, t).
template <int DA, int DW>
__device__ __forceinline__ void draw_tail(uint32_t* tail, const float* act, uint32_t k0, uint32_t k1, uint32_t n,
                                          uint32_t k, uint32_t t, uint32_t planner,
                                          uint32_t stream = VOILA_STREAM_ROLLOUT_OMEGA) {
  constexpr int TE = 2 * ((DA + DW + 1) / 2);
  float e[TE];
#pragma unroll
  for (int i = 0; i < TE; ++i) e[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < DA; ++i) e[i] = __ldg(act + i);
#pragma unroll
  for (int b = 0; b < (DW + 3) / 4; ++b) {
    const float4 z = normal4(k0, k1, n, k, t, stream, planner, (uint32_t)b);
    if (4 * b + 0 < DW) e[DA + 4 * b + 0] = z.x;
    if (4 * b + 1 < DW) e[DA + 4 * b + 1] = z.y;
    if (4 * b + 2 < DW) e[DA + 4 * b + 2] = z.z;
    if (4 * b + 3 < DW) e[DA + 4 * b + 3] = z.w;
  }
#pragma unroll
  for (int j = 0; j < TE / 2; ++j) tail[j] = ptx::pack_bf16x2(e[2 * j], e[2 * j + 1]);
}

// The a_t words of a tail (the odd last one with its high half cleared).
template <int DA>
__device__ __forceinline__ void tail_actions(uint32_t* a_pk, const uint32_t* tail) {
#pragma unroll
  for (int i = 0; i < DA / 2; ++i) a_pk[i] = tail[i];
  if (DA & 1) a_pk[DA / 2] = tail[DA / 2] & 0xFFFFu;
}

// Generator input row [s_t; a_t; omega_T(n, k, t)], zero padded.
template <int DS, int DA, int DW>
__device__ __forceinline__ void write_gen_row(uint8_t* A, int r, const uint32_t* s_pk, const uint32_t* tail) {
  static_assert(DS % 2 == 0, "the state fills whole BF16 pairs");
  constexpr int KP = (DS + DA + DW + 15) / 16 * 16;
  uint32_t x[KP / 2];
#pragma unroll
  for (int i = 0; i < KP / 2; ++i) x[i] = 0u;
#pragma unroll
  for (int i = 0; i < DS / 2; ++i) x[i] = s_pk[i];
#pragma unroll
  for (int i = 0; i < (DA + DW + 1) / 2; ++i) x[DS / 2 + i] = tail[i];
  store_words<KP>(A, r, x);
}

// Reward-head input row [s_{t+1}; a_t], zero padded.
template <int DS, int DA>
__device__ __forceinline__ void write_rew_row(uint8_t* A, int r, const uint32_t* s_pk, const uint32_t* a_pk) {
  constexpr int KP = (DS + DA + 15) / 16 * 16;
  uint32_t x[KP / 2];
#pragma unroll
  for (int i = 0; i < KP / 2; ++i) x[i] = 0u;
#pragma unroll
  for (int i = 0; i < DS / 2; ++i) x[i] = s_pk[i];
#pragma unroll
  for (int i = 0; i < (DA + 1) / 2; ++i) x[DS / 2 + i] = a_pk[i];
  store_words<KP>(A, r, x);
}

// Likelihood input row [s'; a; o] (belief proposal), o as BF16 pairs, zero padded.
template <int DS, int DA>
__device__ __forceinline__ void write_lik_row(uint8_t* A, int r, const uint32_t* s_pk, const float* a,
                                              const float* o) {
  constexpr int DO = 6;
  constexpr int KP = (DS + DA + DO + 15) / 16 * 16;
  float x[KP];
#pragma unroll
  for (int i = 0; i < KP; ++i) x[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < DA; ++i) x[DS + i] = a[i];
#pragma unroll
  for (int i = 0; i < DO; ++i) x[DS + DA + i] = o[i];
  uint32_t w[KP / 2];
#pragma unroll
  for (int i = 0; i < KP / 2; ++i) w[i] = 2 * i < DS ? s_pk[i] : ptx::pack_bf16x2(x[2 * i], x[2 * i + 1]);
  store_words<KP>(A, r, w);
}

// Teacher input row of the DDIM sampler, in the column order the packed first
// layer expects: [x (8) | s (8) | a (2), 0 (6) | 0 (8) | e(t) (64)], 96 BF16
// columns = chunks 0-7 of slab 0 and chunks 0-3 of slab 1.
__device__ __forceinline__ void write_ddim_input(uint8_t* A, int r, const float* x, const float* c,
                                                 const uint4* emb_row) {
  store_row<8>(A, r, x);
  uint4 v;
  v.x = ptx::pack_bf16x2(c[0], c[1]);
  v.y = ptx::pack_bf16x2(c[2], c[3]);
  v.z = ptx::pack_bf16x2(c[4], c[5]);
  v.w = ptx::pack_bf16x2(c[6], c[7]);
  *reinterpret_cast<uint4*>(a_chunk(A, r, 1)) = v;
  v.x = ptx::pack_bf16x2(c[8], c[9]);
  v.y = v.z = v.w = 0u;
  *reinterpret_cast<uint4*>(a_chunk(A, r, 2)) = v;
  v.x = 0u;
  *reinterpret_cast<uint4*>(a_chunk(A, r, 3)) = v;
#pragma unroll
  for (int j = 0; j < 4; ++j) *reinterpret_cast<uint4*>(a_chunk(A, r, 4 + j)) = __ldg(emb_row + j);
#pragma unroll
  for (int j = 0; j < 4; ++j) *reinterpret_cast<uint4*>(a_chunk(A + 128 * 128, r, j)) = __ldg(emb_row + 4 + j);
}

// Likelihood-pair input row [s'_i; a_i; o_j] of pair row `row` (row = i B + j),
// or in the gather form [s'_m; act[node_m]; obs[node_m][branch_m]] (row = m),
// as BF16; zeros for rows past the end or out-of-range indices.
__device__ __forceinline__ void write_pair_row(const TcParams& p, uint8_t* A, int r, long long row, bool valid) {
  long long pi, pa, po;  // rows of s', a and o
  bool in = valid;
  if (p.gather_node) {
    const int an = valid ? __ldg(p.gather_node + row) : -1;
    in = an >= 0 && an < p.gather_n_nodes;
    pi = row;
    pa = in ? an : 0;
    po = in ? (long long)an * p.gather_C_max + __ldg(p.gather_branch + row) : 0;
  } else {
    pi = valid ? row / p.pair_B : 0;
    pa = pi;
    po = valid ? row % p.pair_B : 0;
  }
  float x[16];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = in ? __ldg(p.pair_s + pi * 8 + i) : 0.0f;
  x[8] = in ? __ldg(p.pair_a + pa * 2) : 0.0f;
  x[9] = in ? __ldg(p.pair_a + pa * 2 + 1) : 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) x[10 + i] = in ? __ldg(p.pair_o + po * 6 + i) : 0.0f;
  store_row<16>(A, r, x);
}

// F8: the MLPs contain E4M3 layers (a separate instantiation keeps the BF16
// form free of the FP8 code paths).
// WIDE: layers up to 512 wide. Each CTA owns one 128-row tile per work item
// (256 rows per pair); the two 256-column TMEM halves and the two 64 KB A
// buffers hold the two column halves of a layer (K up to 512); the epilogue
// drains half 0 while the MMAs of half 1 run, and the next layer's MMAs on
// K < 256 start while it drains half 1.
// MODE kModeDdim (with WIDE, DS = 8, DA = 10, DW = 0): the rows are teacher
// samples and the H steps are the sampler's steps; no reward, the output is x
// per row. MODE kModePairs (DS = 8, DA = 2, DW = 6, not WIDE): the rows are
// likelihood pairs; the MLP's scalar output is stored per row.
template <int DS, int DA, int DW, bool F8, bool WIDE, int MODE = kModeRollout, bool QUEUE = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTcThreads, 1)
    rollout_tc_kernel(const __grid_constant__ TcParams p) {
  constexpr bool DDIM = MODE == kModeDdim;
  constexpr bool PAIRS = MODE == kModePairs;
  constexpr bool OBS = MODE == kModeObserve;
  static_assert(!DDIM || (WIDE && !F8 && DS == 8 && DA == 10 && DW == 0), "DDIM sampler layout");
  static_assert(!PAIRS || (!WIDE && !F8 && DS == 8 && DA == 2 && DW == 6), "likelihood pair layout");
  static_assert(!OBS || (!WIDE && !F8), "observation rows use the two-tile kernel");
  constexpr bool PROP = MODE == kModePropose;
  static_assert(!PROP || (!WIDE && DS == 8 && DA == 2 && DW == 8), "belief proposal layout");
  static_assert(!QUEUE || MODE == kModeRollout, "the work-item queue serves the rollout");
  // the static order is dealt serpentine for rollouts (items of uneven cost in
  // a batched launch); the pair mode's look-ahead assumes the plain order
  constexpr bool SERP = MODE == kModeRollout;
  // work items of the launch: the observation rows are counted on the device
  long long total_items = p.total_items;
  if constexpr (OBS) {
    const int cnt = *reinterpret_cast<const volatile int*>(p.obs_count);
    const long long need = cnt > 0 ? ((long long)cnt + kSuperRows - 1) / kSuperRows : 0;
    if (need < total_items) total_items = need;
  }
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* Abuf[2] = {smem, smem + kABytes};
  uint8_t* ring = smem + 2 * kABytes;
  float* bias_s = reinterpret_cast<float*>(ring + kStages * kSlotBytes);
  float* scale_s = bias_s + p.bias_total;  // FP8 channel scales follow the biases
  float* fuse_s = scale_s + p.scale_total;  // fused scalar-output weights and biases
  float* red_s = fuse_s + p.fuse_total;     // [2 tiles][4 column slices][128 rows] partial sums
  uint64_t* bars = reinterpret_cast<uint64_t*>(red_s + (p.fuse_total ? 1024 : 0));
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* accf = bars + 2 * kStages;      // [2]
  uint64_t* ready = bars + 2 * kStages + 2;  // [2]
  uint64_t* drain = bars + 2 * kStages + 4;
  uint64_t* item_full = bars + 2 * kStages + 5;               // [kItemRing]
  uint64_t* item_empty = item_full + kItemRing;               // [kItemRing]
  long long* item_ring = reinterpret_cast<long long*>(item_empty + kItemRing);  // [kItemRing]
  uint64_t* alo_free = reinterpret_cast<uint64_t*>(item_ring + kItemRing);  // wide: A columns 0..255 read
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(alo_free + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = ptx::cluster_ctarank();  // 0: issues the pair MMAs
  const long long cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);   // even CTA's expect_tx; both CTAs' bytes
      ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);  // one multicast commit
    }
    for (int g = 0; g < 2; ++g) {
      ptx::mbar_init(ptx::smem_u32(&accf[g]), 1);
      // every epilogue warp of both CTAs
      ptx::mbar_init(ptx::smem_u32(&ready[g]), 4 * kEpiWarpsPerTile);
    }
    ptx::mbar_init(ptx::smem_u32(drain), 1);
    ptx::mbar_init(ptx::smem_u32(alo_free), 1);
    for (int i = 0; i < kItemRing; ++i) {
      ptx::mbar_init(ptx::smem_u32(&item_full[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&item_empty[i]), kItemTakers);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  for (int i = threadIdx.x; i < p.bias_total + p.scale_total + p.fuse_total; i += blockDim.x)
    bias_s[i] = p.bias_all[i];
  if (warp == 1) {
    ptx::tmem_alloc_pair(ptx::smem_u32(tmem_holder), 512);
    ptx::tmem_relinquish_pair();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();  // barriers of both CTAs initialised before any remote arrive
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  const uint32_t ring_addr = ptx::smem_u32(ring);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      for (int l = 0; l < p.n_total; ++l) ptx::prefetch_tmap(&p.tmap[l]);
      int slot = 0;
      uint32_t phase = 0;  // parity of the ring round of `slot`
      bool ok = true;
      int last_round[kStages];
      for (int s = 0; s < kStages; ++s) last_round[s] = -1;
      long long jq = 0;  // queue: the cluster's item number
      for (long long it = QUEUE ? (rank == 0 ? claim_item(item_full, item_empty, item_ring, jq, p.queue, total_items,
                                                          abort_flag, p.hdr)
                                             : take_item(item_full, item_empty, item_ring, jq, false, abort_flag,
                                                         p.hdr))
                                : cl;
           it >= 0 && it < total_items && ok;
           it = QUEUE ? (rank == 0 ? claim_item(item_full, item_empty, item_ring, ++jq, p.queue, total_items,
                                                abort_flag, p.hdr)
                                   : take_item(item_full, item_empty, item_ring, ++jq, false, abort_flag, p.hdr))
                      : (SERP ? static_item(++jq, cl, ncl, true) : it + ncl)) {
        const int H = p.pl[item_planner(p, it)].H;
        for (int t = 0; t < H && ok; ++t)
          for (int l = 0; l < p.n_total && ok; ++l)
            // two-tile kernel: a chunk is loaded once and serves both tiles' MMAs
            for (int g = 0; g < (WIDE ? p.layers[l].ngroups : 1) && ok; ++g) {
              const TcLayer& L = p.layers[l];
              // rows of this CTA's half of the chunk (wide: of column group g)
              const int rowoff = (WIDE ? g * 256 : 0) + (int)rank * L.box_rows;
              for (int c = 0; c < L.nchunks; ++c) {
                if (!bounded_wait(ptx::smem_u32(&empty[slot]), phase ^ 1, abort_flag, p.hdr, 10)) {
                  ok = false;
                  break;
                }
                const uint32_t full_local = ptx::smem_u32(&full[slot]);
                const int s0 = c * L.spc;
                const int ns = L.nslabs - s0 < L.spc ? L.nslabs - s0 : L.spc;
                if (rank == 0) ptx::mbar_arrive_expect_tx(full_local, (uint32_t)(2 * ns * L.slab_bytes));
                const uint32_t full_leader = ptx::mapa_shared(full_local, 0);
                for (int j = 0; j < ns; ++j)
                  ptx::tma_load_2d_pair(ring_addr + slot * kSlotBytes + j * L.slab_bytes, &p.tmap[l], 0,
                                        L.row0 + (s0 + j) * L.Npad + rowoff, full_leader);
                last_round[slot] = (int)phase;
                if (++slot == kStages) {
                  slot = 0;
                  phase ^= 1;
                }
              }
            }
      }
      if (QUEUE && *abort_flag) ok = false;  // a claim or take that gave up ended the loop
      if (!ok && rank == 0) {  // drain loads still in flight before shared memory goes away
        for (int s = 0; s < kStages; ++s)
          if (last_round[s] >= 0) {
            const long long t0 = clock64();
            while (!ptx::mbar_try_wait_cluster(ptx::smem_u32(&full[s]), (uint32_t)last_round[s] & 1) &&
                   clock64() - t0 < kSpinLimit) {
            }
          }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (even CTA)
    if (lane == 0) {
      if (rank == 0) {
        int slot = 0;
        uint32_t phase = 0;  // parity of the ring round of `slot`
        uint32_t nready0 = 0, nready1 = 0;
        bool ok = true;
        // Descriptors are built once; per chunk and K step only the start
        // address field (bits 0-13, address >> 4) moves. The issuing thread
        // shares its scheduler with epilogue warps, so its loop is kept short.
        const uint64_t adesc0 = ptx::smem_desc(ptx::smem_u32(Abuf[0]), 1024, ptx::kSwizzle128B);
        const uint64_t adesc1 = ptx::smem_desc(ptx::smem_u32(Abuf[1]), 1024, ptx::kSwizzle128B);
        const uint64_t bdesc0 = ptx::smem_desc(ring_addr, 1024, ptx::kSwizzle128B);
        long long jq = 0;
        for (long long it = QUEUE ? take_item(item_full, item_empty, item_ring, jq, false, abort_flag, p.hdr)
                                  : cl;
             it >= 0 && it < total_items && ok;
             it = QUEUE ? take_item(item_full, item_empty, item_ring, ++jq, false, abort_flag, p.hdr)
                        : (SERP ? static_item(++jq, cl, ncl, true) : it + ncl)) {
          const int H = p.pl[item_planner(p, it)].H;
          for (int t = 0; t < H && ok; ++t)
            for (int l = 0; l < p.n_total && ok; ++l) {
              const int nch = p.layers[l].nchunks, ksteps = p.layers[l].ksteps;
              const bool f8 = F8 && p.layers[l].fp8 != 0;
              const int kpc = 4 * p.layers[l].spc;  // K steps per chunk
              const uint32_t slab16 = (uint32_t)p.layers[l].slab_bytes >> 4;
              const uint32_t idesc = p.layers[l].idesc;
              // two-tile kernel: tile 1 reuses the slots tile 0 read (the chunks of
              // a layer, at most four, stay in the ring until tile 1's MMAs on them
              // complete), so every weight chunk crosses from L2 once per layer
              const int slot0 = slot;
              const uint32_t phase0 = phase;
              // wide kernel: ready[0] says the previous layer's epilogue has written A
              // columns 0..255 and read TMEM half 0, ready[1] the same of columns
              // 256..511 and half 1; the MMAs on K < 256 start on ready[0] alone
              bool hi_done = !WIDE;
              const int kchunk = p.layers[l].spc * (f8 ? 128 : 64);  // K of one chunk
              const int last_lo = (256 / kchunk < nch ? 256 / kchunk : nch) - 1;  // last chunk of K < 256
              // A half of K < 256 (16-byte units: 64 KB of BF16 or 32 KB of E4M3 per half)
              const uint32_t amask = (WIDE && p.layers[l].rot) ? (f8 ? 2048u : 4096u) : 0u;
              for (int g = 0; g < (WIDE ? p.layers[l].ngroups : 2) && ok; ++g) {
                if (!WIDE) {
                  slot = slot0;
                  phase = phase0;
                }
                // both CTAs' A operands of tile g are written and their accumulators read
                // (wide: A columns 0..255 and TMEM half 0 before group 0, TMEM half 1
                // before group 1)
                if (!WIDE || g == 0) {
                  if (!bounded_wait(ptx::smem_u32(&ready[g]), (g ? nready1 : nready0) & 1, abort_flag, p.hdr, 21 + g)) {
                    ok = false;
                    break;
                  }
                  if (g) ++nready1;
                  else ++nready0;
                  ptx::tc_fence_after();
                } else if (!hi_done) {
                  if (!bounded_wait(ptx::smem_u32(&ready[1]), nready1 & 1, abort_flag, p.hdr, 22)) {
                    ok = false;
                    break;
                  }
                  ++nready1;
                  hi_done = true;
                  ptx::tc_fence_after();
                }
                const uint64_t ad_tile = (!WIDE && g) ? adesc1 : adesc0;
                const uint32_t ad_lo = (uint32_t)ad_tile, ad_hi = (uint32_t)(ad_tile >> 32);
                const uint32_t bd_lo = (uint32_t)bdesc0, bd_hi = (uint32_t)(bdesc0 >> 32);
                const uint32_t d_tmem = tmem_base + g * 256;
                for (int c = 0; c < nch; ++c) {
                  // the TMA transaction count on this CTA's barrier covers both halves
                  const uint32_t fb = ptx::smem_u32(&full[slot]);
                  bool landed = ptx::mbar_try_wait(fb, phase);
                  if (!landed) {
                    const long long t0 = clock64();
                    while (!(landed = ptx::mbar_try_wait(fb, phase))) {
                      if (*abort_flag) break;
                      if (clock64() - t0 > kSpinLimit) {
                        *abort_flag = 1;
                        set_status(p.hdr, VOILA_ERR_TIMEOUT, 20);
                        break;
                      }
                    }
                  }
                  if (!landed) {
                    ok = false;
                    break;
                  }
                  if (WIDE && !hi_done && c > last_lo) {  // K >= 256: A columns 256..511
                    if (!bounded_wait(ptx::smem_u32(&ready[1]), nready1 & 1, abort_flag, p.hdr, 22)) {
                      ok = false;
                      break;
                    }
                    ++nready1;
                    hi_done = true;
                    ptx::tc_fence_after();
                  }
                  // chunk c = K steps [kpc c, kpc c + kpc): K step j sits in A slab j / 4 and in B
                  // slab (j mod kpc) / 4 of the slot; each K step is +32 bytes (+2 in the
                  // descriptor's address field) inside a slab
                  const int kb = kpc * c;
                  const uint32_t a_lo = ad_lo + (((uint32_t)(kb >> 2) * 1024u) ^ amask);
                  const uint32_t b_lo = bd_lo + (uint32_t)slot * (uint32_t)(kSlotBytes >> 4);
                  const int ks = ksteps - kb < kpc ? ksteps - kb : kpc;
                  if (F8 && kpc == 4 && f8) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                      if (kk < ks)
                        ptx::mma_f8_pair(d_tmem, ptx::desc_with_lo(ad_hi, a_lo + 2 * kk),
                                         ptx::desc_with_lo(bd_hi, b_lo + 2 * kk), idesc, (c | kk) ? 1u : 0u);
                  } else if (kpc == 4) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                      if (kk < ks)
                        ptx::mma_bf16_pair(d_tmem, ptx::desc_with_lo(ad_hi, a_lo + 2 * kk),
                                           ptx::desc_with_lo(bd_hi, b_lo + 2 * kk), idesc, (c | kk) ? 1u : 0u);
                  } else {
                    for (int kk = 0; kk < ks; ++kk)
                      ptx::mma_bf16_pair(d_tmem, ptx::desc_with_lo(ad_hi, a_lo + (kk >> 2) * 1024u + 2 * (kk & 3)),
                                         ptx::desc_with_lo(bd_hi, b_lo + (kk >> 2) * slab16 + 2 * (kk & 3)), idesc,
                                         (c | kk) ? 1u : 0u);
                  }
                  if (WIDE || g == 1) ptx::mma_commit_pair(ptx::smem_u32(&empty[slot]), 0x3);
                  // wide: the layer's MMAs on A columns 0..255 are issued; the
                  // epilogue may overwrite them once these complete
                  if (WIDE && g == p.layers[l].ngroups - 1 && c == last_lo)
                    ptx::mma_commit_pair(ptx::smem_u32(alo_free), 0x3);
                  if (c == nch - 1) ptx::mma_commit_pair(ptx::smem_u32(&accf[g]), 0x3);
                  if (++slot == kStages) {
                    slot = 0;
                    phase ^= 1;
                  }
                }
              }
              if (WIDE && ok && !hi_done) {  // one ready[1] phase per layer
                if (!bounded_wait(ptx::smem_u32(&ready[1]), nready1 & 1, abort_flag, p.hdr, 22)) {
                  ok = false;
                  break;
                }
                ++nready1;
                ptx::tc_fence_after();
              }
            }
        }
        // every MMA issued so far has completed once both CTAs' drain barriers arrive
        ptx::mma_commit_pair(ptx::smem_u32(drain), 0x3);
      }
      const long long t0 = clock64();
      while (!ptx::mbar_try_wait(ptx::smem_u32(drain), 0) && clock64() - t0 < kSpinLimit) {
      }
    }
  } else if constexpr (WIDE) {
    // ------------------------------------------------------------ epilogue (wide)
    // One tile per CTA and work item. A layer's output is drained in two
    // phases, each by all sixteen warps: TMEM half 0 (columns 0..255) as soon
    // as its MMAs complete, while the MMAs of half 1 run, then half 1. Phase 0
    // stores into A columns 0..255 once the MMAs reading them have completed
    // (alo_free) and announces them on ready[0], so the next layer's MMAs on K
    // < 256 start while phase 1 runs; phase 1 announces columns 256..511 on
    // ready[1]. Warp w may read TMEM lanes 32*(w % 4) .. +31 (its rows); the
    // four warps of a lane quadrant take 32-column batches in turn. The
    // slice-0 warps also own the row state.
    const int e = warp - 2;
    const int slice = e >> 2;               // batches slice, slice + 4, ... of a TMEM half
    const int q = warp & 3;                 // TMEM lane quadrant this warp may access
    const int r = 32 * q + lane;            // row within the tile
    const bool owner = slice == 0;          // holds the row state
    uint8_t* A = Abuf[0];                   // with Abuf[1]: one K = 512 operand
    const uint32_t tm = tmem_base + ((uint32_t)(32 * q) << 16);
    const uint32_t ready_lo = ptx::mapa_shared(ptx::smem_u32(&ready[0]), 0);  // even CTA's
    const uint32_t ready_hi = ptx::mapa_shared(ptx::smem_u32(&ready[1]), 0);
    const uint32_t acc_bar = ptx::smem_u32(&accf[0]);
    const uint32_t acc_bar1 = ptx::smem_u32(&accf[1]);
    const uint32_t alo_bar = ptx::smem_u32(alo_free);
    uint32_t nacc = 0, nacc1 = 0, nalo = 0;
    bool ok = true;
    long long jq = 0;
    for (long long it = QUEUE ? take_item(item_full, item_empty, item_ring, jq, true, abort_flag, p.hdr)
                              : cl;
         it >= 0 && it < total_items && ok;
         it = QUEUE ? take_item(item_full, item_empty, item_ring, ++jq, true, abort_flag, p.hdr)
                    : (SERP ? static_item(++jq, cl, ncl, true) : it + ncl)) {
      const int q = item_planner(p, it);
      const long long sp = it - (q ? p.item_end[q - 1] : 0);
      const TcPlanner& PL = p.pl[q];
      const int H = PL.H;
      const long long row = sp * (2 * kTileRows) + (long long)rank * kTileRows + r;
      const bool valid = row < PL.rows;
      const uint32_t n = valid ? (uint32_t)(row % PL.N) : 0u;
      const uint32_t k = valid ? (uint32_t)(row / PL.N) : 0u;
      const float* act_row = PL.actions + (size_t)k * H * DA;
      const uint32_t nc = n + PL.n_off, kc = k + PL.k_off;  // noise counters of the unsharded problem
      float s[DS], a[DA];  // sampler mode: x_t and the conditioning [s; a]
      // rollout mode: the row state as packed BF16 words (s_t, a_t and the
      // next step's tail [a_{t+1}; omega_T(n, k, t + 1)], drawn while the
      // generator's output layer is on the tensor cores)
      uint32_t s_pk[DS / 2], a_pk[(DA + 1) / 2], tn[(DA + DW + 1) / 2];
      if constexpr (DDIM) {
        if (owner) {  // s holds x_t, a the conditioning [s; a] of the row
#pragma unroll
          for (int i = 0; i < DS; ++i) s[i] = valid ? __ldg(PL.particles + (size_t)row * DS + i) : 0.0f;
#pragma unroll
          for (int i = 0; i < 8; ++i) a[i] = valid ? __ldg(p.ddim_s + (size_t)row * 8 + i) : 0.0f;
          a[8] = valid ? __ldg(p.ddim_a + (size_t)row * 2) : 0.0f;
          a[9] = valid ? __ldg(p.ddim_a + (size_t)row * 2 + 1) : 0.0f;
          write_ddim_input(A, r, s, a, p.ddim_emb);
        }
      } else if constexpr (PAIRS) {
        if (owner) write_pair_row(p, A, r, row, valid);
      } else if (owner) {
#pragma unroll
        for (int i = 0; i < DS; ++i) s[i] = valid ? __ldg(PL.particles + (size_t)n * DS + i) : 0.0f;
        pack_state<DS>(s_pk, s);
        draw_tail<DA, DW>(tn, act_row, p.key0, p.key1, nc, kc, 0u, PL.planner);
        write_gen_row<DS, DA, DW>(A, r, s_pk, tn);
        tail_actions<DA>(a_pk, tn);
      }
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        ptx::mbar_arrive_cluster(ready_lo);
        ptx::mbar_arrive_cluster(ready_hi);
      }
      double Gacc = 0.0, disc = 1.0;
      for (int t = 0; t < H && ok; ++t) {
        for (int l = 0; l < p.n_total; ++l) {
          const TcLayer& L = p.layers[l];
          if constexpr (!DDIM && !PAIRS) {
            if (owner && l == p.n_gen - 1 && t + 1 < H)
              draw_tail<DA, DW>(tn, act_row + (t + 1) * DA, p.key0, p.key1, nc, kc, (uint32_t)(t + 1), PL.planner);
          }
          const float* bl = bias_s + L.bias_off;  // shared memory (L1 loads measured slower)
          // no A operand follows the final layer of the final step
          const bool arrive = !(t == H - 1 && l == p.n_total - 1);
          bool lo_free = false;  // the MMAs reading A columns 0..255 have completed
          // The next layer reads its K < 256 from A half rot_next; half h of this
          // output goes to A half h ^ rot_next. When that differs from this layer's
          // own rot (a layer with K <= 256 reads one A half only), phase 0 writes the
          // half this layer does not read and need not wait for alo_free.
          const int rot_next = (L.act >= 0 && l + 1 < p.n_total) ? p.layers[l + 1].rot : 0;
          const bool lo_need = L.act < 0 || rot_next == L.rot;
          for (int h = 0; h < L.ngroups && ok; ++h) {
            if (!bounded_wait(h ? acc_bar1 : acc_bar, (h ? nacc1 : nacc) & 1, abort_flag, p.hdr, 30 + h)) {
              ok = false;
              break;
            }
            if (h) ++nacc1;
            else ++nacc;
            ptx::tc_fence_after();
            if (L.act >= 0) {
              // hidden layer: bias + activation -> A operand of the next layer,
              // 32 columns per TMEM load (measured faster than larger batches)
              const int nb = (L.Npad > 256 ? 256 : L.Npad) >> 5;  // 32-column batches of a TMEM half
              for (int bt = slice; bt < nb; bt += 4) {
                float v[32];
                ptx::tmem_ld32(tm + (uint32_t)(256 * h + 32 * bt), v);
                ptx::tmem_wait_ld32(v);
                if (!lo_free && lo_need) {
                  if (!bounded_wait(alo_bar, nalo & 1, abort_flag, p.hdr, 33)) {
                    ok = false;
                    break;
                  }
                  ++nalo;
                  lo_free = true;
                }
                // batch c of the layer (its biases and scales) is stored as A batch
                // ca; epi_cols32 addresses both through its batch argument
                const int c = 8 * h + bt, ca = c ^ (8 * rot_next);
                const float* blc = bl + 32 * (c - ca);
                const float* slc = scale_s + L.scale_off + 32 * (c - ca);
                if (!F8) {
                  epi_cols32<false, false>(v, blc, nullptr, ca, L.act, A, r);
                } else if (L.out_fp8) {
                  if (L.fp8) epi_cols32<true, true>(v, blc, slc, ca, L.act, A, r);
                  else epi_cols32<false, true>(v, blc, nullptr, ca, L.act, A, r);
                } else {
                  if (L.fp8) epi_cols32<true, false>(v, blc, slc, ca, L.act, A, r);
                  else epi_cols32<false, false>(v, blc, nullptr, ca, L.act, A, r);
                }
              }
            }
            if (h == 1 || !ok) break;
            if (!lo_free && lo_need) {
              if (!bounded_wait(alo_bar, nalo & 1, abort_flag, p.hdr, 33)) {
                ok = false;
                break;
              }
              ++nalo;
              lo_free = true;
            }
            if (L.act >= 0) {
              // hidden layer: stored above
            } else if (PAIRS && owner) {
              float v[16];
              ptx::tmem_ld16(tm, v);
              ptx::tmem_wait_ld();
              if (valid) p.pair_out[row] = v[0] + bl[0];
            } else if (DDIM && owner) {
              // teacher output v: x <- cx[t] x + cv[t] (v + b), then the next step's input
              float v[16];
              ptx::tmem_ld16(tm, v);
              ptx::tmem_wait_ld();
              const float cx = p.ddim_cx[t], cv = p.ddim_cv[t];
#pragma unroll
              for (int i = 0; i < DS; ++i) s[i] = fmaf(cx, s[i], cv * (v[i] + bl[i]));
              if (t + 1 < H) write_ddim_input(A, r, s, a, p.ddim_emb + (size_t)(t + 1) * 8);
            } else if (owner && l == p.n_gen - 1) {
              // generator output: s_{t+1} (FP32 here; BF16 words from here on)
              float v[32];
              ptx::tmem_ld16(tm, v);
              if (DS > 16) ptx::tmem_ld16(tm + 16, v + 16);
              ptx::tmem_wait_ld();
#pragma unroll
              for (int i = 0; i < DS; ++i) s[i] = v[i] + bl[i];
              pack_state<DS>(s_pk, s);
              if (p.reward_kind == VOILA_REWARD_GOAL) {
                if (t + 1 < H) write_gen_row<DS, DA, DW>(A, r, s_pk, tn);
                float acc = 0.0f;
#pragma unroll
                for (int i = 0; i < VOILA_MAX_GOAL; ++i)
                  if (i < p.goal_dims && i < DS) {
                    const float d = s[i] - p.goal[i];
                    acc = fmaf(d, d, acc);
                  }
                Gacc += disc * (double)(-acc);
                disc *= p.gamma;
              } else {
                write_rew_row<DS, DA>(A, r, s_pk, a_pk);
              }
            } else if (owner) {
              // reward output r_t: G += gamma^t r_t in FP64
              float v[16];
              ptx::tmem_ld16(tm, v);
              ptx::tmem_wait_ld();
              if (t + 1 < H) {
                write_gen_row<DS, DA, DW>(A, r, s_pk, tn);
                tail_actions<DA>(a_pk, tn);
              }
              Gacc += disc * (double)(v[0] + bl[0]);
              disc *= p.gamma;
            }
            ptx::tc_fence_before();
            if (arrive) {  // A columns 0..255 written, TMEM half 0 read
              ptx::fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive_cluster(ready_lo);
            }
          }
          if (ok && !lo_free) {  // one alo_free phase per layer
            if (!bounded_wait(alo_bar, nalo & 1, abort_flag, p.hdr, 33)) ok = false;
            ++nalo;
          }
          if (!ok) break;
          ptx::tc_fence_before();
          if (arrive) {  // A columns 256..511 written, TMEM half 1 read
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive_cluster(ready_hi);
          }
        }
      }
      if constexpr (PAIRS) {
      } else if constexpr (DDIM) {
        if (owner && valid && ok) {
#pragma unroll
          for (int i = 0; i < DS; i += 4)
            *reinterpret_cast<float4*>(p.ddim_y + (size_t)row * DS + i) = make_float4(s[i], s[i + 1], s[i + 2], s[i + 3]);
        }
      } else if (owner && valid && ok) {
        PL.G[row] = Gacc;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (two tiles)
    // All sixteen warps serve each tile in turn, in the order the MMA warp
    // issues them (tile 0 of a layer, then tile 1), so one tile's epilogue
    // runs while the other tile's MMAs do. Warp w reads TMEM lanes
    // 32*(w % 4) .. +31 (its rows of the tile) and a quarter of the columns
    // (slice (w - 2) / 4); the slice-0 warps hold the row state of tile 0 (s_t,
    // omega, reward, G), the slice-1 warps that of tile 1.
    const int e = warp - 2;
    const int slice = e >> 2;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const bool owner = slice < 2;
    const int og = slice & 1;  // the tile whose rows an owner holds
    uint8_t* Aown = Abuf[og];
    const uint32_t tq = (uint32_t)(32 * q) << 16;
    const uint32_t ready_remote0 = ptx::mapa_shared(ptx::smem_u32(&ready[0]), 0);  // even CTA's
    const uint32_t ready_remote1 = ptx::mapa_shared(ptx::smem_u32(&ready[1]), 0);
    uint32_t nacc[2] = {0u, 0u};
    bool ok = true;
    long long jq = 0;
    for (long long it = QUEUE ? take_item(item_full, item_empty, item_ring, jq, true, abort_flag, p.hdr)
                              : cl;
         it >= 0 && it < total_items && ok;
         it = QUEUE ? take_item(item_full, item_empty, item_ring, ++jq, true, abort_flag, p.hdr)
                    : (SERP ? static_item(++jq, cl, ncl, true) : it + ncl)) {
      const int pq = item_planner(p, it);
      const long long sp = it - (pq ? p.item_end[pq - 1] : 0);
      const TcPlanner& PL = p.pl[pq];
      const int H = PL.H;
      const long long row = sp * kSuperRows + og * (2 * kTileRows) + (long long)rank * kTileRows + r;
      const bool valid = row < PL.rows;
      const uint32_t n = valid ? (uint32_t)(row % PL.N) : 0u;
      const uint32_t k = valid ? (uint32_t)(row / PL.N) : 0u;
      const float* act_row = PL.actions + (size_t)k * H * DA;
      const uint32_t nc = n + PL.n_off, kc = k + PL.k_off;  // noise counters of the unsharded problem
      // row state of an owner, as packed BF16 words: s_t, a_t, and the tail
      // [a_{t+1}; omega_T(n, k, t + 1)] drawn ahead of the step's end
      uint32_t s_pk[DS / 2], a_pk[(DA + 1) / 2], tn[(DA + DW + 1) / 2];
      float r_pend = 0.0f;  // r_t, added to G in FP64 during the next step
      // pair mode: the next item's input rows are written (and announced) by
      // the last layer's epilogue of this item, one tile at a time, so the
      // next item's first MMA does not wait for the end of this item
      const bool first_item = it == cl;
      const bool has_next = PAIRS && it + ncl < total_items;
      const long long row_next = (it + ncl) * kSuperRows + og * (2 * kTileRows) + (long long)rank * kTileRows + r;
      int obs_m = -1, obs_a = 0;  // observation mode: this row's simulation and node
      if constexpr (PAIRS) {
        if (owner && first_item) write_pair_row(p, Aown, r, row, valid);
      } else if constexpr (OBS) {
        if (owner) {
          const int cnt = *reinterpret_cast<const volatile int*>(p.obs_count);
          if (row < cnt) {
            const int m = __ldg(p.obs_list + row);
            const int a = (m >= 0 && m < p.pair_B) ? __ldg(p.gather_node + m) : -1;
            if (a >= 0 && a < p.gather_n_nodes) {
              obs_m = m;
              obs_a = a;
            }
          }
          float s0[DS], e[2 * ((DA + DW + 1) / 2)];
#pragma unroll
          for (int i = 0; i < DS; ++i) s0[i] = obs_m >= 0 ? __ldg(p.pair_s + (size_t)obs_m * DS + i) : 0.0f;
#pragma unroll
          for (int i = 0; i < 2 * ((DA + DW + 1) / 2); ++i) e[i] = 0.0f;
#pragma unroll
          for (int i = 0; i < DA; ++i) e[i] = obs_m >= 0 ? __ldg(p.pair_a + (size_t)obs_a * DA + i) : 0.0f;
          if (obs_m >= 0) {
#pragma unroll
            for (int b = 0; b < (DW + 3) / 4; ++b) {
              const float4 z = normal4(p.key0, p.key1, (uint32_t)obs_m, 0u, p.obs_step, VOILA_STREAM_OBS_OMEGA,
                                       p.obs_planner, (uint32_t)b);
              if (4 * b + 0 < DW) e[DA + 4 * b + 0] = z.x;
              if (4 * b + 1 < DW) e[DA + 4 * b + 1] = z.y;
              if (4 * b + 2 < DW) e[DA + 4 * b + 2] = z.z;
              if (4 * b + 3 < DW) e[DA + 4 * b + 3] = z.w;
            }
          }
          pack_state<DS>(s_pk, s0);
#pragma unroll
          for (int j = 0; j < (DA + DW + 1) / 2; ++j) tn[j] = ptx::pack_bf16x2(e[2 * j], e[2 * j + 1]);
          write_gen_row<DS, DA, DW>(Aown, r, s_pk, tn);
        }
      } else if (owner) {
        float s0[DS];
#pragma unroll
        for (int i = 0; i < DS; ++i) s0[i] = valid ? __ldg(PL.particles + (size_t)n * DS + i) : 0.0f;
        pack_state<DS>(s_pk, s0);
        if constexpr (PROP)
          draw_tail<DA, DW>(tn, act_row, p.key0, p.key1, n, 0u, p.prop_step, PL.planner, VOILA_STREAM_BELIEF_OMEGA);
        else
          draw_tail<DA, DW>(tn, act_row, p.key0, p.key1, nc, kc, 0u, PL.planner);
        write_gen_row<DS, DA, DW>(Aown, r, s_pk, tn);
        tail_actions<DA>(a_pk, tn);
      }
      if (!PAIRS || first_item) {
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive_cluster(ready_remote0);
          ptx::mbar_arrive_cluster(ready_remote1);
        }
      }
      double Gacc = 0.0, disc = 1.0;
      // with a reward head the owner prepares the next step's input while it
      // waits for the other tile's generator output, so the reward output
      // only has to store it
      const bool ahead = !PAIRS && p.reward_kind == VOILA_REWARD_MLP;
      for (int t = 0; t < H && ok; ++t) {
        for (int l = 0; l < p.n_total && ok; ++l) {
          const TcLayer& L = p.layers[l];
          const float* bl = bias_s + L.bias_off;  // shared memory (L1 loads measured slower)
          // no A operand follows the final layer of the final step (pair mode:
          // unless the next item's input was written in its epilogue)
          const bool arrive = !(t == H - 1 && l == p.n_total - 1) || has_next;
          for (int g = 0; g < 2; ++g) {
            if (ahead && owner && g != og && l == p.n_gen - 1) {
              if (t > 0) {  // r_{t-1}, in step order
                Gacc += disc * (double)r_pend;
                disc *= p.gamma;
              }
              if (t + 1 < H)
                draw_tail<DA, DW>(tn, act_row + (t + 1) * DA, p.key0, p.key1, nc, kc, (uint32_t)(t + 1), PL.planner);
            }
            if (!bounded_wait(ptx::smem_u32(&accf[g]), nacc[g] & 1, abort_flag, p.hdr, 30 + g)) {
              ok = false;
              break;
            }
            ++nacc[g];
            ptx::tc_fence_after();
            uint8_t* A = Abuf[g];
            const uint32_t tm = tmem_base + (uint32_t)(g * 256) + tq;
            if (L.act >= 0 && L.fuse_out) {
              // last hidden layer before a scalar output: the output is computed here on
              // the CUDA cores (each warp's quarter of the columns, then the row owner
              // adds the four partial sums and the bias in a fixed order)
              const int per = L.Npad >> 2;
              const float* wf = fuse_s + L.fuse_off;
              const float* sl = scale_s + L.scale_off;
              uint64_t part2 = 0ull;  // (even, odd) column partial sums, both +0.0f
              if (per >= 16) {
                // 16 columns per TMEM load: the dot products hold fewer live values
                // than the hidden epilogue, and 32-column loads here cost register spills
                // that every other layer then pays for
                const int c0 = slice * (per >> 4);
                for (int c = c0; c < c0 + (per >> 4); ++c) {
                  float v[16];
                  ptx::tmem_ld16(tm + 16 * c, v);
                  ptx::tmem_wait_ld();
                  ptx::tie8(v);
                  ptx::tie8(v + 8);
                  part2 = (F8 && L.fp8) ? fuse_cols<true, 16>(v, bl, sl, c, L.act, wf, part2)
                                        : fuse_cols<false, 16>(v, bl, sl, c, L.act, wf, part2);
                }
              } else {
                float v[16];
                ptx::tmem_ld16(tm + 16 * slice, v);
                ptx::tmem_wait_ld();
                part2 = (F8 && L.fp8) ? fuse_cols<true, 16>(v, bl, sl, slice, L.act, wf, part2)
                                      : fuse_cols<false, 16>(v, bl, sl, slice, L.act, wf, part2);
              }
              float pe, po;
              ptx::f2_unpack(part2, pe, po);
              red_s[(g * 4 + slice) * 128 + r] = pe + po;
              asm volatile("bar.sync %0, 128;" ::"r"(1 + q) : "memory");  // the four warps of quadrant q
              if (owner && og == g) {
                float val = wf[L.fuse_K];
#pragma unroll
                for (int sl4 = 0; sl4 < 4; ++sl4) val += red_s[(g * 4 + sl4) * 128 + r];
                if constexpr (PAIRS) {
                  if (valid) p.pair_out[row] = val;
                  if (has_next && t == H - 1) write_pair_row(p, A, r, row_next, row_next < PL.rows);
                } else if constexpr (PROP) {
                  if (valid) p.prop_ell[row] = (double)val;
                } else if (t + 1 < H) {
                  r_pend = val;
                  write_gen_row<DS, DA, DW>(A, r, s_pk, tn);
                  tail_actions<DA>(a_pk, tn);
                } else {
                  Gacc += disc * (double)val;
                }
              }
            } else if (L.act >= 0) {
              // hidden layer: this warp's quarter of the columns, 32 per TMEM load
              const int per = L.Npad >> 2;
              if (per >= 32) {
                const int c0 = slice * (per >> 5);
                for (int c = c0; c < c0 + (per >> 5); ++c) {
                  float v[32];
                  ptx::tmem_ld32(tm + 32 * c, v);
                  ptx::tmem_wait_ld32(v);
                  if (!F8) {
                    epi_cols32<false, false>(v, bl, nullptr, c, L.act, A, r);
                  } else if (L.out_fp8) {
                    if (L.fp8) epi_cols32<true, true>(v, bl, scale_s + L.scale_off, c, L.act, A, r);
                    else epi_cols32<false, true>(v, bl, nullptr, c, L.act, A, r);
                  } else {
                    if (L.fp8) epi_cols32<true, false>(v, bl, scale_s + L.scale_off, c, L.act, A, r);
                    else epi_cols32<false, false>(v, bl, nullptr, c, L.act, A, r);
                  }
                }
              } else {
                float v[16];
                ptx::tmem_ld16(tm + 16 * slice, v);
                ptx::tmem_wait_ld();
                if (!F8) {
                  epi_cols16<false, false>(v, bl, nullptr, slice, L.act, A, r);
                } else if (L.out_fp8) {
                  if (L.fp8) epi_cols16<true, true>(v, bl, scale_s + L.scale_off, slice, L.act, A, r);
                  else epi_cols16<false, true>(v, bl, nullptr, slice, L.act, A, r);
                } else {
                  if (L.fp8) epi_cols16<true, false>(v, bl, scale_s + L.scale_off, slice, L.act, A, r);
                  else epi_cols16<false, false>(v, bl, nullptr, slice, L.act, A, r);
                }
              }
            } else if (owner && og == g) {
              if constexpr (PAIRS) {
                float v[16];
                ptx::tmem_ld16(tm, v);
                ptx::tmem_wait_ld();
                if (valid) p.pair_out[row] = v[0] + bl[0];
                if (has_next && t == H - 1) write_pair_row(p, A, r, row_next, row_next < PL.rows);
              } else if (OBS && l == p.n_gen - 1) {
                float v[32];
                ptx::tmem_ld16(tm, v);
                ptx::tmem_ld16(tm + 16, v + 16);
                ptx::tmem_wait_ld();
                if (obs_m >= 0) {
                  const int br = __ldg(p.gather_branch + obs_m);
                  if (br >= 0 && br < p.gather_C_max)
                    for (int i = 0; i < p.obs_d; ++i)
                      p.obs_out[((size_t)obs_a * p.gather_C_max + br) * p.obs_d + i] = v[i] + bl[i];
                }
              } else if (l == p.n_gen - 1) {
                // generator output: s_{t+1} (FP32 here; BF16 words from here on)
                float v[32];
                ptx::tmem_ld16(tm, v);
                if (DS > 16) ptx::tmem_ld16(tm + 16, v + 16);
                ptx::tmem_wait_ld();
                float s1[DS];
#pragma unroll
                for (int i = 0; i < DS; ++i) s1[i] = v[i] + bl[i];
                pack_state<DS>(s_pk, s1);
                if (p.reward_kind == VOILA_REWARD_GOAL) {
                  float acc = 0.0f;
#pragma unroll
                  for (int i = 0; i < VOILA_MAX_GOAL; ++i)
                    if (i < p.goal_dims && i < DS) {
                      const float d = s1[i] - p.goal[i];
                      acc = fmaf(d, d, acc);
                    }
                  Gacc += disc * (double)(-acc);
                  disc *= p.gamma;
                  if (t + 1 < H) {
                    draw_tail<DA, DW>(tn, act_row + (t + 1) * DA, p.key0, p.key1, nc, kc, (uint32_t)(t + 1),
                                      PL.planner);
                    write_gen_row<DS, DA, DW>(A, r, s_pk, tn);
                  }
                } else if constexpr (PROP) {
                  if (valid)
                    for (int i = 0; i < DS; ++i) p.prop_s[(size_t)row * DS + i] = s1[i];
                  float av[DA], ov[6];
#pragma unroll
                  for (int i = 0; i < DA; ++i) av[i] = __ldg(act_row + i);
#pragma unroll
                  for (int i = 0; i < 6; ++i) ov[i] = __ldg(p.prop_obs + i);
                  write_lik_row<DS, DA>(A, r, s_pk, av, ov);
                } else {
                  write_rew_row<DS, DA>(A, r, s_pk, a_pk);
                }
              } else {
                // reward output r_t: G += gamma^t r_t in FP64 (during the next step)
                float v[16];
                ptx::tmem_ld16(tm, v);
                ptx::tmem_wait_ld();
                const float val = v[0] + bl[0];
                if (t + 1 < H) {
                  r_pend = val;
                  write_gen_row<DS, DA, DW>(A, r, s_pk, tn);
                  tail_actions<DA>(a_pk, tn);
                } else {
                  Gacc += disc * (double)val;
                }
              }
            }
            ptx::tc_fence_before();
            if (arrive) {
              ptx::fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive_cluster(g ? ready_remote1 : ready_remote0);
            }
          }
        }
      }
      if constexpr (!PAIRS) {
        if (!OBS && !PROP && owner && valid && ok) PL.G[row] = Gacc;
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::cluster_sync();  // neither CTA leaves while the pair may still touch its memory
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc_pair(tmem_base, 512);
}

// One launch packs every layer into the [rows][128-byte] weight tensor that
// the TMA reads: chunk c of layer l is rows row0 + c * Npad + n holding
// W[n][E c .. E c + E - 1], E = 64 BF16 or 128 E4M3 values, zero padded;
// SiLU layers are scaled by 1/2 (exact); an E4M3 row n is W[n][.] / scale_n.
// Biases are copied (scaled alike) and zero padded.
struct PackTable {
  const __nv_bfloat16* W[kMaxTcLayers];
  const float* b[kMaxTcLayers];
  int N[kMaxTcLayers], K[kMaxTcLayers], Npad[kMaxTcLayers];
  int row0[kMaxTcLayers], bias_off[kMaxTcLayers], scale_off[kMaxTcLayers];
  long long elems_end[kMaxTcLayers];
  int half[kMaxTcLayers];  // 1: SiLU layer, pack W and b scaled by 1/2
  int fp8[kMaxTcLayers];
  int ldk[kMaxTcLayers];   // row stride of W[l] (its input width)
  int colmap_layer;        // layer whose packed column kg reads W column colmap[kg] (-1: none)
  short colmap[128];       // -1: zero column
  // fused scalar output layers: weights (FP32 copies) and bias at fuse_base + fuseoff
  int fuse_n, fuse_base;
  const __nv_bfloat16* fuseW[2];
  const float* fuseb[2];
  int fuseK[2], fuseoff[2];
  int n;
  uint8_t* wout;
  float* bout;   // biases, then channel scales
};

// Per-output-channel scale of every E4M3 layer: max_k |W'[n][k]| / 448 (W'
// includes the SiLU 1/2), 1 for all-zero or padded rows. One warp per row.
__global__ void scale_kernel(const __grid_constant__ PackTable t) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int base = 0;
  for (int l = 0; l < t.n; ++l) {
    if (!t.fp8[l]) continue;
    const int rowl = wg - base;
    base += t.Npad[l];
    if (rowl < 0 || rowl >= t.Npad[l]) continue;
    float m = 0.0f;
    if (rowl < t.N[l])
      for (int k = lane; k < t.K[l]; k += 32) m = fmaxf(m, fabsf(__bfloat162float(t.W[l][(size_t)rowl * t.K[l] + k])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (t.half[l]) m *= 0.5f;
    if (lane == 0) t.bout[t.scale_off[l] + rowl] = m > 0.0f ? m / 448.0f : 1.0f;
  }
}

__global__ void pack_kernel(const __grid_constant__ PackTable t) {
  const long long total = t.elems_end[t.n - 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (e >= t.elems_end[l]) ++l;
    const long long e0 = e - (l ? t.elems_end[l - 1] : 0);
    const int Npad = t.Npad[l];
    const int epr = t.fp8[l] ? 128 : 64;  // values per 128-byte row
    const int c = (int)(e0 / (Npad * epr));
    const int rem = (int)(e0 % (Npad * epr));
    const int nrow = rem / epr, kk = rem % epr;
    const int kg = epr * c + kk;
    int src = kg < t.K[l] ? kg : -1;
    if (l == t.colmap_layer) src = kg < 128 ? t.colmap[kg] : -1;
    float w = (nrow < t.N[l] && src >= 0) ? __bfloat162float(t.W[l][(size_t)nrow * t.ldk[l] + src]) : 0.0f;
    if (t.half[l]) w *= 0.5f;  // exact
    uint8_t* row = t.wout + ((size_t)t.row0[l] + (size_t)c * Npad + nrow) * 128;
    if (t.fp8[l]) {
      const __nv_fp8_e4m3 q(w / t.bout[t.scale_off[l] + nrow]);
      row[kk] = *reinterpret_cast<const uint8_t*>(&q);
    } else {
      *reinterpret_cast<__nv_bfloat16*>(row + 2 * kk) = __float2bfloat16(w);
    }
    if (c == 0 && kk == 0)
      t.bout[t.bias_off[l] + nrow] = nrow < t.N[l] ? (t.half[l] ? 0.5f : 1.0f) * t.b[l][nrow] : 0.0f;
  }
}

__global__ void fuse_pack_kernel(const __grid_constant__ PackTable t) {
  for (int f = 0; f < t.fuse_n; ++f) {
    float* dst = t.bout + t.fuse_base + t.fuseoff[f];
    for (int i = threadIdx.x; i < t.fuseK[f]; i += blockDim.x) dst[i] = __bfloat162float(t.fuseW[f][i]);
    if (threadIdx.x == 0) dst[t.fuseK[f]] = t.fuseb[f][0];
  }
}

struct Plan {
  TcParams p;
  PackTable pack;
  int total_rows;
  size_t wbytes, bias_bytes, total;
  bool ok;
  bool wide;  // some layer is wider than 256: the wide kernel
};

int round_up(int v, int m) { return (v + m - 1) / m * m; }

// ddim: g is the DDIM teacher [s (8); a (2); x (8); e (64)] -> ... -> 8; its
// first layer is packed with 96 input columns in the order write_ddim_input
// writes them.
// one_tile: the one-tile shape (the wide kernel: one 128-row tile per CTA and
// work item, the scalar output layers as MMAs) for MLPs of any width.
Plan make_plan(const voila_mlp* g, const voila_reward* R, bool ddim = false, bool one_tile = false) {
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  pl.ok = false;
  pl.pack.colmap_layer = -1;
  pl.wide = one_tile;
  const voila_mlp* mlps[2] = {g, R && R->kind == VOILA_REWARD_MLP ? R->mlp : nullptr};
  int nl = 0, boff = 0, rows = 0, foff = 0;
  long long elems = 0;
  bool any_wide = one_tile;  // a layer wider than 256: the wide kernel, which has no fused outputs
  for (int m = 0; m < 2; ++m)
    if (mlps[m])
      for (int l = 0; l <= mlps[m]->n_layers; ++l) any_wide = any_wide || mlps[m]->dims[l] > 256;
  for (int m = 0; m < 2; ++m) {
    const voila_mlp* M = mlps[m];
    if (!M) continue;
    if ((M->prec != VOILA_BF16 && M->prec != VOILA_FP8E4M3) || M->n_layers < 2) return pl;
    if (M->prec == VOILA_FP8E4M3 && M->act != VOILA_ACT_SILU) return pl;  // the E4M3 epilogues are SiLU's
    // a scalar output layer is computed in the previous layer's epilogue
    const bool fuse = !ddim && !any_wide && M->dims[M->n_layers] == 1;
    for (int l = 0; l < M->n_layers; ++l) {
      if (fuse && l == M->n_layers - 1) {
        TcLayer& P = pl.p.layers[nl - 1];
        P.fuse_out = 1;
        P.fuse_off = foff;
        P.fuse_K = M->dims[l];
        PackTable& T = pl.pack;
        T.fuseW[T.fuse_n] = (const __nv_bfloat16*)M->W[l];
        T.fuseb[T.fuse_n] = M->b[l];
        T.fuseK[T.fuse_n] = M->dims[l];
        T.fuseoff[T.fuse_n] = foff;
        ++T.fuse_n;
        foff += round_up(M->dims[l] + 1, 4);
        continue;
      }
      if (nl >= kMaxTcLayers) return pl;
      const int K = (ddim && l == 0) ? 96 : M->dims[l], N = M->dims[l + 1];
      const bool last = l == M->n_layers - 1;
      if (l == 0 && K > (ddim ? 96 : 64)) return pl;
      if (l > 0 && (K % 64 != 0 || K > 512)) return pl;
      if (!last && (N % 64 != 0 || N > 512 || (N > 256 && N != 512))) return pl;
      if (last && N > 32) return pl;
      if (K > 256 || N > 256) pl.wide = true;
      TcLayer& L = pl.p.layers[nl];
      // FP8 form: hidden x hidden layers in E4M3, first and last layers in BF16
      L.fp8 = (M->prec == VOILA_FP8E4M3 && l > 0 && !last) ? 1 : 0;
      L.out_fp8 = (M->prec == VOILA_FP8E4M3 && l + 1 < M->n_layers - 1) ? 1 : 0;
      L.Kp = round_up(K, L.fp8 ? 32 : 16);
      L.ksteps = L.fp8 ? L.Kp / 32 : L.Kp / 16;
      L.Npad = last ? 32 : N;
      L.nslabs = (L.Kp + (L.fp8 ? 127 : 63)) / (L.fp8 ? 128 : 64);
      L.slab_bytes = ((L.Npad > 256 ? 256 : L.Npad) / 2) * 128;
      L.spc = kSlotBytes / L.slab_bytes;
      if (L.spc > 4) L.spc = 4;  // at most 16 K steps per chunk
      if (L.spc > L.nslabs) L.spc = L.nslabs;
      L.nchunks = (L.nslabs + L.spc - 1) / L.spc;
      L.bias_off = boff;
      L.act = last ? -1 : M->act;
      const int ncols = L.Npad > 256 ? 256 : L.Npad;  // N of one MMA
      L.ngroups = L.Npad > 256 ? 2 : 1;
      L.box_rows = ncols / 2;
      L.idesc = L.fp8 ? ptx::idesc_e4m3(256, ncols) : ptx::idesc_bf16(256, ncols);
      L.row0 = rows;
      PackTable& T = pl.pack;
      T.W[nl] = (const __nv_bfloat16*)M->W[l];
      T.b[nl] = M->b[l];
      T.N[nl] = N;
      T.K[nl] = K;
      T.ldk[nl] = M->dims[l];
      T.Npad[nl] = L.Npad;
      T.row0[nl] = rows;
      T.bias_off[nl] = boff;
      T.half[nl] = (!last && M->act == VOILA_ACT_SILU) ? 1 : 0;
      T.fp8[nl] = L.fp8;
      elems += (long long)L.nslabs * L.Npad * (L.fp8 ? 128 : 64);
      T.elems_end[nl] = elems;
      rows += L.nslabs * L.Npad;
      boff += L.Npad;  // multiple of 32
      ++nl;
    }
    if (m == 0) pl.p.n_gen = nl;
  }
  if (ddim) {  // packed column -> teacher column: x 10..17, s 0..7, a 8..9, zeros, e 18..81
    pl.pack.colmap_layer = 0;
    for (int c = 0; c < 128; ++c)
      pl.pack.colmap[c] = c < 8 ? (short)(10 + c) : c < 18 ? (short)(c - 8)
                        : (c >= 32 && c < 96) ? (short)(c - 14) : (short)-1;
  }
  pl.p.n_total = nl;
  // Wide kernel: a 512-wide layer with K <= 256 reads one A half, so its
  // epilogue can write its first output half into the other A half at once,
  // and the next layer takes its K < 256 from there (rot = 1); a layer whose
  // input the row owner writes (after an output layer, or the first) has
  // rot = 0. Used for the DDIM teacher (sampler 2.96 -> 2.75 ms at 65,536
  // samples); the sweep generator measured 1-3 % slower with it and keeps
  // rot = 0.
  for (int l = 0, r = 0; l < nl; ++l) {
    TcLayer& L = pl.p.layers[l];
    L.rot = r;
    const bool flip = ddim && pl.wide && L.ngroups == 2 && L.Kp <= 256;
    r = L.act >= 0 ? (r ^ (flip ? 1 : 0)) : 0;
  }
  // the two-tile kernel keeps a layer's chunks in the ring for both tiles
  if (!pl.wide)
    for (int l = 0; l < nl; ++l)
      if (pl.p.layers[l].nchunks >= kStages) return pl;
  pl.pack.n = nl;
  pl.p.bias_total = boff;
  int soff = 0;  // channel scales follow the biases in the same vector
  for (int l = 0; l < nl; ++l) {
    pl.p.layers[l].scale_off = soff;
    pl.pack.scale_off[l] = boff + soff;
    if (pl.p.layers[l].fp8) soff += pl.p.layers[l].Npad;
  }
  pl.p.scale_total = soff;
  pl.p.fuse_total = foff;
  pl.pack.fuse_base = boff + soff;
  pl.total_rows = rows;
  pl.wbytes = (size_t)rows * 128;
  pl.bias_bytes = (size_t)(boff + soff + foff) * sizeof(float);
  pl.total = (pl.wbytes + 1023) / 1024 * 1024 + (pl.bias_bytes + 255) / 256 * 256;
  pl.ok = true;
  return pl;
}

size_t tc_smem_bytes(int vec_floats) {
  // barriers (weight ring, accumulators, ready, drain, item ring), item slots, A-free barrier, TMEM
  // address, abort flag
  return 1024 + 2 * kABytes + kStages * kSlotBytes + (size_t)vec_floats * 4 + (2 * kStages + 6 + 3 * kItemRing) * 8 +
         16;
}

// Launches one persistent CTA pair per co-resident cluster slot (at most
// `max_clusters`, never more than there are super-pairs).
template <int DS, int DA, int DW, bool F8, bool WIDE, int MODE = kModeRollout, bool QUEUE = false>
cudaError_t launch_tc(const TcParams& p, size_t smem, long long max_clusters, cudaStream_t s) {
  auto k = rollout_tc_kernel<DS, DA, DW, F8, WIDE, MODE, QUEUE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(2 * max_clusters));
  cfg.blockDim = dim3(kTcThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 2;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  // co-resident cluster slots: queried once per device and instantiation
  static int cached[64] = {};  // one table per instantiation
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int active = (dev >= 0 && dev < 64) ? cached[dev] : 0;
  if (active == 0) {
    e = cudaOccupancyMaxActiveClusters(&active, k, &cfg);
    if (e != cudaSuccess) return e;
    if (active < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) cached[dev] = active;
  }
  long long ncl = max_clusters < active ? max_clusters : active;
  k<<<(unsigned)(2 * ncl), kTcThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point, so the
// library does not link libcuda directly (it loads on hosts without a driver).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

size_t tc_rollout_scratch_bytes(const voila_mlp* g_T, const voila_reward* R) {
  // the larger of the two tile shapes' packed weights (the one-tile shape packs
  // the scalar output layers as MMA operands)
  Plan pl = make_plan(g_T, R);
  Plan p1 = make_plan(g_T, R, false, true);
  size_t b = pl.ok ? pl.total : 0;
  if (p1.ok && p1.total > b) b = p1.total;
  return b;
}

voila_status tc_rollout_batched(const voila_mlp* g_T, const voila_reward* R, const TcProblem* probs, int P,
                                int d_s, int d_a, int d_omega, double gamma, uint32_t key0, uint32_t key1,
                                int order, int max_clusters, int shape, WsHeader* hdr, void* scratch,
                                cudaStream_t s) {
  const bool queue = (shape & kShapeQueue) != 0;
  const bool one_tile = (shape & kShapeOneTile) != 0;
  Plan pl = make_plan(g_T, R, false, one_tile);
  if (!pl.ok) return VOILA_ERR_UNSUPPORTED;
  if (P < 1 || P > kMaxPlanners) return VOILA_ERR_ARG;
  const bool dims_a = d_s == 8 && d_a == 2 && d_omega == 8;
  const bool dims_b = d_s == 12 && d_a == 3 && d_omega == 16;
  if (!dims_a && !dims_b) return VOILA_ERR_UNSUPPORTED;
  const bool f8 = g_T->prec == VOILA_FP8E4M3;
  // the wide kernel is built for the sweep dimensions, and for the mid-size ones in BF16
  if (pl.wide && !dims_b && (!dims_a || f8)) return VOILA_ERR_UNSUPPORTED;
  if ((uintptr_t)scratch % 16) return VOILA_ERR_WORKSPACE;  // TMA global base alignment
  TcParams& p = pl.p;
  // work table: planners with rows and steps, optionally longest horizon first
  int idx[kMaxPlanners];
  int nq = 0;
  for (int i = 0; i < P; ++i) {
    const TcProblem& q = probs[i];
    if ((long long)q.N * q.K == 0) continue;
    if (q.H == 0) {  // no steps: zero returns
      if (cudaMemsetAsync(q.G, 0, (size_t)q.N * q.K * sizeof(double), s) != cudaSuccess) return VOILA_ERR_CUDA;
      continue;
    }
    idx[nq++] = i;
  }
  if (nq == 0) return VOILA_OK;
  if (order == 1)
    for (int i = 1; i < nq; ++i)  // stable insertion sort by descending H
      for (int j = i; j > 0 && probs[idx[j]].H > probs[idx[j - 1]].H; --j) {
        const int t = idx[j];
        idx[j] = idx[j - 1];
        idx[j - 1] = t;
      }
  long long items = 0;
  for (int j = 0; j < nq; ++j) {
    const TcProblem& q = probs[idx[j]];
    TcPlanner& t = p.pl[j];
    t.particles = q.particles;
    t.actions = q.actions;
    t.G = q.G;
    t.rows = (long long)q.N * q.K;
    t.N = q.N;
    t.H = q.H;
    t.planner = q.planner;
    t.n_off = q.n_off;
    t.k_off = q.k_off;
    const long long item_rows = pl.wide ? 2 * kTileRows : kSuperRows;
    items += (t.rows + item_rows - 1) / item_rows;
    p.item_end[j] = items;
  }
  p.P = nq;
  p.total_items = items;

  uint8_t* wst = (uint8_t*)scratch;
  float* bias_all = (float*)((uint8_t*)scratch + (pl.wbytes + 1023) / 1024 * 1024);
  pl.pack.wout = wst;
  pl.pack.bout = bias_all;
  {
    const long long total = pl.pack.elems_end[pl.pack.n - 1];
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (p.scale_total > 0) {
      int srows = 0;
      for (int l = 0; l < pl.pack.n; ++l)
        if (pl.pack.fp8[l]) srows += pl.pack.Npad[l];
      scale_kernel<<<(srows * 32 + 255) / 256, 256, 0, s>>>(pl.pack);
    }
    pack_kernel<<<(int)blocks, 256, 0, s>>>(pl.pack);
    if (pl.pack.fuse_n > 0) fuse_pack_kernel<<<1, 256, 0, s>>>(pl.pack);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  // one tensor map per layer over the [rows][64] BF16 weight tensor
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return VOILA_ERR_CUDA;
  for (int l = 0; l < p.n_total; ++l) {
    const cuuint64_t gdim[2] = {128, (cuuint64_t)pl.total_rows};  // bytes
    const cuuint64_t gstride[1] = {128};
    const cuuint32_t box[2] = {128, (cuuint32_t)p.layers[l].box_rows};
    const cuuint32_t estride[2] = {1, 1};
    if (encode(&p.tmap[l], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)wst, gdim, gstride, box,
                               estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return VOILA_ERR_CUDA;
  }
  p.bias_all = bias_all;
  p.gamma = gamma;
  p.key0 = key0;
  p.key1 = key1;
  p.reward_kind = R->kind;
  p.goal_dims = R->goal_dims;
  for (int i = 0; i < VOILA_MAX_GOAL; ++i) p.goal[i] = R->goal[i];
  p.hdr = hdr;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long nclusters = items < nsm / 2 ? items : nsm / 2;
  if (max_clusters > 0 && nclusters > max_clusters) nclusters = max_clusters;
  const size_t smem = tc_smem_bytes(p.bias_total + p.scale_total + p.fuse_total + (p.fuse_total ? 1024 : 0));
  if (queue) {  // the work-item counter, in the workspace header, starts at zero
    p.queue = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(hdr) + kQueueCounterOffset);
    if (cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return VOILA_ERR_CUDA;
  }
  constexpr int R0 = kModeRollout;
  cudaError_t e;
  if (dims_a && !pl.wide)
    e = f8 ? (queue ? launch_tc<8, 2, 8, true, false, R0, true>(p, smem, nclusters, s)
                    : launch_tc<8, 2, 8, true, false>(p, smem, nclusters, s))
           : (queue ? launch_tc<8, 2, 8, false, false, R0, true>(p, smem, nclusters, s)
                    : launch_tc<8, 2, 8, false, false>(p, smem, nclusters, s));
  else if (dims_a)
    e = queue ? launch_tc<8, 2, 8, false, true, R0, true>(p, smem, nclusters, s)
              : launch_tc<8, 2, 8, false, true>(p, smem, nclusters, s);
  else if (!pl.wide)
    e = f8 ? (queue ? launch_tc<12, 3, 16, true, false, R0, true>(p, smem, nclusters, s)
                    : launch_tc<12, 3, 16, true, false>(p, smem, nclusters, s))
           : (queue ? launch_tc<12, 3, 16, false, false, R0, true>(p, smem, nclusters, s)
                    : launch_tc<12, 3, 16, false, false>(p, smem, nclusters, s));
  else
    e = f8 ? (queue ? launch_tc<12, 3, 16, true, true, R0, true>(p, smem, nclusters, s)
                    : launch_tc<12, 3, 16, true, true>(p, smem, nclusters, s))
           : (queue ? launch_tc<12, 3, 16, false, true, R0, true>(p, smem, nclusters, s)
                    : launch_tc<12, 3, 16, false, true>(p, smem, nclusters, s));
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

namespace {

// Step embeddings of the sampler in launch order (row t is diffusion step
// T-1-t): [sin(tau f_i), cos(tau f_i)], i < 32, as BF16.
struct EmbFreq {
  float f[32];
};

__global__ void ddim_emb_kernel(EmbFreq fr, int T, __nv_bfloat16* out) {
  const int t = blockIdx.x, i = threadIdx.x;
  const float tau = (float)(T - 1 - t);
  const float a = tau * fr.f[i & 31];
  out[t * 64 + i] = __float2bfloat16(i < 32 ? sinf(a) : cosf(a));
}

}  // namespace

bool tc_ddim_supported(const voila_mlp* teacher, int d_s, int d_a, int d_x, int emb_dim) {
  if (!teacher || teacher->prec != VOILA_BF16 || d_s != 8 || d_a != 2 || d_x != 8 || emb_dim != 64) return false;
  if (teacher->dims[0] != 82) return false;
  for (int l = 1; l < teacher->n_layers; ++l)
    if (teacher->dims[l] != 512) return false;
  return make_plan(teacher, nullptr, true).ok;
}

size_t tc_ddim_scratch_bytes(const voila_mlp* teacher, int T) {
  Plan pl = make_plan(teacher, nullptr, true);
  if (!pl.ok) return 0;
  return pl.total + ((size_t)T * 128 + 1023) / 1024 * 1024;
}

voila_status tc_ddim_sample(const voila_mlp* teacher, const float* S, const float* A, const float* omega, int B,
                            int T, const double* cx, const double* cv, const double* freq, float* Y, WsHeader* hdr,
                            void* scratch, cudaStream_t s) {
  Plan pl = make_plan(teacher, nullptr, true);
  if (!pl.ok || !pl.wide) return VOILA_ERR_UNSUPPORTED;
  if (T < 1 || T > 64) return VOILA_ERR_ARG;
  if ((uintptr_t)scratch % 1024) return VOILA_ERR_WORKSPACE;
  TcParams& p = pl.p;
  TcPlanner& q = p.pl[0];
  q.particles = omega;
  q.actions = omega;  // unused by the sampler
  q.G = nullptr;
  q.rows = B;
  q.N = B;
  q.H = T;
  q.planner = 0;
  p.P = 1;
  p.total_items = (B + 2 * kTileRows - 1) / (2 * kTileRows);
  p.item_end[0] = p.total_items;
  uint8_t* wst = (uint8_t*)scratch;
  float* bias_all = (float*)(wst + (pl.wbytes + 1023) / 1024 * 1024);
  __nv_bfloat16* emb = (__nv_bfloat16*)(wst + pl.total);
  pl.pack.wout = wst;
  pl.pack.bout = bias_all;
  {
    const long long total = pl.pack.elems_end[pl.pack.n - 1];
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    pack_kernel<<<(int)blocks, 256, 0, s>>>(pl.pack);
    if (pl.pack.fuse_n > 0) fuse_pack_kernel<<<1, 256, 0, s>>>(pl.pack);
    EmbFreq fr;
    for (int i = 0; i < 32; ++i) fr.f[i] = (float)freq[i];
    ddim_emb_kernel<<<T, 64, 0, s>>>(fr, T, emb);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return VOILA_ERR_CUDA;
  for (int l = 0; l < p.n_total; ++l) {
    const cuuint64_t gdim[2] = {128, (cuuint64_t)pl.total_rows};  // bytes
    const cuuint64_t gstride[1] = {128};
    const cuuint32_t box[2] = {128, (cuuint32_t)p.layers[l].box_rows};
    const cuuint32_t estride[2] = {1, 1};
    if (encode(&p.tmap[l], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)wst, gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return VOILA_ERR_CUDA;
  }
  p.bias_all = bias_all;
  p.reward_kind = VOILA_REWARD_GOAL;
  p.goal_dims = 0;
  p.hdr = hdr;
  p.ddim_s = S;
  p.ddim_a = A;
  p.ddim_emb = reinterpret_cast<const uint4*>(emb);
  p.ddim_y = Y;
  for (int t = 0; t < T; ++t) {
    p.ddim_cx[t] = (float)cx[t];
    p.ddim_cv[t] = (float)cv[t];
  }
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nclusters = p.total_items < nsm / 2 ? p.total_items : nsm / 2;
  const size_t smem = tc_smem_bytes(p.bias_total + p.scale_total + p.fuse_total + (p.fuse_total ? 1024 : 0));
  const cudaError_t e = launch_tc<8, 10, 0, false, true, kModeDdim>(p, smem, nclusters, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

bool tc_pairs_supported(const voila_mlp* ell, int d_s, int d_a, int d_o) {
  if (!ell || ell->prec != VOILA_BF16 || d_s != 8 || d_a != 2 || d_o != 6) return false;
  if (ell->dims[0] != 16 || ell->dims[ell->n_layers] != 1) return false;
  Plan pl = make_plan(ell, nullptr);
  return pl.ok && !pl.wide;
}

size_t tc_pairs_scratch_bytes(const voila_mlp* ell) {
  Plan pl = make_plan(ell, nullptr);
  return pl.ok ? pl.total : 0;
}

voila_status tc_likelihood_pairs(const voila_mlp* ell, const float* S, const float* A, const float* Ob, long long B,
                                 float* out, WsHeader* hdr, void* scratch, cudaStream_t s) {
  return tc_likelihood_rows(ell, S, A, Ob, B, nullptr, nullptr, 0, 0, out, hdr, scratch, s);
}

voila_status tc_likelihood_rows(const voila_mlp* ell, const float* S, const float* A, const float* Ob, long long B,
                                const int32_t* node, const int32_t* branch, int n_nodes, int C_max, float* out,
                                WsHeader* hdr, void* scratch, cudaStream_t s) {
  Plan pl = make_plan(ell, nullptr);
  if (!pl.ok || pl.wide) return VOILA_ERR_UNSUPPORTED;
  if ((uintptr_t)scratch % 1024) return VOILA_ERR_WORKSPACE;
  TcParams& p = pl.p;
  TcPlanner& q = p.pl[0];
  q.particles = S;  // unused by the pair rows
  q.actions = A;
  q.G = nullptr;
  q.rows = node ? B : B * B;
  q.N = 1;
  q.H = 1;
  q.planner = 0;
  p.P = 1;
  p.total_items = (q.rows + kSuperRows - 1) / kSuperRows;
  p.item_end[0] = p.total_items;
  uint8_t* wst = (uint8_t*)scratch;
  float* bias_all = (float*)(wst + (pl.wbytes + 1023) / 1024 * 1024);
  pl.pack.wout = wst;
  pl.pack.bout = bias_all;
  {
    const long long total = pl.pack.elems_end[pl.pack.n - 1];
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    pack_kernel<<<(int)blocks, 256, 0, s>>>(pl.pack);
    if (pl.pack.fuse_n > 0) fuse_pack_kernel<<<1, 256, 0, s>>>(pl.pack);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return VOILA_ERR_CUDA;
  for (int l = 0; l < p.n_total; ++l) {
    const cuuint64_t gdim[2] = {128, (cuuint64_t)pl.total_rows};  // bytes
    const cuuint64_t gstride[1] = {128};
    const cuuint32_t box[2] = {128, (cuuint32_t)p.layers[l].box_rows};
    const cuuint32_t estride[2] = {1, 1};
    if (encode(&p.tmap[l], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)wst, gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return VOILA_ERR_CUDA;
  }
  p.bias_all = bias_all;
  p.reward_kind = VOILA_REWARD_GOAL;
  p.goal_dims = 0;
  p.hdr = hdr;
  p.pair_s = S;
  p.pair_a = A;
  p.pair_o = Ob;
  p.pair_B = B;
  p.pair_out = out;
  p.gather_node = node;
  p.gather_branch = branch;
  p.gather_n_nodes = n_nodes;
  p.gather_C_max = C_max;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nclusters = p.total_items < nsm / 2 ? p.total_items : nsm / 2;
  const size_t smem = tc_smem_bytes(p.bias_total + p.scale_total + p.fuse_total + (p.fuse_total ? 1024 : 0));
  const cudaError_t e = launch_tc<8, 2, 6, false, false, kModePairs>(p, smem, nclusters, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

bool tc_observe_supported(const voila_mlp* g_Z, int d_s, int d_a, int d_omega, int d_o) {
  if (!g_Z || g_Z->prec != VOILA_BF16 || d_s != 8 || d_a != 2 || d_omega != 8 || d_o < 1 || d_o > 32) return false;
  if (g_Z->dims[0] != d_s + d_a + d_omega || g_Z->dims[g_Z->n_layers] != d_o) return false;
  Plan pl = make_plan(g_Z, nullptr);
  return pl.ok && !pl.wide && pl.p.n_total == pl.p.n_gen;
}

size_t tc_observe_scratch_bytes(const voila_mlp* g_Z) {
  Plan pl = make_plan(g_Z, nullptr);
  return pl.ok ? pl.total : 0;
}

voila_status tc_observe_rows(const voila_mlp* g_Z, const float* S, const float* act, const int32_t* list,
                             const int32_t* count, long long M, const int32_t* node, const int32_t* branch,
                             int n_nodes, int C_max, float* obs, int d_o, uint32_t key0, uint32_t key1,
                             uint32_t step, uint32_t planner, WsHeader* hdr, void* scratch, cudaStream_t s) {
  Plan pl = make_plan(g_Z, nullptr);
  if (!pl.ok || pl.wide || pl.p.n_total != pl.p.n_gen) return VOILA_ERR_UNSUPPORTED;
  if ((uintptr_t)scratch % 1024) return VOILA_ERR_WORKSPACE;
  TcParams& p = pl.p;
  TcPlanner& q = p.pl[0];
  q.particles = S;
  q.actions = act;
  q.G = nullptr;
  q.rows = M;  // at most M listed rows; the kernel reads the count
  q.N = 1;
  q.H = 1;
  q.planner = planner;
  p.P = 1;
  p.total_items = (M + kSuperRows - 1) / kSuperRows;
  p.item_end[0] = p.total_items;
  if (p.total_items == 0) return VOILA_OK;
  uint8_t* wst = (uint8_t*)scratch;
  float* bias_all = (float*)(wst + (pl.wbytes + 1023) / 1024 * 1024);
  pl.pack.wout = wst;
  pl.pack.bout = bias_all;
  {
    const long long total = pl.pack.elems_end[pl.pack.n - 1];
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    pack_kernel<<<(int)blocks, 256, 0, s>>>(pl.pack);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return VOILA_ERR_CUDA;
  for (int l = 0; l < p.n_total; ++l) {
    const cuuint64_t gdim[2] = {128, (cuuint64_t)pl.total_rows};  // bytes
    const cuuint64_t gstride[1] = {128};
    const cuuint32_t box[2] = {128, (cuuint32_t)p.layers[l].box_rows};
    const cuuint32_t estride[2] = {1, 1};
    if (encode(&p.tmap[l], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)wst, gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return VOILA_ERR_CUDA;
  }
  p.bias_all = bias_all;
  p.reward_kind = VOILA_REWARD_GOAL;
  p.goal_dims = 0;
  p.key0 = key0;
  p.key1 = key1;
  p.hdr = hdr;
  p.pair_s = S;
  p.pair_a = act;
  p.pair_B = M;
  p.gather_node = node;
  p.gather_branch = branch;
  p.gather_n_nodes = n_nodes;
  p.gather_C_max = C_max;
  p.obs_list = list;
  p.obs_count = count;
  p.obs_out = obs;
  p.obs_d = d_o;
  p.obs_step = step;
  p.obs_planner = planner;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nclusters = p.total_items < nsm / 2 ? p.total_items : nsm / 2;
  const size_t smem = tc_smem_bytes(p.bias_total + p.scale_total + p.fuse_total + (p.fuse_total ? 1024 : 0));
  const cudaError_t e = launch_tc<8, 2, 8, false, false, kModeObserve>(p, smem, nclusters, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

bool tc_propose_supported(const voila_mlp* g_T, const voila_mlp* ell, int d_s, int d_a, int d_omega, int d_o) {
  if (!g_T || !ell) return false;
  if ((g_T->prec != VOILA_BF16 && g_T->prec != VOILA_FP8E4M3) || (ell->prec != VOILA_BF16 && ell->prec != VOILA_FP8E4M3))
    return false;
  if (d_s != 8 || d_a != 2 || d_omega != 8 || d_o != 6) return false;
  if (g_T->dims[0] != 18 || g_T->dims[g_T->n_layers] != 8 || ell->dims[0] != 16 || ell->dims[ell->n_layers] != 1)
    return false;
  voila_reward R;
  memset(&R, 0, sizeof(R));
  R.kind = VOILA_REWARD_MLP;
  R.mlp = ell;
  Plan pl = make_plan(g_T, &R);
  return pl.ok && !pl.wide && pl.p.layers[pl.p.n_total - 1].fuse_out;
}

size_t tc_propose_scratch_bytes(const voila_mlp* g_T, const voila_mlp* ell) {
  voila_reward R;
  memset(&R, 0, sizeof(R));
  R.kind = VOILA_REWARD_MLP;
  R.mlp = ell;
  Plan pl = make_plan(g_T, &R);
  return pl.ok ? pl.total : 0;
}

voila_status tc_belief_propose(const voila_mlp* g_T, const voila_mlp* ell, const float* particles, const float* action,
                               const float* obs, long long N, uint32_t key0, uint32_t key1, uint32_t step,
                               uint32_t planner, float* s_prop, double* ell_out, WsHeader* hdr, void* scratch,
                               cudaStream_t s) {
  voila_reward R;
  memset(&R, 0, sizeof(R));
  R.kind = VOILA_REWARD_MLP;
  R.mlp = ell;
  Plan pl = make_plan(g_T, &R);
  if (!pl.ok || pl.wide) return VOILA_ERR_UNSUPPORTED;
  if ((uintptr_t)scratch % 1024) return VOILA_ERR_WORKSPACE;
  if (N <= 0) return VOILA_OK;
  TcParams& p = pl.p;
  TcPlanner& q = p.pl[0];
  q.particles = particles;
  q.actions = action;  // one action for every row (sequence index 0)
  q.G = nullptr;
  q.rows = N;
  q.N = (int)N;
  q.H = 1;
  q.planner = planner;
  p.P = 1;
  p.total_items = (N + kSuperRows - 1) / kSuperRows;
  p.item_end[0] = p.total_items;
  uint8_t* wst = (uint8_t*)scratch;
  float* bias_all = (float*)(wst + (pl.wbytes + 1023) / 1024 * 1024);
  pl.pack.wout = wst;
  pl.pack.bout = bias_all;
  {
    const long long total = pl.pack.elems_end[pl.pack.n - 1];
    long long blocks = (total + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    if (p.scale_total > 0) {  // E4M3 hidden layers: per-channel scales first
      int srows = 0;
      for (int l = 0; l < pl.pack.n; ++l)
        if (pl.pack.fp8[l]) srows += pl.pack.Npad[l];
      scale_kernel<<<(srows * 32 + 255) / 256, 256, 0, s>>>(pl.pack);
    }
    pack_kernel<<<(int)blocks, 256, 0, s>>>(pl.pack);
    if (pl.pack.fuse_n > 0) fuse_pack_kernel<<<1, 256, 0, s>>>(pl.pack);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return VOILA_ERR_CUDA;
  for (int l = 0; l < p.n_total; ++l) {
    const cuuint64_t gdim[2] = {128, (cuuint64_t)pl.total_rows};  // bytes
    const cuuint64_t gstride[1] = {128};
    const cuuint32_t box[2] = {128, (cuuint32_t)p.layers[l].box_rows};
    const cuuint32_t estride[2] = {1, 1};
    if (encode(&p.tmap[l], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)wst, gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return VOILA_ERR_CUDA;
  }
  p.bias_all = bias_all;
  p.reward_kind = VOILA_REWARD_MLP;
  p.goal_dims = 0;
  p.gamma = 1.0;
  p.key0 = key0;
  p.key1 = key1;
  p.hdr = hdr;
  p.prop_obs = obs;
  p.prop_s = s_prop;
  p.prop_ell = ell_out;
  p.prop_step = step;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long nclusters = p.total_items < nsm / 2 ? p.total_items : nsm / 2;
  const size_t smem = tc_smem_bytes(p.bias_total + p.scale_total + p.fuse_total + (p.fuse_total ? 1024 : 0));
  const cudaError_t e = p.scale_total > 0 ? launch_tc<8, 2, 8, true, false, kModePropose>(p, smem, nclusters, s)
                                          : launch_tc<8, 2, 8, false, false, kModePropose>(p, smem, nclusters, s);
  return e == cudaSuccess ? VOILA_OK : VOILA_ERR_CUDA;
}

voila_status tc_rollout(const voila_mlp* g_T, const voila_reward* R, const RolloutArgs& a,
                        WsHeader* hdr, void* scratch, cudaStream_t s) {
  TcProblem q;
  q.particles = a.particles;
  q.actions = a.actions;
  q.G = a.G;
  q.N = a.N;
  q.K = a.K;
  q.H = a.H;
  q.planner = a.planner;
  q.n_off = a.n_off;
  q.k_off = a.k_off;
  return tc_rollout_batched(g_T, R, &q, 1, a.d_s, a.d_a, a.d_omega, a.gamma, a.key0, a.key1, 0, 0, 0, hdr, scratch,
                            s);
}

namespace {

// Self-test of the bounded waits: one thread waits, through the same
// bounded_wait the tensor-core kernels use, on an mbarrier that nothing
// arrives on; when `limit` SM cycles have passed it records VOILA_ERR_TIMEOUT
// (site 99) in the status word and the kernel returns.
__global__ void wait_timeout_selftest_kernel(WsHeader* hdr, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    ptx::mbar_init(ptx::smem_u32(&bar), 1);
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) bounded_wait(ptx::smem_u32(&bar), 0u, &abort_flag, hdr, 99, limit);
}

}  // namespace

cudaError_t launch_wait_timeout_selftest(WsHeader* hdr, long long limit, cudaStream_t s) {
  wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(hdr, limit);
  return cudaGetLastError();
}

}  // namespace voila

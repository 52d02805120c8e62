// Vectorised progressive widening of observation branches (Sec. 4.3).
//
// A batch of M simulations, each with the action node it reached and its
// successor state s', is processed in five phases, all on the GPU:
//   1. group by action node: stable radix sort of the 64-bit keys
//      node << 32 | m on the node (each node's simulations keep batch order);
//   2. widening decisions: the r-th simulation of a node group widens when
//      C < C_max and C < k_o (N + r + 1)^alpha_o (FP64), creating branch C;
//      otherwise it joins branch floor(u C), u the 24-bit Philox uniform of
//      counter (m, step, 0, stream 6); N and C are updated. One warp per node
//      finds all of its widenings at once (the rule is monotone in N), one
//      thread per simulation then takes its branch;
//   3. the observation sampler f_Z (Eq. 5) fills the new branches:
//      o = f_Z([s'; a; omega_Z]), omega_Z at counter (m, 0, step, stream 3);
//   4. the likelihood l(s', a, o_branch) of every simulation;
//   5. group by (node, branch) (a second stable radix sort, keys node << 40 |
//      branch << 24 | m) and, one warp per group, the SIR step: log-sum-exp normalisation
//      of l / lambda, 2^-52 quantisation, exact prefix sum, systematic
//      resampling with u0 from counter (node, branch, step, stream 2 block 1).
#include <math.h>
#include <string.h>

#include "../../include/voila.h"
#include "trace.h"
#include "common.cuh"
#include "kernels.h"
#include "simt_mlp.cuh"
#include "tc.h"

namespace voila {
namespace {

__global__ void pw_keys_node_kernel(const int32_t* __restrict__ node, int M, int n_pad, int n_nodes,
                                    unsigned long long* __restrict__ keys, WsHeader* hdr) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
    unsigned long long k = ~0ull;
    if (i < M) {
      const int a = node[i];
      if (a < 0 || a >= n_nodes) {
        set_status(hdr, VOILA_ERR_ARG, 60);
        k = 0xffffffffull << 32 | (unsigned)i;  // sorts after every valid node; skipped later
      } else {
        k = (unsigned long long)a << 32 | (unsigned)i;
      }
    }
    keys[i] = k;
  }
}

__global__ void pw_keys_branch_kernel(const unsigned long long* __restrict__ keys_node, const int32_t* __restrict__ branch,
                                      int M, int n_pad, unsigned long long* __restrict__ keys) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pad; p += gridDim.x * blockDim.x) {
    unsigned long long k = ~0ull;
    if (p < M) {
      const unsigned long long kn = keys_node[p];
      const unsigned a = (unsigned)(kn >> 32), m = (unsigned)(kn & 0xffffffffu);
      k = a == 0xffffffffu ? ~0ull : ((unsigned long long)a << 40 | (unsigned long long)branch[m] << 24 | m);
    }
    keys[p] = k;
  }
}

// Stable LSD radix sort of the 64-bit grouping keys on a derived sort value
// (8-bit digits; each pass: per-tile digit counts, an exclusive scan over
// [digit][tile] (done by each scatter tile itself when there are few tiles),
// a stable scatter). Sort value of a key:
//   by node:          node, invalid or padding keys n_nodes (last);
//   by (node, branch): node * C_max + branch, invalid or padding n_nodes * C_max.
// Keys enter in the order whose ties must be kept (batch order for the first
// sort, node-then-batch order for the second), so the result is ordered by
// (value, input position).
constexpr int kRadixWarps = 8, kRadixThreads = 32 * kRadixWarps;
constexpr int kRadixPerWarp = 256, kRadixTile = kRadixWarps * kRadixPerWarp;  // keys per tile (one CTA)

struct SortSpec {
  int by_branch;  // 0: by node, 1: by (node, branch)
  int n_nodes, C_max;
};

__device__ __forceinline__ unsigned long long sort_value(unsigned long long k, const SortSpec& sp) {
  if (!sp.by_branch) {
    const unsigned a = (unsigned)(k >> 32);
    return a >= (unsigned)sp.n_nodes ? (unsigned long long)sp.n_nodes : (unsigned long long)a;
  }
  if (k == ~0ull) return (unsigned long long)sp.n_nodes * (unsigned long long)sp.C_max;
  return (k >> 40) * (unsigned long long)sp.C_max + ((k >> 24) & 0xffffull);
}

__global__ void __launch_bounds__(kRadixThreads) radix_count_kernel(const unsigned long long* __restrict__ keys, int n,
                                                                   SortSpec sp, int shift, int* __restrict__ hist,
                                                                   int tiles) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kRadixTile;
  for (int i = base + threadIdx.x; i < base + kRadixTile && i < n; i += kRadixThreads) {
    const unsigned d = (unsigned)(sort_value(keys[i], sp) >> shift) & 255u;
    const unsigned peers = __match_any_sync(__activemask(), d);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[d], __popc(peers));
  }
  __syncthreads();
  hist[threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of the [digit][tile] counts, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) radix_scan_kernel(int* __restrict__ hist, int total) {
  __shared__ int part[1024];
  const int per = (total + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(total, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += hist[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the per-thread sums
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = lo; i < hi; ++i) {
    const int v = hist[i];
    hist[i] = run;
    run += v;
  }
}

// Stable scatter: warp w of tile t takes keys [t * kRadixTile + w * kRadixPerWarp, +kRadixPerWarp)
// 32 at a time in order; a key's destination is the scanned count of its digit
// for the tile, plus the keys of that digit in earlier warps of the tile, plus
// those earlier in its own warp.
__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(const unsigned long long* __restrict__ in,
                                                                     unsigned long long* __restrict__ out, int n,
                                                                     SortSpec sp, int shift,
                                                                     const int* __restrict__ hist, int tiles,
                                                                     int scanned) {
  __shared__ int wcnt[kRadixWarps][256];
  __shared__ int boff[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kRadixWarps * 256; i += kRadixThreads) (&wcnt[0][0])[i] = 0;
  if (scanned) {
    boff[threadIdx.x] = hist[threadIdx.x * tiles + blockIdx.x];
  } else {
    // few tiles: this tile's offsets straight from the counts (keys of smaller
    // digits in all tiles, plus keys of its digit in earlier tiles)
    const int d = threadIdx.x;
    int tot = 0, pre = 0;
    for (int t = 0; t < tiles; ++t) {
      const int v = hist[d * tiles + t];
      tot += v;
      if (t < (int)blockIdx.x) pre += v;
    }
    boff[d] = tot;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {  // inclusive scan of the digit totals
      const int v = d >= o ? boff[d - o] : 0;
      __syncthreads();
      boff[d] += v;
      __syncthreads();
    }
    const int incl = boff[d];
    __syncthreads();
    boff[d] = incl - tot + pre;
  }
  __syncthreads();
  constexpr int kIt = kRadixPerWarp / 32;
  const int base = blockIdx.x * kRadixTile + warp * kRadixPerWarp;
  unsigned long long kk[kIt];
  int dd[kIt], lr[kIt];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int i = base + it * 32 + lane;
    const bool valid = i < n;
    kk[it] = valid ? in[i] : 0ull;
    const int d = valid ? (int)((sort_value(kk[it], sp) >> shift) & 255ull) : 256;  // 256: no key
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    dd[it] = d;
    lr[it] = d < 256 ? wcnt[warp][d] + __popc(peers & lt) : 0;
    __syncwarp();
    if (d < 256 && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: keys of that digit in earlier warps of the tile
    int run = 0;
    for (int w = 0; w < kRadixWarps; ++w) {
      const int v = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kIt; ++it)
    if (dd[it] < 256) out[boff[dd[it]] + wcnt[warp][dd[it]] + lr[it]] = kk[it];
}

// Sorts keys[0, n) by their sort value; tmp holds n keys and hist 256 * tiles
// ints. Returns the buffer that holds the result (keys or tmp).
unsigned long long* radix_sort(unsigned long long* keys, unsigned long long* tmp, int* hist, int n, SortSpec sp,
                               cudaStream_t s) {
  const int tiles = (n + kRadixTile - 1) / kRadixTile;
  const unsigned long long vmax = sp.by_branch ? (unsigned long long)sp.n_nodes * (unsigned long long)sp.C_max
                                               : (unsigned long long)sp.n_nodes;
  unsigned long long* a = keys;
  unsigned long long* b = tmp;
  for (int shift = 0; shift < 64 && (vmax >> shift) != 0; shift += 8) {
    radix_count_kernel<<<tiles, kRadixThreads, 0, s>>>(a, n, sp, shift, hist, tiles);
    const int scanned = tiles > 64;  // else each scatter tile reads the counts itself
    if (scanned) radix_scan_kernel<<<1, 1024, 0, s>>>(hist, 256 * tiles);
    radix_scatter_kernel<<<tiles, kRadixThreads, 0, s>>>(a, b, n, sp, shift, hist, tiles, scanned);
    unsigned long long* c = a;
    a = b;
    b = c;
  }
  return a;
}

struct PwArgs {
  int M, n_nodes, d_s, d_a, d_o, C_max, d_omega;
  double k_o, alpha;
  float lambda, sigma;
  int lik_kind;
  uint32_t key0, key1, step, planner;
  const float* act;
  long long* N;
  int32_t* C;
  float* obs;
  const float* s_next;
  int32_t* branch;
  uint8_t* widened;
  float* ell;
  double* w;
  int32_t* idx;
  float* s_out;
  double* cw;
  int32_t* list;
  int32_t* count;
  int32_t* gstart;  // [n_nodes] first sorted position of the node's group, -1 if absent
  int32_t* gend;    // [n_nodes]
  int32_t* c0;      // [n_nodes] branch count before the batch
  int32_t* nwid;    // [n_nodes] widenings in the batch
  int32_t* wpos;    // [n_nodes][C_max] group ranks of the widening simulations
  long long* thr;   // [C_max] T(C): the smallest visit count n with C < k_o n^alpha_o
  int32_t* big;     // [M] first sorted positions of the (node, branch) groups left to the warp kernel
  int32_t* big_count;
  WsHeader* hdr;
};

constexpr long long kNever = 0x7fffffffffffffffLL;  // a threshold no visit count reaches

// Phase 2 set-up: T(C) for every branch count C < C_max, the smallest visit
// count n >= 1 with C < k_o * pow(n, alpha_o) (the per-simulation rule, same
// FP64 expression). The rule is monotone in n, so a node holding C branches
// widens at its first visit with count >= T(C), whatever node it is: one FP64
// search per branch count per call instead of one per node. One warp per C:
// the lanes test 32 visit counts around the inverse (C / k_o)^(1 / alpha_o)
// at once; a boundary outside that window is bracketed and bisected.
__global__ void pw_thresholds_kernel(PwArgs p) {
  const int C = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (C >= p.C_max) return;
  constexpr long long kCap = 4000000000000000000LL;
  auto pred = [&](long long n) { return (double)C < p.k_o * pow((double)n, p.alpha); };
  const double est = pow((double)C / p.k_o, 1.0 / p.alpha);
  long long T = kNever;
  if (est < 1.0e18) {
    // the 32 lanes test the visit counts around the estimate at once
    long long n0 = (long long)floor(est) - 15;
    if (n0 < 1) n0 = 1;
    const unsigned ball = __ballot_sync(0xffffffffu, pred(n0 + lane));
    if (ball != 0u && ((ball & 1u) == 0u || n0 == 1)) {
      T = n0 + __ffs(ball) - 1;  // the rule is monotone: false below, true from here
    } else if (lane == 0) {
      // not bracketed by the window: bracket by doubling steps from the
      // estimate, then bisect (bounded whatever the estimate's error)
      long long n = n0, lo, hi;
      bool found = true;
      if (pred(n)) {
        hi = n;
        long long d = 1;
        lo = n - d;
        while (lo >= 1 && pred(lo)) {
          hi = lo;
          d <<= 1;
          lo = n - d;
        }
        if (lo < 1) lo = 0;
      } else {
        lo = n;
        long long d = 1;
        hi = n + d;
        while (hi < kCap && !pred(hi)) {
          lo = hi;
          d <<= 1;
          hi = n + d;
        }
        found = hi < kCap;
      }
      if (found) {
        while (hi - lo > 1) {
          const long long mid = lo + (hi - lo) / 2;
          if (pred(mid)) hi = mid;
          else lo = mid;
        }
        T = hi;
      }
    }
  }
  if (lane == 0) p.thr[C] = T;
}

// Phase 2a: first and one-past-last sorted position of every node's group.
__global__ void pw_bounds_kernel(const unsigned long long* __restrict__ keys, PwArgs p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.M) return;
  const unsigned a = (unsigned)(keys[q] >> 32);
  if (a == 0xffffffffu) return;
  if (q == 0 || (unsigned)(keys[q - 1] >> 32) != a) p.gstart[a] = q;
  if (q == p.M - 1 || (unsigned)(keys[q + 1] >> 32) != a) p.gend[a] = q + 1;
}

// Phase 2b: one warp per visited node. The j-th widening of the batch (branch
// count C0 + j before it) happens at rank r_j = max(r_{j-1} + 1, t_j), t_j the
// rank at which the visit count reaches T(C0 + j); so r_j = j + max_{i <= j}
// (t_i - i): the lanes take 32 consecutive branch counts at once and a prefix
// maximum gives the ranks. The warp updates N and C and lists the widened
// simulations for the observation sampler (slots reserved atomically; each
// entry fills its own branch, so their order does not matter).
__global__ void pw_widen_kernel(const unsigned long long* __restrict__ keys, PwArgs p) {
  const int a = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (a >= p.n_nodes) return;
  const int q = p.gstart[a];
  if (q < 0) return;
  const int g = p.gend[a] - q;
  const long long n0 = p.N[a];
  const int C0 = p.C[a];
  int* wpos = p.wpos + (size_t)a * p.C_max;
  int nw = 0, carry = 0;  // widenings found; running max of t_i - i
  for (int base = 0; base < p.C_max - C0; base += 32) {
    const int j = base + lane;
    // threshold rank of branch count C0 + j: the rank whose visit count n0 + r + 1 reaches T
    int t = g;
    if (j < p.C_max - C0) {
      const long long T = p.thr[C0 + j];
      if (T <= n0 + g) t = T > n0 + 1 ? (int)(T - n0 - 1) : 0;
    }
    int m = t - j;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, m, o);
      if (lane >= o) m = max(m, v);
    }
    m = max(m, carry);
    const int r = j + m;  // strictly increasing in j
    const bool w = j < p.C_max - C0 && r < g;
    if (w) wpos[j] = r;
    nw += __popc(__ballot_sync(0xffffffffu, w));
    carry = __shfl_sync(0xffffffffu, m, 31);
    if (!__shfl_sync(0xffffffffu, w, 31)) break;  // the later ones fall past the batch
  }
  if (lane == 0) {
    p.c0[a] = C0;
    p.nwid[a] = nw;
    p.N[a] = n0 + g;
    p.C[a] = C0 + nw;
  }
  if (nw) {
    int slot = 0;
    if (lane == 0) slot = atomicAdd(p.count, nw);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    __syncwarp();
    for (int i = lane; i < nw; i += 32) p.list[slot + i] = (int32_t)(keys[q + wpos[i]] & 0xffffffffu);
  }
}

// Phase 2c: one thread per simulation. Its rank r in the node group gives the
// branch count it saw (C0 + the widenings ranked before it); a widening
// simulation takes the new branch, the others join branch floor(u C), u the
// 24-bit uniform of Philox counter (m, step, 0, stream 6) (u C is exact in FP64:
// a 24-bit fraction times an integer).
__global__ void pw_assign_kernel(const unsigned long long* __restrict__ keys, PwArgs p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.M) return;
  const unsigned a = (unsigned)(keys[q] >> 32);
  if (a == 0xffffffffu) return;
  const unsigned m = (unsigned)(keys[q] & 0xffffffffu);
  const int r = q - p.gstart[a], nw = p.nwid[a];
  const int* wpos = p.wpos + (size_t)a * p.C_max;
  int cnt = 0;
  while (cnt < nw && wpos[cnt] < r) ++cnt;
  const int C = p.c0[a] + cnt;
  if (cnt < nw && wpos[cnt] == r) {
    p.branch[m] = C;
    p.widened[m] = 1;
  } else {
    const uint4 x = philox(make_uint4(m, p.step, 0u, ctr_word3(6u, p.planner, 0u)), p.key0, p.key1);
    const int b = (int)floor((double)uniform24(x.x) * (double)C);
    p.branch[m] = b < C - 1 ? b : C - 1;
    p.widened[m] = 0;
  }
}

MlpDev mlp_dev(const voila_mlp* M) {
  MlpDev m;
  memset(&m, 0, sizeof(m));
  m.n_layers = M->n_layers;
  m.act = M->act;
  m.prec = M->prec;
  for (int l = 0; l <= VOILA_MAX_LAYERS; ++l) m.dims[l] = M->dims[l];
  for (int l = 0; l < M->n_layers; ++l) {
    m.W[l] = M->W[l];
    m.b[l] = M->b[l];
  }
  return m;
}

// Phase 3b: o = f_Z([s'_m; a; omega_Z(m)]) for the listed simulations -> obs[a][branch_m].
template <typename TW>
__global__ void __launch_bounds__(kSimtThreads) pw_observe_kernel(MlpDev gz, const int32_t* __restrict__ node, PwArgs p,
                                                                  int ld) {
  extern __shared__ __align__(16) float sm[];
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  __shared__ int rows_m[kSimtRows];
  const int cnt = *p.count;
  const int din = p.d_s + p.d_a + p.d_omega;
  for (int t0 = blockIdx.x * kSimtRows; t0 < cnt; t0 += gridDim.x * kSimtRows) {
    const int nr = min(kSimtRows, cnt - t0);
    __syncthreads();
    if (threadIdx.x < kSimtRows) rows_m[threadIdx.x] = threadIdx.x < nr ? p.list[t0 + threadIdx.x] : 0;
    __syncthreads();
    for (int e = threadIdx.x; e < kSimtRows * din; e += blockDim.x) {
      const int r = e / din, c = e % din;
      float v = 0.0f;
      if (r < nr && c < p.d_s + p.d_a) {
        const int m = rows_m[r];
        v = c < p.d_s ? p.s_next[(size_t)m * p.d_s + c] : p.act[(size_t)node[m] * p.d_a + c - p.d_s];
      }
      bufA[r * ld + c] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * ((p.d_omega + 3) / 4); e += blockDim.x) {
      const int r = e / ((p.d_omega + 3) / 4), b = e % ((p.d_omega + 3) / 4);
      const float4 z = normal4(p.key0, p.key1, (uint32_t)rows_m[r], 0u, p.step, VOILA_STREAM_OBS_OMEGA, p.planner,
                               (uint32_t)b);
      const float zz[4] = {z.x, z.y, z.z, z.w};
      for (int i = 0; i < 4 && 4 * b + i < p.d_omega; ++i) bufA[r * ld + p.d_s + p.d_a + 4 * b + i] = zz[i];
    }
    const float* y = simt_mlp<TW>(gz, bufA, bufB, ld, nr);
    for (int e = threadIdx.x; e < nr * p.d_o; e += blockDim.x) {
      const int r = e / p.d_o, c = e % p.d_o;
      const int m = rows_m[r];
      p.obs[((size_t)node[m] * p.C_max + p.branch[m]) * p.d_o + c] = y[r * ld + c];
    }
  }
}

// Phase 4: l(s'_m, a, o_branch) for every simulation (MLP on the CUDA cores,
// or the analytic Gaussian kind).
template <typename TW>
__global__ void __launch_bounds__(kSimtThreads) pw_likelihood_kernel(MlpDev lm, const int32_t* __restrict__ node,
                                                                     PwArgs p, int ld) {
  extern __shared__ __align__(16) float sm[];
  float* bufA = sm;
  float* bufB = bufA + kSimtRows * ld;
  const int din = p.d_s + p.d_a + p.d_o;
  for (int t0 = blockIdx.x * kSimtRows; t0 < p.M; t0 += gridDim.x * kSimtRows) {
    const int nr = min(kSimtRows, p.M - t0);
    if (p.lik_kind == VOILA_LIK_GAUSSIAN) {
      for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const int m = t0 + r, a = node[m];
        float l = 0.0f;
        if (a >= 0 && a < p.n_nodes) {
          const float* o = p.obs + ((size_t)a * p.C_max + p.branch[m]) * p.d_o;
          float acc = 0.0f;
          for (int d = 0; d < p.d_o; ++d) {
            const float df = o[d] - p.s_next[(size_t)m * p.d_s + d];
            acc = fmaf(df, df, acc);
          }
          l = -acc / (2.0f * p.sigma * p.sigma);
        }
        p.ell[m] = l;
      }
      continue;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kSimtRows * din; e += blockDim.x) {
      const int r = e / din, c = e % din;
      float v = 0.0f;
      if (r < nr) {
        const int m = t0 + r, a = node[m];
        if (a >= 0 && a < p.n_nodes) {
          if (c < p.d_s) v = p.s_next[(size_t)m * p.d_s + c];
          else if (c < p.d_s + p.d_a) v = p.act[(size_t)a * p.d_a + c - p.d_s];
          else v = p.obs[((size_t)a * p.C_max + p.branch[m]) * p.d_o + c - p.d_s - p.d_a];
        }
      }
      bufA[r * ld + c] = v;
    }
    const float* y = simt_mlp<TW>(lm, bufA, bufB, ld, nr);
    for (int r = threadIdx.x; r < nr; r += blockDim.x) p.ell[t0 + r] = y[r * ld];
  }
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kSmallGroup = 16;  // groups up to this size: one thread each

__device__ __forceinline__ double quantise(double w) { return rint(w * 4503599627370496.0) * 2.220446049250313e-16; }

// Phase 5a: one thread per sorted position; the first position of a (node,
// branch) group of at most kSmallGroup simulations does the group's SIR step
// alone (FP64 lanes are scarce: a warp per two-element group would leave most
// of them idle); the start of a larger group is listed for phase 5b. Same
// arithmetic as 5b: l / lambda as a product, exp(l / lambda - max) in FP32,
// FP64 sum, normalisation and 2^-52 quantisation, exact running sum, and the
// systematic positions p_j = (u0 + j) total / n (FP64, as the oracle) merged
// against the running sum (the first i with cw_i > p_j, else n - 1).
__global__ void __launch_bounds__(256) pw_resample_small_kernel(const unsigned long long* __restrict__ keys, PwArgs p) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.M) return;
  const unsigned long long k0 = keys[q];
  if (k0 == ~0ull) return;
  const unsigned long long g = k0 >> 24;
  if (q > 0 && (keys[q - 1] >> 24) == g) return;
  int n = 1;
  while (n <= kSmallGroup && q + n < p.M && (keys[q + n] >> 24) == g) ++n;
  if (n > kSmallGroup) {
    p.big[atomicAdd(p.big_count, 1)] = q;
    return;
  }
  auto sim = [&](int i) { return (int)(keys[q + i] & 0xffffffull); };
  const double inv_lam = 1.0 / (double)p.lambda;
  double mx = -INFINITY;
  for (int i = 0; i < n; ++i) {
    const double lw = (double)p.ell[sim(i)] * inv_lam;
    if (isnan(lw) || lw == INFINITY) {
      set_status(p.hdr, VOILA_ERR_NONFINITE, 61);
      return;
    }
    mx = fmax(mx, lw);
  }
  if (mx == -INFINITY) {
    set_status(p.hdr, VOILA_ERR_DEGENERATE, 62);
    return;
  }
  double Z = 0.0;
  for (int i = 0; i < n; ++i) {
    const double e = (double)expf((float)((double)p.ell[sim(i)] * inv_lam - mx));
    p.w[sim(i)] = e;
    Z += e;
  }
  const double inv_z = 1.0 / Z;
  double total = 0.0;
  for (int i = 0; i < n; ++i) {
    const double qv = quantise(p.w[sim(i)] * inv_z);
    p.w[sim(i)] = qv;
    total += qv;  // exact: multiples of 2^-52 summing to at most about 1
  }
  const unsigned a = (unsigned)(g >> 16), br = (unsigned)(g & 0xffffu);
  const uint4 x = philox(make_uint4(a, br, p.step, ctr_word3(VOILA_STREAM_RESAMPLE, p.planner, 1u)), p.key0, p.key1);
  const double u0 = uniform53(x.x, x.y);
  int i = 0;
  double c = p.w[sim(0)];  // cw_i
  for (int j = 0; j < n; ++j) {
    const double pj = __ddiv_rn(__dmul_rn(u0 + (double)j, total), (double)n);
    while (i < n - 1 && !(c > pj)) {
      ++i;
      c += p.w[sim(i)];
    }
    const int mj = sim(j), ms = sim(i);
    if (p.idx) p.idx[mj] = ms;
    for (int d = 0; d < p.d_s; ++d) p.s_out[(size_t)mj * p.d_s + d] = p.s_next[(size_t)ms * p.d_s + d];
  }
}

// Phase 5b: one warp per listed (node, branch) group (more than kSmallGroup
// simulations).
__global__ void __launch_bounds__(256) pw_resample_kernel(const unsigned long long* __restrict__ keys, PwArgs p) {
  const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wi >= *p.big_count) return;
  const int q = p.big[wi];
  const unsigned long long g = keys[q] >> 24;
  int n = 0;  // group size
  while (true) {
    const int e = q + n + lane;
    const bool same = e < p.M && (keys[e] >> 24) == g;
    const unsigned ball = __ballot_sync(0xffffffffu, same);
    if (ball == 0xffffffffu) {
      n += 32;
      continue;
    }
    n += __popc(~ball) == 32 ? 0 : __ffs(~ball) - 1;
    break;
  }
  const unsigned a = (unsigned)(g >> 16), br = (unsigned)(g & 0xffffu);
  auto sim = [&](int i) { return (int)(keys[q + i] & 0xffffffull); };
  // FP64 is scarce on this part: l / lambda as a product with 1 / lambda, one
  // exponential per weight, exp(l / lambda - max) <= 1 in FP32 (relative error
  // below 3e-7; a weight under 2^-53 of the group's largest quantises to zero
  // either way), kept in w between the passes; the sum Z, the normalisation
  // (a product with 1 / Z), the 2^-52 quantisation and the scan stay FP64
  const double inv_lam = 1.0 / (double)p.lambda;
  double mx = -INFINITY;
  bool bad = false;
  for (int i = lane; i < n; i += 32) {
    const double lw = (double)p.ell[sim(i)] * inv_lam;
    if (isnan(lw) || lw == INFINITY) bad = true;
    mx = fmax(mx, lw);
  }
  mx = wmax(mx);
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) set_status(p.hdr, VOILA_ERR_NONFINITE, 61);
    return;
  }
  if (mx == -INFINITY) {
    if (lane == 0) set_status(p.hdr, VOILA_ERR_DEGENERATE, 62);
    return;
  }
  double Z = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double e = (double)expf((float)((double)p.ell[sim(i)] * inv_lam - mx));
    p.w[sim(i)] = e;  // read back by this lane below
    Z += e;
  }
  Z = wsum(Z);
  const double inv_z = 1.0 / Z;
  // quantised weights and their inclusive prefix sum (exact in any order)
  double carry = 0.0;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    double qv = 0.0;
    if (i < n) {
      const double wv = p.w[sim(i)] * inv_z;
      qv = quantise(wv);
      p.w[sim(i)] = qv;
    }
    double inc = qv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (i < n) p.cw[q + i] = carry + inc;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  const uint4 x = philox(make_uint4(a, br, p.step, ctr_word3(VOILA_STREAM_RESAMPLE, p.planner, 1u)), p.key0, p.key1);
  const double u0 = uniform53(x.x, x.y);
  const double total = p.cw[q + n - 1];
  for (int j = lane; j < n; j += 32) {
    const double pj = __ddiv_rn(__dmul_rn(u0 + (double)j, total), (double)n);
    int lo = 0, hi = n;  // first i with cw[i] > pj
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (p.cw[q + mid] > pj) hi = mid;
      else lo = mid + 1;
    }
    const int src = lo < n ? lo : n - 1;
    const int mj = sim(j), ms = sim(src);
    if (p.idx) p.idx[mj] = ms;
    for (int d = 0; d < p.d_s; ++d) p.s_out[(size_t)mj * p.d_s + d] = p.s_next[(size_t)ms * p.d_s + d];
  }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int pow2_at_least(int m) {
  int n = 2;
  while (n < m) n <<= 1;
  return n;
}

// Workspace: header | tensor-core scratch (packed likelihood) | keys by node
// [n_pad] | keys by branch [n_pad] | cw [M] f64 | list [M] i32 | count |
// widened [M] u8 | ell [M] f32 | w [M] f64 | per node: gstart, gend, c0, nwid
// [n_nodes] i32 and wpos [n_nodes][C_max] i32
struct PwLayout {
  size_t tc, tcz, keys1, keys2, ktmp, hist, cw, list, count, widened, ell, w, gstart, gend, c0, nwid, wpos, thr,
      big, big_count, total;
};

bool pw_tc_likelihood(const voila_likelihood* ell, int d_s, int d_a, int d_o) {
  return ell && ell->kind == VOILA_LIK_MLP && ell->mlp && tc_pairs_supported(ell->mlp, d_s, d_a, d_o);
}

PwLayout pw_layout(const voila_pw_tree* tree, const voila_mlp* g_Z, const voila_likelihood* ell, int M) {
  PwLayout L;
  const size_t n_pad = (size_t)pow2_at_least(M < 2 ? 2 : M);
  size_t o = 1024;
  L.tc = o;
  if (ell && ell->kind == VOILA_LIK_MLP && ell->mlp) o += (tc_pairs_scratch_bytes(ell->mlp) + 1023) / 1024 * 1024;
  L.tcz = 0;  // packed f_Z weights of the tensor-core observation sampler (0: none)
  if (g_Z && tc_observe_supported(g_Z, 8, tree->d_a, g_Z->dims[0] - 8 - tree->d_a, tree->d_o)) {
    L.tcz = o;
    o += (tc_observe_scratch_bytes(g_Z) + 1023) / 1024 * 1024;
  }
  L.keys1 = o; o += a256(n_pad * 8);
  L.keys2 = o; o += a256(n_pad * 8);
  L.ktmp = o; o += a256(n_pad * 8);
  L.hist = o; o += a256((size_t)256 * ((n_pad + kRadixTile - 1) / kRadixTile) * 4);
  L.cw = o; o += a256((size_t)M * 8);
  L.list = o; o += a256((size_t)M * 4);
  L.count = o; o += 256;
  L.widened = o; o += a256((size_t)M);
  L.ell = o; o += a256((size_t)M * 4);
  L.w = o; o += a256((size_t)M * 8);
  const size_t nn = (size_t)tree->n_nodes;
  L.gstart = o; o += a256(nn * 4);
  L.gend = o; o += a256(nn * 4);
  L.c0 = o; o += a256(nn * 4);
  L.nwid = o; o += a256(nn * 4);
  L.wpos = o; o += a256(nn * (size_t)tree->C_max * 4);
  L.thr = o; o += a256((size_t)tree->C_max * 8);
  L.big = o; o += a256((size_t)M * 4);
  L.big_count = o; o += 256;
  L.total = o;
  return L;
}

int grid_of(long long n, int per) {
  long long g = (n + per - 1) / per;
  if (g > 148 * 16) g = 148 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace voila

using namespace voila;

extern "C" {

voila_status voila_progressive_widening_workspace_size(const voila_pw_tree* tree, const voila_mlp* g_Z,
                                                       const voila_likelihood* ell,
                                                       int32_t M, size_t* bytes) {
  VOILA_NVTX_RANGE();
  if (!tree || !ell || M < 0 || M > (1 << 24) || !bytes || tree->n_nodes < 1 || tree->n_nodes >= (1 << 24) ||
      tree->C_max < 1 || tree->C_max > 65535)
    return VOILA_ERR_ARG;
  *bytes = pw_layout(tree, g_Z, ell, M).total;
  return VOILA_OK;
}

voila_status voila_progressive_widening(const voila_pw_tree* tree, const int32_t* node, const float* s_next,
                                        int32_t M, int32_t d_s, const voila_mlp* g_Z, const voila_likelihood* ell,
                                        int32_t d_omega, double k_o, double alpha_o, float lambda, uint64_t seed,
                                        uint32_t step, uint32_t planner_id, int32_t* branch_out,
                                        uint8_t* widened_out, float* ell_out, double* w_out, int32_t* idx_out,
                                        float* s_out, void* workspace, size_t ws_bytes, voila_stream_t stream) {
  VOILA_NVTX_RANGE();
  if (!tree || !g_Z || !ell || M < 0 || M > (1 << 24) || d_s < 1 || d_omega < 0 || !(k_o > 0.0) ||
      !(alpha_o > 0.0) || !(lambda > 0.0f) || planner_id >= 65536)
    return VOILA_ERR_ARG;
  if (tree->n_nodes < 1 || tree->n_nodes >= (1 << 24) || tree->C_max < 1 || tree->C_max > 65535 || tree->d_a < 0 ||
      tree->d_o < 1 || !tree->N || !tree->C || !tree->obs || (tree->d_a && !tree->act))
    return VOILA_ERR_ARG;
  if (g_Z->n_layers < 1 || g_Z->n_layers > VOILA_MAX_LAYERS || (g_Z->prec != VOILA_FP32 && g_Z->prec != VOILA_BF16))
    return VOILA_ERR_UNSUPPORTED;
  if (g_Z->dims[0] != d_s + tree->d_a + d_omega || g_Z->dims[g_Z->n_layers] != tree->d_o) return VOILA_ERR_SHAPE;
  if (ell->kind == VOILA_LIK_MLP) {
    const voila_mlp* lm = ell->mlp;
    if (!lm || lm->n_layers < 1 || lm->n_layers > VOILA_MAX_LAYERS) return VOILA_ERR_ARG;
    if (lm->prec != VOILA_FP32 && lm->prec != VOILA_BF16) return VOILA_ERR_UNSUPPORTED;
    if (lm->dims[0] != d_s + tree->d_a + tree->d_o || lm->dims[lm->n_layers] != 1) return VOILA_ERR_SHAPE;
  } else if (ell->kind == VOILA_LIK_GAUSSIAN) {
    if (!(ell->sigma > 0.0f) || tree->d_o > d_s) return VOILA_ERR_ARG;
  } else {
    return VOILA_ERR_ARG;
  }
  const PwLayout L = pw_layout(tree, g_Z, ell, M);
  if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 1023)) return VOILA_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  if (cudaMemsetAsync(ws, 0, sizeof(WsHeader), s) != cudaSuccess) return VOILA_ERR_CUDA;
  if (M == 0) return VOILA_OK;
  if (!node || !s_next || !branch_out || !s_out) return VOILA_ERR_ARG;

  PwArgs p;
  memset(&p, 0, sizeof(p));
  p.M = M;
  p.n_nodes = tree->n_nodes;
  p.d_s = d_s;
  p.d_a = tree->d_a;
  p.d_o = tree->d_o;
  p.C_max = tree->C_max;
  p.d_omega = d_omega;
  p.k_o = k_o;
  p.alpha = alpha_o;
  p.lambda = lambda;
  p.sigma = ell->sigma;
  p.lik_kind = ell->kind;
  p.key0 = (uint32_t)(seed & 0xffffffffu);
  p.key1 = (uint32_t)(seed >> 32);
  p.step = step;
  p.planner = planner_id;
  p.act = tree->act;
  p.N = (long long*)tree->N;
  p.C = tree->C;
  p.obs = tree->obs;
  p.s_next = s_next;
  p.branch = branch_out;
  p.widened = (uint8_t*)(ws + L.widened);
  p.ell = ell_out ? ell_out : (float*)(ws + L.ell);
  p.w = w_out ? w_out : (double*)(ws + L.w);
  p.idx = idx_out;
  p.s_out = s_out;
  p.cw = (double*)(ws + L.cw);
  p.list = (int32_t*)(ws + L.list);
  p.count = (int32_t*)(ws + L.count);
  p.gstart = (int32_t*)(ws + L.gstart);
  p.gend = (int32_t*)(ws + L.gend);
  p.c0 = (int32_t*)(ws + L.c0);
  p.nwid = (int32_t*)(ws + L.nwid);
  p.wpos = (int32_t*)(ws + L.wpos);
  p.thr = (long long*)(ws + L.thr);
  p.big = (int32_t*)(ws + L.big);
  p.big_count = (int32_t*)(ws + L.big_count);
  p.hdr = (WsHeader*)ws;
  unsigned long long* keys1 = (unsigned long long*)(ws + L.keys1);
  unsigned long long* keys2 = (unsigned long long*)(ws + L.keys2);
  const int n_pad = pow2_at_least(M < 2 ? 2 : M);

  // 1. group by node
  pw_keys_node_kernel<<<grid_of(n_pad, 256), 256, 0, s>>>(node, M, n_pad, tree->n_nodes, keys1, p.hdr);
  unsigned long long* ktmp = (unsigned long long*)(ws + L.ktmp);
  int* hist = (int*)(ws + L.hist);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  SortSpec by_node;
  by_node.by_branch = 0;
  by_node.n_nodes = tree->n_nodes;
  by_node.C_max = tree->C_max;
  unsigned long long* spare = keys1;  // the buffer the first sort leaves free
  keys1 = radix_sort(keys1, ktmp, hist, M, by_node, s);
  if (keys1 == spare) spare = ktmp;
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  // 2. widening decisions
  if (cudaMemsetAsync(p.count, 0, sizeof(int32_t), s) != cudaSuccess) return VOILA_ERR_CUDA;
  if (cudaMemsetAsync(p.gstart, 0xff, (size_t)tree->n_nodes * sizeof(int32_t), s) != cudaSuccess)
    return VOILA_ERR_CUDA;
  pw_thresholds_kernel<<<(int)(((long long)tree->C_max * 32 + 255) / 256), 256, 0, s>>>(p);
  pw_bounds_kernel<<<(M + 255) / 256, 256, 0, s>>>(keys1, p);
  pw_widen_kernel<<<(int)(((long long)tree->n_nodes * 32 + 255) / 256), 256, 0, s>>>(keys1, p);
  pw_assign_kernel<<<(M + 255) / 256, 256, 0, s>>>(keys1, p);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  // 3. observations of the new branches (tensor cores for a BF16 f_Z of the
  // generator's shape, else CUDA cores)
  if (L.tcz && tc_observe_supported(g_Z, d_s, tree->d_a, d_omega, tree->d_o)) {
    const voila_status st = tc_observe_rows(g_Z, s_next, tree->act, p.list, p.count, M, node, branch_out,
                                            tree->n_nodes, tree->C_max, tree->obs, tree->d_o, p.key0, p.key1, step,
                                            planner_id, p.hdr, ws + L.tcz, s);
    if (st != VOILA_OK) return st;
  } else {
    const MlpDev gz = mlp_dev(g_Z);
    int wmax = 0;
    for (int l = 0; l <= g_Z->n_layers; ++l) wmax = g_Z->dims[l] > wmax ? g_Z->dims[l] : wmax;
    if (wmax > VOILA_MAX_WIDTH) return VOILA_ERR_SHAPE;
    const int ld = simt_ld(wmax);
    const size_t smem = (size_t)2 * kSimtRows * ld * sizeof(float);
    auto k = g_Z->prec == VOILA_BF16 ? pw_observe_kernel<__nv_bfloat16> : pw_observe_kernel<float>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return VOILA_ERR_CUDA;
    k<<<grid_of(M, kSimtRows), kSimtThreads, smem, s>>>(gz, node, p, ld);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  // 4. likelihood of every simulation against its branch's observation
  if (pw_tc_likelihood(ell, d_s, tree->d_a, tree->d_o)) {
    const voila_status st = tc_likelihood_rows(ell->mlp, s_next, tree->act, tree->obs, M, node, branch_out,
                                               tree->n_nodes, tree->C_max, p.ell, p.hdr, ws + L.tc, s);
    if (st != VOILA_OK) return st;
  } else {
    MlpDev lm;
    memset(&lm, 0, sizeof(lm));
    int ld = 1;
    size_t smem = 0;
    bool bf16 = false;
    if (ell->kind == VOILA_LIK_MLP) {
      lm = mlp_dev(ell->mlp);
      int wmax = 0;
      for (int l = 0; l <= ell->mlp->n_layers; ++l) wmax = ell->mlp->dims[l] > wmax ? ell->mlp->dims[l] : wmax;
      if (wmax > VOILA_MAX_WIDTH) return VOILA_ERR_SHAPE;
      ld = simt_ld(wmax);
      smem = (size_t)2 * kSimtRows * ld * sizeof(float);
      bf16 = ell->mlp->prec == VOILA_BF16;
    }
    auto k = bf16 ? pw_likelihood_kernel<__nv_bfloat16> : pw_likelihood_kernel<float>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem < 16 ? 16 : smem)) !=
        cudaSuccess)
      return VOILA_ERR_CUDA;
    k<<<grid_of(M, kSimtRows), kSimtThreads, smem, s>>>(lm, node, p, ld);
    if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  }
  // 5. group by (node, branch) and resample each group
  pw_keys_branch_kernel<<<grid_of(n_pad, 256), 256, 0, s>>>(keys1, branch_out, M, n_pad, keys2);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  SortSpec by_branch = by_node;
  by_branch.by_branch = 1;
  keys2 = radix_sort(keys2, spare, hist, M, by_branch, s);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  if (cudaMemsetAsync(p.big_count, 0, sizeof(int32_t), s) != cudaSuccess) return VOILA_ERR_CUDA;
  pw_resample_small_kernel<<<(M + 255) / 256, 256, 0, s>>>(keys2, p);
  // at most M / (kSmallGroup + 1) large groups
  pw_resample_kernel<<<(int)(((long long)(M / (kSmallGroup + 1) + 1) * 32 + 255) / 256), 256, 0, s>>>(keys2, p);
  if (cudaGetLastError() != cudaSuccess) return VOILA_ERR_CUDA;
  if (widened_out && cudaMemcpyAsync(widened_out, p.widened, (size_t)M, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return VOILA_ERR_CUDA;
  return VOILA_OK;
}

}  // extern "C"

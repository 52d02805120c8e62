// BF16 tensor-core GEMM (tcgen05) with MLP-training epilogues; host launcher.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace voila {

enum { kGemmFwdHidden = 0, kGemmFwdOut = 1, kGemmBwd = 2, kGemmPartial = 3 };

// D[M][N] = A[M][K] . B[N][K]^T (BF16 row-major operands, leading dimensions
// lda, ldb in elements, multiples of 8; N a multiple of 16, <= 256).
//   kGemmFwdHidden: z = D + bias; H = act(z), AD = act'(z) ([M][N], BF16),
//                   HT = H^T ([N][ldT], BF16; ldT >= M, a multiple of 8;
//                   columns from M on are not written).
//   kGemmFwdOut:    Y[m][n] = D + bias for n < n_real (FP32, row stride ldY).
//   kGemmBwd:       H = D * AD_in ([M][N], BF16, the backpropagated delta)
//                   and HT = its transpose.
//   kGemmPartial:   P[split][m][n] = D over the split's share of K (FP32);
//                   `splits` ways along K.
struct TcGemm {
  const __nv_bfloat16* A;
  long long lda;
  const __nv_bfloat16* B;
  long long ldb;
  long long M, K;
  int N;
  int splits;
  int mode, act;
  const float* bias;
  __nv_bfloat16* H;
  __nv_bfloat16* AD;
  __nv_bfloat16* HT;
  int ldT;
  const __nv_bfloat16* AD_in;
  float* Y;
  int ldY, n_real;
  float* P;
  WsHeader* hdr;
  bool spread;  // one CTA per unit instead of one persistent CTA per SM: the
                // units start on SMs as other work on the device releases them
};

size_t tc_gemm_smem_bytes();
cudaError_t tc_gemm(const TcGemm& g, cudaStream_t s);

}  // namespace voila

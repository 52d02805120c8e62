// MLP training forward/backward on the tensor cores (used by the distillation
// and InfoNCE steps for BF16 models).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/voila.h"
#include "common.cuh"

namespace voila {

// BF16 MLP, 2..8 layers, input and output widths <= 256, hidden widths
// multiples of 16 up to 256.
bool tc_train_supported(const voila_mlp* m);
// Scratch (1024-byte aligned) for a batch of M rows: operands, activations,
// deltas, transposes and split-K partials.
size_t tc_train_bytes(const voila_mlp* m, long long M);
// Y [M][d_L] FP32 = mlp(X), X [M][d_0] FP32; keeps what the backward needs in scratch.
// spread: the GEMMs launch one CTA per 128-row unit (see TcGemm::spread).
voila_status tc_train_forward(const voila_mlp* m, const float* X, long long M, float* Y, void* scratch,
                              WsHeader* hdr, cudaStream_t s, bool spread = false);
// grads (flat [W_0, b_0, W_1, b_1, ...], FP32) of the loss with dL/dY = dY [M][d_L]
// after tc_train_forward on the same scratch.
voila_status tc_train_backward(const voila_mlp* m, const float* dY, long long M, float* grads, void* scratch,
                               WsHeader* hdr, cudaStream_t s, bool spread = false);

}  // namespace voila

// Tensor-core (tcgen05) rollout: host-side entry points used by the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/voila.h"
#include "kernels.h"

namespace voila {

// Scratch bytes (packed, swizzled BF16 weight stream) the tensor-core
// rollout needs inside the caller's workspace.
size_t tc_rollout_scratch_bytes(const voila_mlp* g_T, const voila_reward* R);

// Launches the BF16 tcgen05 rollout; writes G [K][N]. Returns
// VOILA_ERR_UNSUPPORTED for shapes the kernel does not cover.
voila_status tc_rollout(const voila_mlp* g_T, const voila_reward* R, const RolloutArgs& a,
                        WsHeader* hdr, void* scratch, cudaStream_t s);

}  // namespace voila

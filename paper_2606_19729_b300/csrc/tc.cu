#include "tc.h"
namespace voila {
size_t tc_rollout_scratch_bytes(const voila_mlp*, const voila_reward*) { return 0; }
voila_status tc_rollout(const voila_mlp*, const voila_reward*, const RolloutArgs&, WsHeader*, void*, cudaStream_t) {
  return VOILA_ERR_UNSUPPORTED;
}
}  // namespace voila

// NVTX ranges around the C-ABI entry points: a profiler that records NVTX
// (ncu --nvtx, Nsight Systems) shows every call as a range named after the
// entry point, around the kernels it launches. NVTX3 is header-only; with no
// tool attached a range costs a function call into an empty handler.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace voila {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace voila

#define VOILA_NVTX_RANGE() ::voila::NvtxRange voila_nvtx_range_(__func__)

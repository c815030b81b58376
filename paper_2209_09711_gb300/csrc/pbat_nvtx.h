// pbat_nvtx.h -- NVTX range over a scope, for timelines and profiler filters
// (header-only NVTX v3 from the CUDA toolkit: a no-op unless a tool is
// attached).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace pbat {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace pbat

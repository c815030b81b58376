// pbat_nvtx.h -- NVTX range over a scope, for timelines and profiler filters
// (header-only NVTX v3 from the CUDA toolkit: a no-op unless a tool is
// attached).  Where the toolkit ships no NVTX headers the range compiles to
// nothing.
#pragma once
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define PBAT_HAVE_NVTX 1
#endif
#endif

namespace pbat {

struct NvtxRange {
#ifdef PBAT_HAVE_NVTX
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char*) {}
#endif
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace pbat

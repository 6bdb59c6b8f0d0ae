// Tracing of library calls: an NVTX range per entry point, so that Nsight
// timelines show the calls by name (a no-op unless a tool is attached).
#pragma once

#include <nvtx3/nvToolsExt.h>

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Named NVTX ranges around the library's host entry points that enqueue device work, so that a
// profiler can attribute launches to them (ncu --nvtx --nvtx-include). Header-only NVTX 3: with
// no profiler attached a push and a pop cost a few nanoseconds.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mcl {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace mcl

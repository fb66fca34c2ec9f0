// haf_nvtx.h -- NVTX ranges around the library's host entry points, so that
// a profiler's timeline (Nsight Systems; ncu with --nvtx filters) shows each
// call by name.  NVTX 3 is header-only: with no profiler attached a range
// costs one check of a function pointer.  Host code only.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace hafgb {

class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace hafgb

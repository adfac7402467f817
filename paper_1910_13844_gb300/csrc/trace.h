// NVTX ranges for profilers and tracers: one range per public call, per batched solve and per
// pass launch (named after the ls_kernel_kind).  NVTX is header-only: with no tool attached
// (NVTX_INJECTION64_PATH unset) a push or pop is one call through a no-op function pointer.
// Launches recorded into the solver's CUDA graph get their pass ranges once, at capture; a
// replayed iteration shows as one graph launch inside its "solve" range.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lsgpu {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// range name of a launch kind (LS_K_FX .. LS_K_OTHER)
inline const char* trace_kind_name(int kind) {
  static const char* const names[] = {"FX", "FY", "Z", "IY", "IX", "update", "scalar", "far", "other"};
  return kind >= 0 && kind < (int)(sizeof(names) / sizeof(names[0])) ? names[kind] : "other";
}

}  // namespace lsgpu

// Index checks of the debug build (compiled with -DLS_DEBUG_BOUNDS: libls_debug.so).
//
// LS_IN_BOUNDS(cond, site) guards a global or shared memory access of the hot kernels: in the
// debug build a false condition records `site` in this translation unit's error word (the first
// failure wins) and the access is skipped, so a wrong index shows up as a site code read back by
// ls_debug_bounds() instead of a fault; in the normal build it is the constant true and compiles
// away.  A site code is (kernel << 8) | access, listed below.
#pragma once

#include <cuda_runtime.h>

namespace lsgpu {

enum BoundsSite : unsigned {
  BS_FX_VEC = 0x101,      // FX: vector element (r, p, v, s) of a slot
  BS_FX_F = 0x102,        // FX: potential element
  BS_FX_DST = 0x103,      // FX: A1 element
  BS_FXB_COPY = 0x111,    // bulk-staged FX: a row block's copy range
  BS_FXB_SMEM = 0x112,    // bulk-staged FX: a staged element
  BS_ST_SRC = 0x201,      // FY/IY: source element
  BS_ST_DST = 0x202,      // FY/IY: destination element
  BS_ST_SMEM = 0x203,     // FY/IY: exchange entry
  BS_Z_TILE = 0x301,      // z pass: tile number / slot coordinate of a TMA copy
  BS_Z_SMEM = 0x302,      // z pass: view-buffer or exchange offset
  BS_Z_GREEN = 0x303,     // z pass: Green octant element
  BS_IX_SRC = 0x401,      // IX: A1 element
  BS_IX_VEC = 0x402,      // IX: vector element of a slot
  BS_IX_PART = 0x403,     // IX: per-block partial sums
  BS_UPD_VEC = 0x501,     // update: vector element of a slot
  BS_UPD_PART = 0x502,    // update: per-block partial sums
  BS_SLOT = 0x601,        // any pass: slot index beyond the launch's slots
};

#ifdef LS_DEBUG_BOUNDS
namespace {
__device__ unsigned g_bounds_site;   // internal linkage: one word per translation unit
}
__device__ __noinline__ static bool bounds_fail(unsigned site) {
  atomicCAS(&g_bounds_site, 0u, site);
  return false;
}
#define LS_IN_BOUNDS(cond, site) ((cond) ? true : ::lsgpu::bounds_fail(site))
// Host reader of this translation unit's word (returns it, optionally clearing it; 0xffffffff if
// it cannot be read); one LS_BOUNDS_READER(tag) line, inside namespace lsgpu, per translation unit
// that holds checked kernels.
#define LS_BOUNDS_READER(tag)                                                                      \
  unsigned bounds_site_##tag(bool clear) {                                                         \
    unsigned v = 0;                                                                                \
    if (cudaMemcpyFromSymbol(&v, g_bounds_site, sizeof(v)) != cudaSuccess) return 0xffffffffu;     \
    if (clear) {                                                                                   \
      const unsigned z = 0;                                                                        \
      cudaMemcpyToSymbol(g_bounds_site, &z, sizeof(z));                                            \
    }                                                                                              \
    return v;                                                                                      \
  }
#else
#define LS_IN_BOUNDS(cond, site) true
#define LS_BOUNDS_READER(tag)
#endif

}  // namespace lsgpu

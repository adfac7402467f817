// Launch parameters, slot selection and FFT geometry shared by the pencil FFT passes (passes.cuh)
// and the z pass (zpass.cuh).
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor map is encoded on the host through the runtime's driver entry point)

#include "common.cuh"
#include "debug_bounds.cuh"
#include "dft.cuh"

namespace lsgpu {

enum FxMode : int { FX_F_TIMES = 0, FX_COPY = 1, FX_BICG_P = 2, FX_BICG_S = 3 };
enum IxMode : int { IX_STORE = 0, IX_MATVEC = 1, IX_BICG_V = 2, IX_BICG_T = 3, IX_RESID = 4 };

struct SlotSel {
  const SlotDev* slots = nullptr;      // null: every slot runs with the defaults below
  unsigned mask = 0;                   // run slot s iff (slots[s].flags & mask) != 0 (mask 0: all)
  const float* f_default = nullptr;    // potential when slots == null
  int adj_default = 0;                 // adjoint flag when slots == null
  unsigned long long* runs = nullptr;  // if set: +1 per slot that ran (counted by its first CTA)
  int nslots = 0;                      // slots covered by this launch
};

// Upper bound on the views of one call (slot tables are sized by it).
constexpr int kMaxLaunchSlots = 1024;

struct FxParams {
  SlotSel sel;
  int nx, rows;                // transform length is 2nx; rows = ny*nz pencils per slot
  int mode;
  const float2* src;           // F_TIMES/COPY: vector; BICG_P/BICG_S: r
  float2* vp;                  // BICG_P: p (read, then overwritten with the new p)
  const float2* vv;            // BICG_P/BICG_S: v
  float2* vs;                  // BICG_S: s (written)
  size_t vstride;              // elements between slots for src/vp/vv/vs and f (f is shared unless slots)
  float2* dst;                 // [rows][2nx]
  size_t dst_stride;
  const float2* tw2;           // tw2[k1*R2 + n2] = exp(-2 pi i n2 k1 / L)
  int views_fastest = 0;       // launch grid (slots, row blocks) instead of (row blocks, slots) (autotuned)
  int bulk = 0;                // bulk-copy-staged persistent variant in the BiCGStab modes (autotuned)
  int sms = 0;                 // SMs of the device (grid of the bulk-staged variant)
  int* err = nullptr;          // set to 1 if a wait for a bulk copy gave up (bulk-staged variant)
  int dbg_probe = 0;           // debug build, test only: the plain kernel's slot check excludes the last slot
};

struct StridedParams {
  SlotSel sel;
  int ncont;                   // contiguous length of a row (2nx); the strided axis has length L
  int planes;                  // number of independent planes (nz for FY/IY)
  int out_o, out_m;            // IY: output window [out_o, out_o + out_m) of the cropped axis
  const float2* src; size_t src_stride;
  float2* dst; size_t dst_stride;
  size_t src_plane, dst_plane; // elements between planes
  const float2* tw;            // tw[j] = exp(-2 pi i j / L)
  int wide = 0;                // 32 pencils per CTA instead of 16 (autotuned)
};

struct ZParams {
  CUtensorMap tmap;            // A2 of all slots as floats [slot][nz][2ny][4nx], box {32, 1, nz, 1}, 128B swizzle
  CUtensorMap gmap;            // x-unfolded Green array as floats [nz+1][ny+1][4nx], box {32, 1, nz+1}, 128B swizzle
  SlotSel sel;
  int nx, ny, nz;              // A2 is [nz][2ny][2nx]
  float2* a2; size_t a2_stride;
  const float2* gocta;         // [(nz+1)][(ny+1)][(nx+1)], scaled by 1/(8 nx ny nz)
  const float2* twa;           // twa[t*R1 + k1] = exp(-2 pi i t k1 / L), t < R2 (forward split)
  const float2* twb;           // twb[t*R2 + j1] = exp(-2 pi i t j1 / L), t < R1 (transposed split)
  const float2* zwa;           // the same two tables for the split of the TMA-staged pass (ZRadix)
  const float2* zwb;
  int use_tma;                 // tmap is valid: the TMA-staged z pass may run
  int slot0;                   // slot coordinate of this launch's slot 0 in tmap
  int* err;                    // set to 1 if a wait for a TMA copy gave up (the launch's output is invalid)
  unsigned long long wait_ns = 0;   // limit of the TMA-staged pass's per-view waits (0: one second)
  int sms = 0;                 // SMs of the device: the persistent z passes launch (resident CTAs per SM) x sms CTAs
  int alt = 0;                 // TMA-staged z pass with the second split (zwa/zwb are that split's tables)
  int persist = 0;             // persistent TMA-staged z pass: 1 tiles assigned round-robin, 2 work units from a counter
  int gmap_ok = 0;             // gmap is valid (the dynamically scheduled form may run)
  unsigned* ctr = nullptr;     // work-unit counter of the dynamically scheduled form (zeroed before each launch)
  int stall = 0;               // test only: the compute warps' first wait is on a barrier nothing completes
};

struct IxParams {
  SlotSel sel;
  int nx, rows;                // input rows of length 2nx; output rows of length nx (or window)
  int mode;
  const float2* src; size_t src_stride;   // A1
  const float2* in0;           // MATVEC: x; BICG_V: p; BICG_T: s; RESID: x
  const float2* in1;           // BICG_V: rh; RESID: b
  float2* out0;                // STORE/MATVEC: y; BICG_V: v; BICG_T: t; RESID: r
  float2* out1;                // RESID: rh (= r)
  size_t vstride;              // slot stride for in*/out* (STORE: stride of out0)
  int out_o, out_m;            // STORE: output window [out_o, out_o+out_m) of x; out rows are out_m long
  double* partials;            // [slot][gridDim.x][4]
  int maxparts = 0;            // partial-sum blocks allocated per slot (0: not checked)
  const float2* tw2;
  int prefetch = 0;            // ask L2 for the epilogue operands at kernel start (autotuned)
};

// Debug-build index check: element `off` of slot `slot` of a [slots][stride] array whose slots
// hold `extent` elements each (stride 0 or unused when the launch covers one slot).
__device__ __forceinline__ bool slot_elem_ok(int slot, int nslots, size_t off, size_t extent, size_t stride) {
  return slot >= 0 && slot < nslots && off < extent && (nslots <= 1 || extent <= stride);
}

__device__ __forceinline__ bool slot_runs(const SlotSel& s, int slot) {
  return !(s.slots && s.mask && !(s.slots[slot].flags & s.mask));
}
__device__ __forceinline__ void count_run(const SlotSel& s) {
  if (s.runs && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(s.runs, 1ull);
}
// the same for kernels whose first block of a slot is `first`
__device__ __forceinline__ void count_run_if(const SlotSel& s, bool first) {
  if (s.runs && first && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(s.runs, 1ull);
}
__device__ __forceinline__ int slot_adj(const SlotSel& s, int slot);

// Ordered list of the slots of this launch that run (every CTA builds the same list).  An entry is
// the slot index with the slot's adjoint flag in bit 16 (read once here, not in the view loops:
// see active_slot / active_adj).  Block size must be a multiple of 32.  Returns the number of
// active slots.
__device__ __forceinline__ int active_slot(int e) { return e & 0xffff; }
__device__ __forceinline__ bool active_adj(int e) { return (e >> 16) != 0; }
__device__ __forceinline__ int build_active(const SlotSel& s, int* list, int* wsum) {
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nth = blockDim.x * blockDim.y;
  const int lane = tid & 31, w = tid >> 5, nw = nth >> 5;
  const int chunk = (s.nslots + nth - 1) / nth;
  const int beg = tid * chunk;
  const int end = min(beg + chunk, s.nslots);
  int c = 0;
  for (int i = beg; i < end; ++i) c += slot_runs(s, i) ? 1 : 0;
  int x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int v = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;
  }
  __syncthreads();
  int off = (w > 0 ? wsum[w - 1] : 0) + x - c;
  for (int i = beg; i < end; ++i)
    if (slot_runs(s, i)) list[off++] = i | (slot_adj(s, i) ? 1 << 16 : 0);
  const int total = wsum[nw - 1];
  __syncthreads();
  return total;
}

__device__ __forceinline__ const float* slot_f(const SlotSel& s, int slot) {
  return s.slots ? s.slots[slot].f : s.f_default;
}
__device__ __forceinline__ int slot_adj(const SlotSel& s, int slot) {
  return s.slots ? s.slots[slot].adjoint : s.adj_default;
}

__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

template <int L> struct Radix;
template <> struct Radix<16>  { static constexpr int R1 = 4,  R2 = 4;  };
template <> struct Radix<24>  { static constexpr int R1 = 4,  R2 = 6;  };
template <> struct Radix<32>  { static constexpr int R1 = 8,  R2 = 4;  };
template <> struct Radix<48>  { static constexpr int R1 = 8,  R2 = 6;  };
template <> struct Radix<64>  { static constexpr int R1 = 8,  R2 = 8;  };
template <> struct Radix<96>  { static constexpr int R1 = 8,  R2 = 12; };
template <> struct Radix<128> { static constexpr int R1 = 16, R2 = 8;  };
template <> struct Radix<144> { static constexpr int R1 = 12, R2 = 12; };
template <> struct Radix<192> { static constexpr int R1 = 16, R2 = 12; };
template <> struct Radix<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct Radix<288> { static constexpr int R1 = 12, R2 = 24; };
template <> struct Radix<384> { static constexpr int R1 = 16, R2 = 24; };

template <int L>
struct Geo {
  static constexpr int R1 = Radix<L>::R1, R2 = Radix<L>::R2;
  static constexpr int T = imax(R1, R2);
  // rows per CTA, contiguous passes: the largest count <= 256/T that makes whole warps
  static constexpr int PC = (T * (256 / T)) % 32 == 0 ? 256 / T : (T * (192 / T)) % 32 == 0 ? 192 / T : 32;
  static constexpr int PS = 16;                              // pencils per CTA, strided passes
  static constexpr int ZMINB = (T * PS > 256) ? 1 : 2;   // resident CTAs per SM asked of the z pass
  static constexpr int SROW = R2 + 1;                        // padded row of the contiguous exchange
  static constexpr size_t smem_contig = (size_t)PC * R1 * SROW * sizeof(float2);
  static constexpr size_t smem_strided = (size_t)L * PS * sizeof(float2);
  static constexpr size_t smem_z = (size_t)(2 * L + L) * PS * sizeof(float2);   // exchange + Ghat + 2 staging halves
};

}  // namespace lsgpu

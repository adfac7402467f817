// Pencil FFT passes of the zero-padded Green convolution (Theorem 1 with the
// twofold padding of Prop. 1), with the BiCGStab vector updates fused into the
// first and last passes.
//
// One matvec y = x - G (f x) on an nx*ny*nz grid is five passes, each one
// kernel, over complex64 arrays in HBM:
//   FX  rows (z,y):   f*x, zero-pad x -> 2nx, FFT along x      [nz][ny][nx]   -> A1 [nz][ny][2nx]
//   FY  pencils (z,kx): zero-pad y, FFT along y                 A1             -> A2 [nz][2ny][2nx]
//   Z   pencils (ky,kx): zero-pad z, FFT, * Ghat, IFFT, crop z  A2 in place (first nz planes)
//   IY  pencils (z,kx): IFFT along y, crop y                    A2             -> A1
//   IX  rows (z,y):   IFFT along x, crop x, epilogue            A1             -> [nz][ny][nx]
// The inverse normalisation 1/(8 nx ny nz) is folded into Ghat.
//
// Each length-L transform (L = 2n) is split L = R1 * R2 and done by T = max(R1, R2)
// threads per pencil in two register stages with one shared-memory exchange:
//   X[k1 + R1 k2] = sum_n2 W_R2^{n2 k2} W_L^{n2 k1} sum_n1 x[R2 n1 + n2] W_R1^{n1 k1}.
// Zero padding means the stage-1 inputs with n1 >= R1/2 vanish; cropping means
// stage 2 only produces k2 < R2/2.  The z pass chains forward stage 2, the
// Green multiply and inverse stage 1 in registers (the inverse uses the
// transposed split), so it needs two exchanges for a forward+inverse pair.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor map is encoded on the host through the runtime's driver entry point)

#include "common.cuh"
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
};

struct ZParams {
  CUtensorMap tmap;            // A2 of all slots as floats [slot][nz][2ny][4nx], box {32, 1, nz, 1}, 128B swizzle
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
  const float2* tw2;
  int prefetch = 0;            // ask L2 for the epilogue operands at kernel start (autotuned)
};

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

// Block reduction of NV per-thread float partial sums; thread 0 writes doubles to out[0..NV).
// Every sum across threads is float64: the partials are gathered in shared memory, each lane of
// the first warp adds a strided share of them in float64, and a float64 warp-shuffle tree combines
// the 32 lanes.  Only one warp issues float64 instructions (GB300's float64 rate is low: a shuffle
// tree in every warp cost the last FFT pass a quarter of its speed).  Blocks of at most 256
// threads; one call per kernel (the shared array is not guarded against reuse).
template <int NV>
__device__ __forceinline__ void block_sum_store(const float (&acc)[NV], double* out) {
  constexpr int kMaxThreads = 256;
  __shared__ float part[NV][kMaxThreads];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int j = 0; j < NV; ++j) part[j][tid] = acc[j];
  __syncthreads();
  if (tid < 32) {
    double d[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) d[j] = 0.0;
    for (int i = tid; i < nthreads; i += 32)
#pragma unroll
      for (int j = 0; j < NV; ++j) d[j] += (double)part[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < NV; ++j) d[j] += __shfl_xor_sync(0xffffffffu, d[j], o);
    if (tid == 0)
#pragma unroll
      for (int j = 0; j < NV; ++j) out[j] = d[j];
  }
}

// ------------------------------------------------------------------------- FX
template <int L>
__global__ void __launch_bounds__(Geo<L>::T * Geo<L>::PC, 6) k_fx(FxParams a) {
  using G = Geo<L>;
  constexpr int R1 = G::R1, R2 = G::R2;
  extern __shared__ float2 sm[];
  // with views_fastest the CTAs of all views that share a row block (and the potential's rows,
  // common to the views of one sample) run together and f is read from L2
  const int slot = a.views_fastest ? blockIdx.x : blockIdx.y;
  const int rb = a.views_fastest ? blockIdx.y : blockIdx.x;
  if (!slot_runs(a.sel, slot)) return;
  count_run_if(a.sel, rb == 0);
  const int t = threadIdx.x, p = threadIdx.y;
  const int nx = L / 2;
  const int row = rb * G::PC + p;
  const bool valid = row < a.rows;
  const size_t voff = (size_t)slot * a.vstride + (size_t)row * nx;
  const float* f = slot_f(a.sel, slot);
  float2 v[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
  if (valid && t < R2) {
    float fa = 1.f, fb = 0.f, al_re = 0.f, al_im = 0.f, om_re = 0.f, om_im = 0.f;
    bool first = false;
    if (a.mode == FX_BICG_P) {
      const SlotDev& sd = a.sel.slots[slot];
      first = sd.first != 0;
      fa = (float)sd.beta.x; fb = (float)sd.beta.y;
      om_re = (float)sd.omega.x; om_im = (float)sd.omega.y;
    } else if (a.mode == FX_BICG_S) {
      const SlotDev& sd = a.sel.slots[slot];
      al_re = (float)sd.alpha.x; al_im = (float)sd.alpha.y;
    }
#pragma unroll
    for (int n1 = 0; n1 < R1 / 2; ++n1) {
      const int x = R2 * n1 + t;
      const size_t i = voff + x;
      float2 val = __ldg(a.src + i);
      if (a.mode == FX_BICG_P) {
        if (!first) {
          // p = r + beta (p - omega v)
          float2 pv = a.vp[i], vv = __ldg(a.vv + i);
          float2 d = csub(pv, cmul(make_float2(om_re, om_im), vv));
          val = cadd(val, cmul(make_float2(fa, fb), d));
        }
        a.vp[i] = val;
      } else if (a.mode == FX_BICG_S) {
        // s = r - alpha v
        float2 vv = __ldg(a.vv + i);
        val = csub(val, cmul(make_float2(al_re, al_im), vv));
        a.vs[i] = val;
      }
      if (a.mode != FX_COPY) {
        const float fv = __ldg(f + (size_t)row * nx + x);
        val = cscale(val, fv);
      }
      v[n1] = val;
    }
  }
  float2* S = sm + (size_t)p * R1 * G::SROW;
  if (t < R2) {
    Dft<R1, -1, R1 / 2, R1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], __ldg(a.tw2 + k1 * R2 + t));
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) S[k1 * G::SROW + t] = v[k1];
  }
  __syncthreads();
  if (valid && t < R1) {
    float2 u[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = S[t * G::SROW + n2];
    Dft<R2, -1>::run(u);
    float2* d = a.dst + (size_t)slot * a.dst_stride + (size_t)row * L;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) d[t + R1 * k2] = u[k2];
  }
}

// ------------------------------------------------------------------------- FY / IY
// Pencils along a strided axis; tile = 16 consecutive entries of the contiguous axis.
template <int L, int DIR>
__global__ void __launch_bounds__(Geo<L>::T * Geo<L>::PS) k_strided(StridedParams a) {
  using G = Geo<L>;
  constexpr int R1 = G::R1, R2 = G::R2, P = G::PS;
  extern __shared__ float2 sm[];
  const int slot = blockIdx.y;
  if (!slot_runs(a.sel, slot)) return;
  count_run(a.sel);
  const int p = threadIdx.x, t = threadIdx.y;
  const int tiles_c = (a.ncont + P - 1) / P;
  const int plane = blockIdx.x / tiles_c;
  const int c = (blockIdx.x % tiles_c) * P + p;
  const bool valid = c < a.ncont;
  const float2* src = a.src + (size_t)slot * a.src_stride + (size_t)plane * a.src_plane + c;
  float2 v[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
  if (valid && t < R2) {
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int y = R2 * n1 + t;
      if (DIR < 0 ? (n1 < R1 / 2) : true) v[n1] = __ldg(src + (size_t)y * a.ncont);
    }
  }
  if (t < R2) {
    Dft<R1, DIR, (DIR < 0 ? R1 / 2 : R1), R1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      float2 w = __ldg(a.tw + k1 * t);
      v[k1] = DIR < 0 ? cmul(v[k1], w) : cmulc(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) sm[(k1 * R2 + t) * P + p] = v[k1];
  }
  __syncthreads();
  if (valid && t < R1) {
    float2 u[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = sm[(t * R2 + n2) * P + p];
    Dft<R2, DIR, R2, (DIR < 0 ? R2 : R2 / 2)>::run(u);
    float2* dst = a.dst + (size_t)slot * a.dst_stride + (size_t)plane * a.dst_plane + c;
    if (DIR < 0) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) dst[(size_t)(t + R1 * k2) * a.ncont] = u[k2];
    } else {
#pragma unroll
      for (int k2 = 0; k2 < R2 / 2; ++k2) {
        const int y = t + R1 * k2;
        const int yo = y - a.out_o;
        if (yo >= 0 && yo < a.out_m) dst[(size_t)yo * a.ncont] = u[k2];
      }
    }
  }
}

// ------------------------------------------------------------------------- Z
// Asynchronous global -> shared copies (no registers held while in flight).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// One CTA owns one (ky, 16-wide kx) tile of the z pencils and loops over the views of the launch:
// its Ghat tile is loaded into shared memory once, and the next view's pencils are copied into a
// second staging buffer while the current view is transformed.
template <int L>
__global__ void __launch_bounds__(Geo<L>::T * Geo<L>::PS, Geo<L>::ZMINB) k_z(ZParams a) {
  using G = Geo<L>;
  constexpr int R1 = G::R1, R2 = G::R2, P = G::PS, NZ = L / 2;
  constexpr int NT = G::T * P;
  extern __shared__ __align__(16) float2 sm[];
  float2* xs = sm;                 // exchange, [L][P]
  float2* gs = sm + L * P;         // Ghat tile, [L][P]
  float2* stage = gs + L * P;      // two staging buffers, [2][NZ][P]
  __shared__ int s_list[kMaxLaunchSlots];
  __shared__ int s_ws[32];
  const int nact = build_active(a.sel, s_list, s_ws);
  if (nact == 0) return;
  const int p = threadIdx.x, t = threadIdx.y, tid = t * P + p;
  const int ncont = 2 * a.nx;
  const int tiles_c = (ncont + P - 1) / P;
  const int ky = blockIdx.x / tiles_c;
  const int kx0 = (blockIdx.x % tiles_c) * P;
  const int kx = kx0 + p;
  const bool valid = kx < ncont;
  const size_t zstride = (size_t)(2 * a.ny) * ncont;
  // Ghat for kz in [0, L) of this tile, folded into the stored octant (Ghat is even per axis)
  const int fy = ky <= a.ny ? ky : 2 * a.ny - ky;
  for (int i = tid; i < L * P; i += NT) {
    const int kz = i / P, pp = i % P, kxx = kx0 + pp;
    if (kxx < ncont) {
      const int fz = kz <= a.nz ? kz : L - kz;
      const int fx = kxx <= a.nx ? kxx : ncont - kxx;
      cp_async8(&gs[i], a.gocta + ((size_t)fz * (a.ny + 1) + fy) * (a.nx + 1) + fx);
    }
  }
  // staging of one view: NZ rows of P complex values, as 16-byte pairs
  auto stage_view = [&](int slot, float2* buf) {
    const float2* base = a.a2 + (size_t)slot * a.a2_stride + (size_t)ky * ncont + kx0;
    for (int c = tid; c < NZ * (P / 2); c += NT) {
      const int z = c / (P / 2), j = 2 * (c % (P / 2));
      if (kx0 + j < ncont) cp_async16(&buf[z * P + j], base + (size_t)z * zstride + j);
    }
  };
  stage_view(active_slot(s_list[0]), stage);
  cp_async_commit();
#pragma unroll 1
  for (int iv = 0; iv < nact; ++iv) {
    const int slot = active_slot(s_list[iv]);
    const bool adj = active_adj(s_list[iv]);
    if (iv + 1 < nact) stage_view(active_slot(s_list[iv + 1]), stage + ((iv + 1) & 1) * NZ * P);
    cp_async_commit();
    cp_async_wait<1>();   // every group but the newest: this view's pencils (and the Ghat tile)
    __syncthreads();
    count_run(a.sel);
    const float2* stg = stage + (iv & 1) * NZ * P;
    float2* col = a.a2 + (size_t)slot * a.a2_stride + (size_t)ky * ncont + kx;
    // forward stage 1: inputs z = R2 n1 + t, n1 < R1/2 (z < nz)
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
    if (t < R2) {
#pragma unroll
      for (int n1 = 0; n1 < R1 / 2; ++n1) v[n1] = stg[(R2 * n1 + t) * P + p];
      Dft<R1, -1, R1 / 2, R1>::run(v);
      // stage twiddles exp(-2 pi i t k1 / L), read two at a time from this thread's row
      const float4* tw4 = reinterpret_cast<const float4*>(a.twa + t * R1);
#pragma unroll
      for (int k = 0; k < R1 / 2; ++k) {
        const float4 w = __ldg(tw4 + k);
        if (k > 0) v[2 * k] = cmul(v[2 * k], make_float2(w.x, w.y));
        v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w.z, w.w));
      }
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) xs[(k1 * R2 + t) * P + p] = v[k1];
    }
    __syncthreads();
    float2 u[R2];
    if (t < R1) {
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) u[n2] = xs[(t * R2 + n2) * P + p];
      Dft<R2, -1>::run(u);
      // Green multiply: u[k2] holds kz = t + R1 k2
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const float2 gv = gs[(t + R1 * k2) * P + p];
        u[k2] = adj ? cmulc(u[k2], gv) : cmul(u[k2], gv);
      }
      // inverse stage 1 (transposed split): DFT_R2 over k2, twiddle exp(+2 pi i j1 t / L)
      Dft<R2, +1>::run(u);
      const float4* twb4 = reinterpret_cast<const float4*>(a.twb + t * R2);
#pragma unroll
      for (int k = 0; k < R2 / 2; ++k) {
        const float4 w = __ldg(twb4 + k);
        if (k > 0) u[2 * k] = cmulc(u[2 * k], make_float2(w.x, w.y));
        u[2 * k + 1] = cmulc(u[2 * k + 1], make_float2(w.z, w.w));
      }
    }
    __syncthreads();
    if (t < R1) {
#pragma unroll
      for (int j1 = 0; j1 < R2; ++j1) xs[(j1 * R1 + t) * P + p] = u[j1];
    }
    __syncthreads();
    if (valid && t < R2) {
      float2 w[R1];
#pragma unroll
      for (int m2 = 0; m2 < R1; ++m2) w[m2] = xs[(t * R1 + m2) * P + p];
      Dft<R1, +1, R1, R1 / 2>::run(w);
      // outputs z = t + R2 j2, keep z < nz  (j2 < R1/2)
#pragma unroll
      for (int j2 = 0; j2 < R1 / 2; ++j2) col[(size_t)(t + R2 * j2) * zstride] = w[j2];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------- Z (TMA-staged)
// Same transform as k_z, for lengths whose pencil thread count T divides 32.  Each warp owns 32/T
// whole columns, so both exchanges are warp-local (__syncwarp); a view costs one CTA barrier.  The
// 16-column tile of a view is loaded by one TMA copy (128-byte swizzle, so column reads by row are
// free of bank conflicts), transformed in place, and written back by one TMA store; the next
// view's tile is loaded into the other buffer meanwhile.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait for phase `parity` of `bar`, giving up after about a second.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
// mbar_wait that also gives up as soon as another thread of the CTA has set *abort, or after
// limit_ns; a wait that runs out sets *abort itself.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t* bar, unsigned parity, volatile int* abort,
                                                unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n"
               ::"l"(map), "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Split of the TMA-staged z pass: the pass split where its thread count divides 32, else one that does
// (both factors even, so zero padding and cropping stay whole stages).
template <int L> struct ZRadix { static constexpr int R1 = Radix<L>::R1, R2 = Radix<L>::R2; };
template <> struct ZRadix<96>  { static constexpr int R1 = 16, R2 = 6;  };
template <> struct ZRadix<384> { static constexpr int R1 = 12, R2 = 32; };

template <int L>
struct ZW {
  static constexpr int R1 = ZRadix<L>::R1, R2 = ZRadix<L>::R2;
  static constexpr int T = imax(R1, R2);
  static constexpr bool ok = (32 % T) == 0;
  static constexpr int CPW = ok ? 32 / T : 1;   // whole columns per warp (lane = t * CPW + column)
  static constexpr int P = 16;                  // columns per CTA: one 128-byte TMA row
  static constexpr int NW = P / CPW;             // compute warps
  static constexpr int NT = 32 * NW + 32;        // + one producer warp (TMA loads and stores)
  static constexpr int NZ = L / 2;
  static constexpr int MINB = NT >= 512 ? 1 : NT >= 256 ? 2 : 512 / NT;
  // exchange pitch per column (in float2) congruent to 16/CPW mod 16: the CPW columns of a half-warp
  // then fall on disjoint banks; the Ghat rows [kz][P + CPW] are conflict-free for the same reason
  static constexpr int pitch(int n) { return n + (((16 / CPW) - n % 16) % 16 + 16) % 16; }
  static constexpr int GR = P + CPW;                                          // Ghat row [kz][GR], kz folded to [0, NZ]
  // exchange rows of R + 2 entries: a thread reads its row with 16-byte loads (two entries each)
  static constexpr int XP = pitch(imax(R1 * (R2 + 2), R2 * (R1 + 2)));
  static constexpr int TWA = R1 + 2, TWB = R2 + 2;                            // twiddle rows (16-byte aligned)
  static constexpr int NS = 4;                                                // view buffers (TMA pipeline depth)
  // each thread's Green values stay in registers across the view loop where they fit (R2 <= 16);
  // the Green tile is then dead once they are loaded, and the exchange area reuses it
  static constexpr bool GREG = R2 <= 16;
  static constexpr size_t r16(size_t b) { return (b + 15) / 16 * 16; }       // every region 16-byte aligned
  static constexpr size_t stage_bytes = (size_t)NZ * P * sizeof(float2);
  static constexpr size_t g_bytes = r16((size_t)(NZ + 1) * GR * sizeof(float2));
  static constexpr size_t x_bytes = r16((size_t)P * XP * sizeof(float2));
  static constexpr size_t off_g = NS * stage_bytes;
  static constexpr size_t off_x = GREG ? off_g : off_g + g_bytes;
  static constexpr size_t off_twa = off_x + (GREG ? (g_bytes > x_bytes ? g_bytes : x_bytes) : x_bytes);
  static constexpr size_t off_twb = off_twa + r16((size_t)R2 * TWA * sizeof(float2));
  static constexpr size_t off_bar = off_twb + r16((size_t)R1 * TWB * sizeof(float2));
  static constexpr int NBAR = 2 * NS + 1;                                     // full[NS], done[NS], never
  static constexpr size_t smem = off_bar + NBAR * sizeof(uint64_t) + 1024;    // + room to align the base to 1024
};

// Byte offset of element (z, c) of a [NZ][16] complex64 tile written by TMA with the 128-byte swizzle
// (16-byte chunk index XOR row mod 8).
__device__ __forceinline__ unsigned swz128(int z, int c) {
  return (unsigned)(z * 128 + ((((c >> 1) ^ (z & 7)) << 4) | ((c & 1) << 3)));
}

template <bool ADJ, int R1, int R2, int L, int GR>
__device__ __forceinline__ void green_mul(float2 (&u)[R2], const float2* gc, int t) {
  // u[k2] holds kz = t + R1 k2; Ghat(kz) = Ghat(L - kz), stored for kz in [0, L/2] with row pitch GR
#pragma unroll
  for (int k2 = 0; k2 < R2; ++k2) {
    const float2 g = k2 < R2 / 2 ? gc[(t + R1 * k2) * GR] : gc[(L - R1 * k2 - t) * GR];
    u[k2] = ADJ ? cmulc(u[k2], g) : cmul(u[k2], g);
  }
}

template <int L>
__global__ void __launch_bounds__(ZW<L>::NT, ZW<L>::MINB) k_zw(const __grid_constant__ ZParams a) {
  using W = ZW<L>;
  constexpr int R1 = W::R1, R2 = W::R2, P = W::P, NZ = W::NZ, CPW = W::CPW, T = W::T, NW = W::NW;
  static_assert(W::ok, "k_zw needs T | 32");
  static_assert(R1 % 2 == 0 && R2 % 2 == 0 && W::XP % 2 == 0, "16-byte exchange reads need even rows");
  extern __shared__ __align__(16) unsigned char zw_raw[];
  const unsigned raw = smem_addr(zw_raw);
  unsigned char* base = zw_raw + (((raw + 1023u) & ~1023u) - raw);
  float2* stage = reinterpret_cast<float2*>(base);
  float2* gs = reinterpret_cast<float2*>(base + W::off_g);
  float2* xs = reinterpret_cast<float2*>(base + W::off_x);
  float2* twa = reinterpret_cast<float2*>(base + W::off_twa);
  float2* twb = reinterpret_cast<float2*>(base + W::off_twb);
  constexpr int NS = W::NS;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + W::off_bar);   // [NS]: a view's tile has landed
  uint64_t* done = full + NS;                                         // [NS]: the compute warps are done with it
  uint64_t* never = done + NS;                                        // no thread arrives on it (stall test)
  __shared__ int s_list[kMaxLaunchSlots];
  __shared__ int s_ws[32];
  __shared__ int s_abort;
  const int nact = build_active(a.sel, s_list, s_ws);
  if (nact == 0) return;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int ncont = 2 * a.nx;
  const int tiles_c = ncont / P;
  const int ky = blockIdx.x / tiles_c;
  const int kx0 = (blockIdx.x % tiles_c) * P;
  const bool producer = warp == NW;
  const unsigned long long limit_ns = a.wait_ns ? a.wait_ns : 1000000000ull;
  if (producer && lane == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&done[k], NW);
    }
    mbar_init(never, 1);
    mbar_init_fence();
    for (int k = 0; k < NS && k < nact; ++k) {
      mbar_expect_tx(&full[k], (unsigned)W::stage_bytes);
      tma_load_4d(stage + (size_t)k * NZ * P, &a.tmap, &full[k], 2 * kx0, ky, 0, a.slot0 + active_slot(s_list[k]));
    }
  }
  // Ghat tile with kz folded into [0, NZ] (Ghat is even in every axis), and the stage twiddles
  const int fy = ky <= a.ny ? ky : 2 * a.ny - ky;
  for (int i = tid; i < (NZ + 1) * P; i += W::NT) {
    const int kz = i / P, cc = i % P, kx = kx0 + cc;
    const int fx = kx <= a.nx ? kx : ncont - kx;
    gs[kz * W::GR + cc] = __ldg(a.gocta + ((size_t)kz * (a.ny + 1) + fy) * (a.nx + 1) + fx);
  }
  for (int i = tid; i < R1 * R2; i += W::NT) {
    twa[(i / R1) * W::TWA + i % R1] = __ldg(a.zwa + i);
    twb[(i / R2) * W::TWB + i % R2] = __ldg(a.zwb + i);
  }
  __syncthreads();
  if (producer) {
    // producer: after the compute warps release a view's buffer, store it and refill it with the
    // view NS ahead
    if (lane != 0) return;
    int iv = 0;
    for (; iv < nact; ++iv) {
      const int buf = iv % NS;
      if (!mbar_wait_abort(&done[buf], (unsigned)(iv / NS) & 1u, &s_abort, limit_ns)) break;
      float2* sb = stage + (size_t)buf * NZ * P;
      tma_store_4d(&a.tmap, sb, 2 * kx0, ky, 0, a.slot0 + active_slot(s_list[iv]));
      bulk_commit();
      if (iv + NS < nact) {
        bulk_wait_read_all();   // the store has read the buffer
        mbar_expect_tx(&full[buf], (unsigned)W::stage_bytes);
        tma_load_4d(sb, &a.tmap, &full[buf], 2 * kx0, ky, 0, a.slot0 + active_slot(s_list[iv + NS]));
      }
    }
    bulk_wait_read_all();
    if (iv < nact) {
      // gave up at view iv: flag it, and give the loads still in flight into this CTA's buffers
      // (views iv .. iv + NS - 1, all issued) a bounded time to land (one second each, whatever
      // the per-view limit)
      atomicExch(a.err, 1);
      for (int j = iv; j < iv + NS && j < nact; ++j) mbar_wait(&full[j % NS], (unsigned)(j / NS) & 1u);
    }
    return;
  }
  // compute warps: each owns CPW whole columns (lane = t * CPW + column)
  const int t = lane / CPW;
  const int c = warp * CPW + lane % CPW;
  float2* xc = xs + c * W::XP;
  const float2* gc = gs + c;
  // byte offset of (z = t + R2 j, c) in a tile: row base for j = 0, plus j R2 rows
  const unsigned rb = swz128(t, c);
  // this thread's Green values (kz = t + R1 k2, the same for every view) stay in registers where
  // they fit (R2 <= 16); longer splits read them from the shared tile for every view
  constexpr bool GREG = W::GREG;
  float2 g[GREG ? R2 : 1];
#pragma unroll
  for (int k2 = 0; k2 < (GREG ? R2 : 1); ++k2)
    g[k2] = (GREG && (R1 == T || t < R1))
                ? (k2 < R2 / 2 ? gc[(t + R1 * k2) * W::GR] : gc[(L - R1 * k2 - t) * W::GR])
                : make_float2(0.f, 0.f);
  // the exchange area overlays the Green tile: every compute warp has its values before any writes
  if constexpr (GREG) asm volatile("bar.sync 1, %0;\n" ::"r"(NW * 32) : "memory");
#pragma unroll 1
  for (int iv = 0; iv < nact; ++iv) {
    const int buf = iv % NS;
    const bool ok = (a.stall && iv == 0) ? mbar_wait_abort(never, 0u, &s_abort, limit_ns)
                                         : mbar_wait_abort(&full[buf], (unsigned)(iv / NS) & 1u, &s_abort, limit_ns);
    if (!__all_sync(0xffffffffu, ok)) break;
    count_run(a.sel);
    unsigned char* sb = reinterpret_cast<unsigned char*>(stage + (size_t)buf * NZ * P);
    float2 u[R2];
    if (R2 == T || t < R2) {
      // forward stage 1: inputs z = R2 n1 + t, n1 < R1/2 (z < nz)
      float2 v[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
#pragma unroll
      for (int n1 = 0; n1 < R1 / 2; ++n1)
        v[n1] = *reinterpret_cast<const float2*>(sb + (R2 % 8 == 0 ? rb + R2 * n1 * 128 : swz128(R2 * n1 + t, c)));
      Dft<R1, -1, R1 / 2, R1>::run(v);
      const float4* tw4 = reinterpret_cast<const float4*>(twa + t * W::TWA);
#pragma unroll
      for (int k = 0; k < R1 / 2; ++k) {
        const float4 w = tw4[k];
        if (k > 0) v[2 * k] = cmul(v[2 * k], make_float2(w.x, w.y));
        v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w.z, w.w));
      }
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) xc[k1 * (R2 + 2) + t] = v[k1];
    }
    __syncwarp();
    if (R1 == T || t < R1) {
#pragma unroll
      for (int i = 0; i < R2 / 2; ++i) {
        const float4 q = *reinterpret_cast<const float4*>(xc + t * (R2 + 2) + 2 * i);
        u[2 * i] = make_float2(q.x, q.y);
        u[2 * i + 1] = make_float2(q.z, q.w);
      }
      Dft<R2, -1>::run(u);
      // the adjoint flag is read from the active list where it is used (not held across the stages)
      const bool adj = active_adj(s_list[iv]);
      if constexpr (GREG) {
        if (adj) {
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) u[k2] = cmulc(u[k2], g[k2]);
        } else {
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) u[k2] = cmul(u[k2], g[k2]);
        }
      } else if (adj) {
        green_mul<true, R1, R2, L, W::GR>(u, gc, t);
      } else {
        green_mul<false, R1, R2, L, W::GR>(u, gc, t);
      }
      // inverse stage 1 (transposed split): DFT_R2 over k2, twiddle exp(+2 pi i j1 t / L)
      Dft<R2, +1>::run(u);
      const float4* tw4 = reinterpret_cast<const float4*>(twb + t * W::TWB);
#pragma unroll
      for (int k = 0; k < R2 / 2; ++k) {
        const float4 w = tw4[k];
        if (k > 0) u[2 * k] = cmulc(u[2 * k], make_float2(w.x, w.y));
        u[2 * k + 1] = cmulc(u[2 * k + 1], make_float2(w.z, w.w));
      }
    }
    __syncwarp();
    if (R1 == T || t < R1) {
#pragma unroll
      for (int j1 = 0; j1 < R2; ++j1) xc[j1 * (R1 + 2) + t] = u[j1];
    }
    __syncwarp();
    if (R2 == T || t < R2) {
      float2 w[R1];
#pragma unroll
      for (int i = 0; i < R1 / 2; ++i) {
        const float4 q = *reinterpret_cast<const float4*>(xc + t * (R1 + 2) + 2 * i);
        w[2 * i] = make_float2(q.x, q.y);
        w[2 * i + 1] = make_float2(q.z, q.w);
      }
      Dft<R1, +1, R1, R1 / 2>::run(w);
      // outputs z = t + R2 j2 (j2 < R1/2: z < nz), in place
#pragma unroll
      for (int j2 = 0; j2 < R1 / 2; ++j2)
        *reinterpret_cast<float2*>(sb + (R2 % 8 == 0 ? rb + R2 * j2 * 128 : swz128(t + R2 * j2, c))) = w[j2];
    }
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[buf]);
  }
}

// ------------------------------------------------------------------------- IX
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

template <int L>
__global__ void __launch_bounds__(Geo<L>::T * Geo<L>::PC, 5) k_ix(IxParams a) {
  using G = Geo<L>;
  constexpr int R1 = G::R1, R2 = G::R2;
  extern __shared__ float2 sm[];
  const int slot = blockIdx.y;
  if (!slot_runs(a.sel, slot)) return;
  count_run(a.sel);
  const int t = threadIdx.x, p = threadIdx.y;
  const int nx = L / 2;
  const int row = blockIdx.x * G::PC + p;
  const bool valid = row < a.rows;
  // the epilogue's operands are read after both transforms: ask L2 for their lines now (one
  // 128-byte line per thread and vector; a row holds nx/16 lines)
  if (a.prefetch && valid && a.mode != IX_STORE) {
    constexpr int lines = (L / 2) / 16;
    const size_t voff0 = (size_t)slot * a.vstride + (size_t)row * nx;
    if (t < lines) prefetch_l2(a.in0 + voff0 + 16 * t);
    else if (t < 2 * lines && (a.mode == IX_BICG_V || a.mode == IX_RESID)) prefetch_l2(a.in1 + voff0 + 16 * (t - lines));
  }
  float2 v[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
  if (valid && t < R2) {
    const float2* s = a.src + (size_t)slot * a.src_stride + (size_t)row * L;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = __ldg(s + R2 * n1 + t);
  }
  float2* S = sm + (size_t)p * R1 * G::SROW;
  if (t < R2) {
    Dft<R1, +1>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmulc(v[k1], __ldg(a.tw2 + k1 * R2 + t));
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) S[k1 * G::SROW + t] = v[k1];
  }
  __syncthreads();
  float acc[3] = {0.f, 0.f, 0.f};
  if (valid && t < R1) {
    float2 u[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = S[t * G::SROW + n2];
    Dft<R2, +1, R2, R2 / 2>::run(u);
    const size_t voff = (size_t)slot * a.vstride + (size_t)row * nx;
#pragma unroll
    for (int k2 = 0; k2 < R2 / 2; ++k2) {
      const int x = t + R1 * k2;
      const float2 g = u[k2];
      const size_t i = voff + x;
      switch (a.mode) {
        case IX_STORE: {
          const int xo = x - a.out_o;
          if (xo >= 0 && xo < a.out_m) a.out0[(size_t)slot * a.vstride + (size_t)row * a.out_m + xo] = g;
        } break;
        case IX_MATVEC:
          a.out0[i] = csub(__ldg(a.in0 + i), g);
          break;
        case IX_BICG_V: {
          float2 vv = csub(__ldg(a.in0 + i), g);
          a.out0[i] = vv;
          float2 d = cdotterm(__ldg(a.in1 + i), vv);   // conj(rh) v
          acc[0] += d.x; acc[1] += d.y;
          acc[2] += vv.x * vv.x + vv.y * vv.y;          // ||v||^2 (relative breakdown test)
        } break;
        case IX_BICG_T: {
          float2 ss = __ldg(a.in0 + i);
          float2 tt = csub(ss, g);
          a.out0[i] = tt;
          float2 d = cdotterm(tt, ss);                  // conj(t) s
          acc[0] += d.x; acc[1] += d.y;
          acc[2] += tt.x * tt.x + tt.y * tt.y;
        } break;
        case IX_RESID: {
          float2 b = __ldg(a.in1 + i);
          float2 r = cadd(csub(b, __ldg(a.in0 + i)), g);   // b - (x - G f x)
          a.out0[i] = r;
          a.out1[i] = r;
          acc[0] += r.x * r.x + r.y * r.y;
          acc[1] += b.x * b.x + b.y * b.y;
        } break;
      }
    }
  }
  if (a.mode >= IX_BICG_V) {
    block_sum_store<3>(acc, a.partials + ((size_t)slot * gridDim.x + blockIdx.x) * 4);
  }
}

// ------------------------------------------------------------------------- launchers
struct PassLaunch {
  void (*fx)(const FxParams&, int nslots, cudaStream_t);
  void (*fy)(const StridedParams&, int nslots, cudaStream_t);
  void (*iy)(const StridedParams&, int nslots, cudaStream_t);
  void (*z)(const ZParams&, int nslots, cudaStream_t);
  void (*ix)(const IxParams&, int nslots, cudaStream_t);
  int rows_per_cta_contig;
  int pencils_per_cta_strided;
  int r1, r2;   // the split L = r1 * r2 of the two register stages (twiddle tables follow it)
  int zr1, zr2; // the split of the TMA-staged z pass
};

template <int L>
struct PassImpl {
  using G = Geo<L>;
  static void fx(const FxParams& a, int nslots, cudaStream_t st) {
    const unsigned rbs = (unsigned)((a.rows + G::PC - 1) / G::PC);
    dim3 blk(G::T, G::PC), grd = a.views_fastest ? dim3(nslots, rbs) : dim3(rbs, nslots);
    k_fx<L><<<grd, blk, G::smem_contig, st>>>(a);
  }
  static void ix(const IxParams& a, int nslots, cudaStream_t st) {
    dim3 blk(G::T, G::PC), grd((a.rows + G::PC - 1) / G::PC, nslots);
    k_ix<L><<<grd, blk, G::smem_contig, st>>>(a);
  }
  static void fy(const StridedParams& a, int nslots, cudaStream_t st) {
    dim3 blk(G::PS, G::T), grd(((a.ncont + G::PS - 1) / G::PS) * a.planes, nslots);
    k_strided<L, -1><<<grd, blk, G::smem_strided, st>>>(a);
  }
  static void iy(const StridedParams& a, int nslots, cudaStream_t st) {
    dim3 blk(G::PS, G::T), grd(((a.ncont + G::PS - 1) / G::PS) * a.planes, nslots);
    k_strided<L, +1><<<grd, blk, G::smem_strided, st>>>(a);
  }
  static void z(const ZParams& a0, int nslots, cudaStream_t st) {
    ZParams a = a0;
    a.sel.nslots = nslots;
    if constexpr (ZW<L>::ok) {
      if (a.use_tma && (2 * a.nx) % ZW<L>::P == 0 && a.nz <= 256) {
        k_zw<L><<<(2 * a.nx / ZW<L>::P) * (2 * a.ny), ZW<L>::NT, ZW<L>::smem, st>>>(a);
        return;
      }
    }
    dim3 blk(G::PS, G::T), grd(((2 * a.nx + G::PS - 1) / G::PS) * (2 * a.ny));
    k_z<L><<<grd, blk, G::smem_z, st>>>(a);
  }
  static cudaError_t setup() {
    cudaError_t e = cudaSuccess;
    {
      e = cudaFuncSetAttribute(k_fx<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_contig);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ix<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_contig);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strided<L, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_strided);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_strided<L, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_strided);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_z<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_z);
      if constexpr (ZW<L>::ok)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_zw<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZW<L>::smem);
    }
    return e;
  }
  static PassLaunch table() {
    PassLaunch t;
    t.fx = &fx; t.fy = &fy; t.iy = &iy; t.z = &z; t.ix = &ix;
    t.rows_per_cta_contig = G::PC;
    t.pencils_per_cta_strided = G::PS;
    t.r1 = G::R1;
    t.r2 = G::R2;
    t.zr1 = ZRadix<L>::R1;
    t.zr2 = ZRadix<L>::R2;
    return t;
  }
};

// Defined in one translation unit per length (passes_L*.cu).
#define LS_DECLARE_LENGTH(L) \
  PassLaunch pass_table_##L(); \
  cudaError_t pass_setup_##L();
LS_DECLARE_LENGTH(16)
LS_DECLARE_LENGTH(24)
LS_DECLARE_LENGTH(32)
LS_DECLARE_LENGTH(48)
LS_DECLARE_LENGTH(64)
LS_DECLARE_LENGTH(96)
LS_DECLARE_LENGTH(128)
LS_DECLARE_LENGTH(144)
LS_DECLARE_LENGTH(192)
LS_DECLARE_LENGTH(256)
LS_DECLARE_LENGTH(288)
LS_DECLARE_LENGTH(384)
#undef LS_DECLARE_LENGTH

#define LS_DEFINE_LENGTH(L) \
  PassLaunch pass_table_##L() { return PassImpl<L>::table(); } \
  cudaError_t pass_setup_##L() { return PassImpl<L>::setup(); }

}  // namespace lsgpu

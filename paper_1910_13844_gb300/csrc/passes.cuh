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

#include <algorithm>

#include "pass_common.cuh"
#include "zpass.cuh"

namespace lsgpu {

// Block reduction of NV per-thread float partial sums; out[0..NV) receives them as doubles.
// Every sum across threads is float64: the partials are gathered in shared memory, and warp j
// (j < NV) adds partial j of all threads, each lane a strided share in float64, combined by a
// float64 warp-shuffle tree.  Only NV warps issue float64 instructions, one sum each, in parallel
// (GB300's float64 rate is low: a shuffle tree of every sum in every warp cost the last FFT pass a
// quarter of its speed, and one warp doing all NV sums lengthens the block's tail).  Blocks of at
// least 32 NV and at most 256 threads; one call per kernel (the shared array is not guarded against
// reuse).
template <int NV>
__device__ __forceinline__ void block_sum_store(const float (&acc)[NV], double* out) {
  constexpr int kMaxThreads = 256;
  __shared__ float part[NV][kMaxThreads];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int j = 0; j < NV; ++j) part[j][tid] = acc[j];
  __syncthreads();
  const int j = tid >> 5, lane = tid & 31;
  if (j < NV) {
    double d = 0.0;
    for (int i = lane; i < nthreads; i += 32) d += (double)part[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) out[j] = d;
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
  if (!LS_IN_BOUNDS(slot < a.sel.nslots - (a.dbg_probe ? 1 : 0), BS_SLOT)) return;
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
      fa = sd.beta_f.x; fb = sd.beta_f.y;
      om_re = sd.omega_f.x; om_im = sd.omega_f.y;
    } else if (a.mode == FX_BICG_S) {
      const SlotDev& sd = a.sel.slots[slot];
      al_re = sd.alpha_f.x; al_im = sd.alpha_f.y;
    }
#pragma unroll
    for (int n1 = 0; n1 < R1 / 2; ++n1) {
      const int x = R2 * n1 + t;
      const size_t i = voff + x;
      if (!LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)row * nx + x, (size_t)a.rows * nx, a.vstride),
                        BS_FX_VEC))
        continue;
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
    for (int k2 = 0; k2 < R2; ++k2)
      if (LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)row * L + t + R1 * k2, (size_t)a.rows * L,
                                    a.dst_stride), BS_FX_DST))
        d[t + R1 * k2] = u[k2];
  }
}

// ------------------------------------------------------------------------- FX (bulk-copy staged)
// The same pass with the rows of every input vector staged in shared memory by bulk copies
// (cp.async.bulk, one per vector and row block: the rows of a block are contiguous), NSTG row blocks
// ahead, behind one mbarrier per stage.  Persistent: one CTA per SM walks the (active view, row
// block) items blockIdx.x, blockIdx.x + gridDim.x, ...; a thread loads its inputs from shared memory
// instead of issuing eight 8-byte loads per vector.  A potential row that is not 16-byte aligned is
// read from global memory instead of staged.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

template <int L>
struct FXB {
  using G = Geo<L>;
  static constexpr int PC = G::PC, NX = L / 2;
  static constexpr int NSTG = 3;                                        // row blocks in flight per CTA
  static constexpr size_t vec_bytes = (size_t)PC * NX * sizeof(float2);
  static constexpr size_t f_bytes = (size_t)PC * NX * sizeof(float);
  static constexpr size_t stage_bytes = 3 * vec_bytes + f_bytes;       // r, v, p and f (the BiCGStab p update)
  static constexpr size_t off_x = NSTG * stage_bytes;                  // exchange area of the two DFT stages
  static constexpr size_t off_bar = off_x + (G::smem_contig + 15) / 16 * 16;
  static constexpr size_t smem = off_bar + NSTG * sizeof(uint64_t);
  static constexpr bool ok = smem <= 227 * 1024 && stage_bytes % 16 == 0 && vec_bytes % 16 == 0;
};

template <int L>
__global__ void __launch_bounds__(Geo<L>::T * Geo<L>::PC, 1) k_fxb(FxParams a) {
  using G = Geo<L>;
  using B = FXB<L>;
  constexpr int R1 = G::R1, R2 = G::R2, PC = G::PC, NX = B::NX, NSTG = B::NSTG;
  constexpr int NT = G::T * G::PC;
  extern __shared__ __align__(16) unsigned char fxb_raw[];
  float2* S0 = reinterpret_cast<float2*>(fxb_raw + B::off_x);
  uint64_t* full = reinterpret_cast<uint64_t*>(fxb_raw + B::off_bar);
  __shared__ int s_list[kMaxLaunchSlots];
  __shared__ int s_ws[32];
  __shared__ int s_fb[NSTG];   // stage s holds the potential's rows
  const int nact = build_active(a.sel, s_list, s_ws);
  if (nact == 0) return;
  const int t = threadIdx.x, p = threadIdx.y, tid = p * G::T + t;
  const int nrb = (a.rows + PC - 1) / PC;
  const int nitems = nact * nrb;
  const int nmine = (nitems - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  if (nmine <= 0) return;
  const int nvec = a.mode == FX_BICG_P ? 3 : a.mode == FX_BICG_S ? 2 : 1;   // src (r), v, p
  auto stage = [&](int s) { return fxb_raw + (size_t)s * B::stage_bytes; };
  // issue the copies of this CTA's m-th item into stage s (thread 0)
  auto issue = [&](int m, int s) {
    const int k = (int)blockIdx.x + m * (int)gridDim.x;
    const int slot = active_slot(s_list[k / nrb]);
    const int row0 = (k % nrb) * PC;
    const int nrows = min(PC, a.rows - row0);
    const unsigned vb = (unsigned)(nrows * NX * sizeof(float2));
    const size_t voff = (size_t)slot * a.vstride + (size_t)row0 * NX;
    if (!LS_IN_BOUNDS(slot < a.sel.nslots && row0 >= 0 && row0 + nrows <= a.rows &&
                          (a.sel.nslots <= 1 || (size_t)a.rows * NX <= a.vstride), BS_FXB_COPY)) {
      s_fb[s] = 0;
      mbar_arrive(&full[s]);   // nothing copied: the stage's phase completes at once
      return;
    }
    const float* f = a.mode == FX_COPY ? nullptr : slot_f(a.sel, slot) + (size_t)row0 * NX;
    const bool fb = f && ((reinterpret_cast<uintptr_t>(f) & 15) == 0);
    s_fb[s] = fb ? 1 : 0;
    mbar_expect_tx(&full[s], (unsigned)(nvec * vb + (fb ? nrows * NX * sizeof(float) : 0)));
    unsigned char* st = stage(s);
    bulk_load(st, a.src + voff, vb, &full[s]);
    if (nvec >= 2) bulk_load(st + B::vec_bytes, a.vv + voff, vb, &full[s]);
    if (nvec >= 3) bulk_load(st + 2 * B::vec_bytes, a.vp + voff, vb, &full[s]);
    if (fb) bulk_load(st + 3 * B::vec_bytes, f, (unsigned)(nrows * NX * sizeof(float)), &full[s]);
  };
  if (tid == 0) {
    for (int s = 0; s < NSTG; ++s) mbar_init(&full[s], 1);
    mbar_init_fence();
    for (int m = 0; m < NSTG && m < nmine; ++m) issue(m, m);
  }
  __syncthreads();
  // this thread's stage twiddles exp(-2 pi i t k1 / L), the same for every item, in registers
  float2 twr[R1];
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) twr[k1] = t < R2 ? __ldg(a.tw2 + k1 * R2 + t) : make_float2(0.f, 0.f);
  for (int m = 0; m < nmine; ++m) {
    const int s = m % NSTG;
    const bool ok = mbar_wait(&full[s], (unsigned)(m / NSTG) & 1u);
    if (!__syncthreads_and(ok)) {
      // a copy did not land within its time limit: flag the launch, give the copies still in flight
      // into this CTA's stages a bounded time to land, and stop
      if (tid == 0) {
        atomicExch(a.err, 1);
        for (int q = m; q < m + NSTG && q < nmine; ++q) mbar_wait(&full[q % NSTG], (unsigned)(q / NSTG) & 1u);
      }
      __syncthreads();
      return;
    }
    const int k = (int)blockIdx.x + m * (int)gridDim.x;
    const int slot = active_slot(s_list[k / nrb]);
    const int rb = k % nrb;
    count_run_if(a.sel, rb == 0);
    const int row = rb * PC + p;
    const bool valid = row < a.rows;
    const unsigned char* st = stage(s);
    const float2* r_s = reinterpret_cast<const float2*>(st) + (size_t)p * NX;
    const float2* v_s = reinterpret_cast<const float2*>(st + B::vec_bytes) + (size_t)p * NX;
    const float2* p_s = reinterpret_cast<const float2*>(st + 2 * B::vec_bytes) + (size_t)p * NX;
    const float* f_s = reinterpret_cast<const float*>(st + 3 * B::vec_bytes) + (size_t)p * NX;
    const bool fb = s_fb[s] != 0;
    const float* f = slot_f(a.sel, slot);
    const size_t voff = (size_t)slot * a.vstride + (size_t)row * NX;
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
    if (valid && t < R2) {
      float fa = 1.f, fbb = 0.f, al_re = 0.f, al_im = 0.f, om_re = 0.f, om_im = 0.f;
      bool first = false;
      if (a.mode == FX_BICG_P) {
        const SlotDev& sd = a.sel.slots[slot];
        first = sd.first != 0;
        fa = sd.beta_f.x; fbb = sd.beta_f.y;
        om_re = sd.omega_f.x; om_im = sd.omega_f.y;
      } else if (a.mode == FX_BICG_S) {
        const SlotDev& sd = a.sel.slots[slot];
        al_re = sd.alpha_f.x; al_im = sd.alpha_f.y;
      }
#pragma unroll
      for (int n1 = 0; n1 < R1 / 2; ++n1) {
        const int x = R2 * n1 + t;
        if (!LS_IN_BOUNDS(x < NX && p < PC, BS_FXB_SMEM) ||
            !LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)row * NX + x, (size_t)a.rows * NX, a.vstride),
                          BS_FX_VEC))
          continue;
        float2 val = r_s[x];
        if (a.mode == FX_BICG_P) {
          if (!first) {
            // p = r + beta (p - omega v)
            const float2 d = csub(p_s[x], cmul(make_float2(om_re, om_im), v_s[x]));
            val = cadd(val, cmul(make_float2(fa, fbb), d));
          }
          a.vp[voff + x] = val;
        } else if (a.mode == FX_BICG_S) {
          // s = r - alpha v
          val = csub(val, cmul(make_float2(al_re, al_im), v_s[x]));
          a.vs[voff + x] = val;
        }
        if (a.mode != FX_COPY) val = cscale(val, fb ? f_s[x] : __ldg(f + (size_t)row * NX + x));
        v[n1] = val;
      }
    }
    float2* S = S0 + (size_t)p * R1 * G::SROW;
    if (t < R2) {
      Dft<R1, -1, R1 / 2, R1>::run(v);
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], twr[k1]);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) S[k1 * G::SROW + t] = v[k1];
    }
    __syncthreads();
    // every thread has read its inputs from stage s: refill it with the item NSTG ahead
    if (tid == 0 && m + NSTG < nmine) issue(m + NSTG, s);
    if (valid && t < R1) {
      float2 u[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) u[n2] = S[t * G::SROW + n2];
      Dft<R2, -1>::run(u);
      float2* d = a.dst + (size_t)slot * a.dst_stride + (size_t)row * L;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2)
        if (LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)row * L + t + R1 * k2, (size_t)a.rows * L,
                                      a.dst_stride), BS_FX_DST))
          d[t + R1 * k2] = u[k2];
    }
    __syncthreads();   // the exchange area is free for the next item
  }
  (void)NT;
}

// ------------------------------------------------------------------------- FY / IY
// Pencils along a strided axis; tile = 16 consecutive entries of the contiguous axis.
// P = 16 or 32 pencils per CTA (P 8-byte entries of a row: 128 or 256 contiguous bytes per load).
// CTAs of 257-384 threads (24 threads per pencil at the 288/384-point lengths) run as k_strided3, which
// asks for three resident per SM: FY at 192^3 ran at 5.5 TB/s with two (70 registers) and 6.5 TB/s
// with three; the other sizes keep the compiler's own register choice (k_strided).
template <int L, int DIR, int P>
__device__ __forceinline__ void strided_body(const StridedParams& a) {
  using G = Geo<L>;
  constexpr int R1 = G::R1, R2 = G::R2;
  extern __shared__ float2 sm[];
  const int slot = blockIdx.y;
  if (!LS_IN_BOUNDS(slot < a.sel.nslots, BS_SLOT)) return;
  if (!slot_runs(a.sel, slot)) return;
  count_run(a.sel);
  const int p = threadIdx.x, t = threadIdx.y;
  const int tiles_c = (a.ncont + P - 1) / P;
  const int plane = blockIdx.x / tiles_c;
  const int c = (blockIdx.x % tiles_c) * P + p;
  const bool valid = c < a.ncont;
  const float2* src = a.src + (size_t)slot * a.src_stride + (size_t)plane * a.src_plane + c;
  // debug build: a slot's extent in the source (FY reads L/2 rows of a plane, IY all L) and the
  // destination (FY writes L rows, IY the out_m rows of its window)
  const size_t src_ext = (size_t)(a.planes - 1) * a.src_plane + (size_t)(DIR < 0 ? L / 2 : L) * a.ncont;
  const size_t dst_ext = (size_t)(a.planes - 1) * a.dst_plane + (size_t)(DIR < 0 ? L : a.out_m) * a.ncont;
  (void)src_ext; (void)dst_ext;
  float2 v[R1];
#pragma unroll
  for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
  if (valid && t < R2) {
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int y = R2 * n1 + t;
      if ((DIR < 0 ? (n1 < R1 / 2) : true) &&
          LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)plane * a.src_plane + (size_t)y * a.ncont + c,
                                    src_ext, a.src_stride), BS_ST_SRC))
        v[n1] = __ldg(src + (size_t)y * a.ncont);
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
    for (int k1 = 0; k1 < R1; ++k1)
      if (LS_IN_BOUNDS((k1 * R2 + t) * P + p < L * P, BS_ST_SMEM)) sm[(k1 * R2 + t) * P + p] = v[k1];
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
      for (int k2 = 0; k2 < R2; ++k2)
        if (LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots,
                                      (size_t)plane * a.dst_plane + (size_t)(t + R1 * k2) * a.ncont + c,
                                      dst_ext, a.dst_stride), BS_ST_DST))
          dst[(size_t)(t + R1 * k2) * a.ncont] = u[k2];
    } else {
#pragma unroll
      for (int k2 = 0; k2 < R2 / 2; ++k2) {
        const int y = t + R1 * k2;
        const int yo = y - a.out_o;
        if (yo >= 0 && yo < a.out_m &&
            LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)plane * a.dst_plane + (size_t)yo * a.ncont + c,
                                      dst_ext, a.dst_stride), BS_ST_DST))
          dst[(size_t)yo * a.ncont] = u[k2];
      }
    }
  }
}

template <int L, int DIR, int P>
__global__ void __launch_bounds__(Geo<L>::T * P) k_strided(const StridedParams a) { strided_body<L, DIR, P>(a); }
template <int L, int DIR, int P>
__global__ void __launch_bounds__(Geo<L>::T * P, 3) k_strided3(const StridedParams a) { strided_body<L, DIR, P>(a); }
template <int L, int P> struct StridedThree { static constexpr bool on = Geo<L>::T * P > 256 && Geo<L>::T * P <= 384; };

// ------------------------------------------------------------------------- IX
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// Five resident CTAs of 256 threads, six of 192 (24 or 12 threads per row): IX at 192^3 ran at 5.07
// TB/s with five and 5.70 with six, at 144^3 4.32 and 4.89; at 128^3 six cost 15%.
template <int L>
__global__ void __launch_bounds__(Geo<L>::T * Geo<L>::PC, Geo<L>::T * Geo<L>::PC <= 192 ? 6 : 5) k_ix(IxParams a) {
  using G = Geo<L>;
  constexpr int R1 = G::R1, R2 = G::R2;
  extern __shared__ float2 sm[];
  const int slot = blockIdx.y;
  if (!LS_IN_BOUNDS(slot < a.sel.nslots, BS_SLOT)) return;
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
    for (int n1 = 0; n1 < R1; ++n1)
      if (LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)row * L + R2 * n1 + t, (size_t)a.rows * L,
                                    a.src_stride), BS_IX_SRC))
        v[n1] = __ldg(s + R2 * n1 + t);
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
      if (!LS_IN_BOUNDS(a.mode == IX_STORE ||
                            slot_elem_ok(slot, a.sel.nslots, (size_t)row * nx + x, (size_t)a.rows * nx, a.vstride),
                        BS_IX_VEC))
        continue;
      switch (a.mode) {
        case IX_STORE: {
          const int xo = x - a.out_o;
          if (xo >= 0 && xo < a.out_m &&
              LS_IN_BOUNDS(slot_elem_ok(slot, a.sel.nslots, (size_t)row * a.out_m + xo, (size_t)a.rows * a.out_m,
                                        a.vstride), BS_IX_VEC))
            a.out0[(size_t)slot * a.vstride + (size_t)row * a.out_m + xo] = g;
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
  if (a.mode >= IX_BICG_V && LS_IN_BOUNDS(a.maxparts == 0 || (int)gridDim.x <= a.maxparts, BS_IX_PART)) {
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
  int zalt_ok;  // a second split of the TMA-staged z pass exists (autotuned)
  int zdyn_ok;  // the dynamically scheduled TMA-staged z pass exists for this length
  int zauto_small, zauto_large;   // z-pass form of untuned plans up to kZSmallBatch views and above (ZAuto)
  int zr1b, zr2b;
};

template <int L>
struct PassImpl {
  using G = Geo<L>;
  static bool aligned16(const void* q) { return q == nullptr || (reinterpret_cast<uintptr_t>(q) & 15) == 0; }
  static void fx(const FxParams& a, int nslots, cudaStream_t st) {
    if constexpr (FXB<L>::ok) {
      // the BiCGStab modes only (three or two staged vectors per row block; with one, the plain
      // kernel's six CTAs per SM keep more loads in flight)
      if (a.bulk && a.mode >= FX_BICG_P && a.sms > 0 && a.err && aligned16(a.src) && aligned16(a.vv) &&
          aligned16(a.vp) && a.vstride % 2 == 0) {
        const int nrb = (a.rows + G::PC - 1) / G::PC;
        FxParams b = a;
        b.sel.nslots = nslots;   // the kernel builds its list of active views from the selector
        k_fxb<L><<<std::min(nrb * nslots, a.sms), dim3(G::T, G::PC), FXB<L>::smem, st>>>(b);
        return;
      }
    }
    const unsigned rbs = (unsigned)((a.rows + G::PC - 1) / G::PC);
    dim3 blk(G::T, G::PC), grd = a.views_fastest ? dim3(nslots, rbs) : dim3(rbs, nslots);
    FxParams b = a;
    b.sel.nslots = nslots;
    k_fx<L><<<grd, blk, G::smem_contig, st>>>(b);
  }
  static void ix(const IxParams& a0, int nslots, cudaStream_t st) {
    IxParams a = a0;
    a.sel.nslots = nslots;
    dim3 blk(G::T, G::PC), grd((a.rows + G::PC - 1) / G::PC, nslots);
    k_ix<L><<<grd, blk, G::smem_contig, st>>>(a);
  }
  template <int DIR>
  static void strided(const StridedParams& a0, int nslots, cudaStream_t st) {
    StridedParams a = a0;
    a.sel.nslots = nslots;
    if (a.wide && G::T * 32 <= 1024) {
      constexpr int W = G::T * 32 <= 1024 ? 32 : 16;
      dim3 blk(W, G::T), grd(((a.ncont + W - 1) / W) * a.planes, nslots);
      if constexpr (StridedThree<L, W>::on)
        k_strided3<L, DIR, W><<<grd, blk, (size_t)L * W * sizeof(float2), st>>>(a);
      else
        k_strided<L, DIR, W><<<grd, blk, (size_t)L * W * sizeof(float2), st>>>(a);
    } else {
      dim3 blk(G::PS, G::T), grd(((a.ncont + G::PS - 1) / G::PS) * a.planes, nslots);
      if constexpr (StridedThree<L, G::PS>::on)
        k_strided3<L, DIR, G::PS><<<grd, blk, G::smem_strided, st>>>(a);
      else
        k_strided<L, DIR, G::PS><<<grd, blk, G::smem_strided, st>>>(a);
    }
  }
  static void fy(const StridedParams& a, int nslots, cudaStream_t st) { strided<-1>(a, nslots, st); }
  static void iy(const StridedParams& a, int nslots, cudaStream_t st) { strided<+1>(a, nslots, st); }
  static void z(const ZParams& a0, int nslots, cudaStream_t st) {
    ZParams a = a0;
    a.sel.nslots = nslots;
    if constexpr (ZW<L, true>::ok) {
      if (a.alt && a.use_tma && (2 * a.nx) % ZW<L, true>::P == 0 && a.nz <= 256) {
        launch_zw<true>(a, st);
        return;
      }
    }
    if constexpr (ZWD<L>::ok) {
      if (a.persist == 2 && a.gmap_ok && a.ctr && a.sms > 0 && a.use_tma && (2 * a.nx) % ZWD<L>::P == 0 &&
          a.nz <= 255) {
        const int ntiles = (2 * a.nx / ZWD<L>::P) * (2 * a.ny);
        cudaMemsetAsync(a.ctr, 0, sizeof(unsigned), st);
        k_zwd<L><<<std::min(ntiles, a.sms * ZWD<L>::MINB), ZWD<L>::NT, ZWD<L>::smem, st>>>(a);
        return;
      }
    }
    if constexpr (ZW<L>::ok) {
      if (a.use_tma && (2 * a.nx) % ZW<L>::P == 0 && a.nz <= 256) {
        launch_zw<false>(a, st);
        return;
      }
    } else if constexpr (ZG<L>::ok) {
      if (a.use_tma && (2 * a.nx) % ZG<L>::P == 0 && a.nz <= 256) {
        const int ntiles = (2 * a.nx / ZG<L>::P) * (2 * a.ny);
        if (a.persist && a.sms > 0)
          k_zg<L, true><<<std::min(ntiles, a.sms * ZG<L>::MINB), ZG<L>::NT, ZG<L>::smem, st>>>(a);
        else
          k_zg<L, false><<<ntiles, ZG<L>::NT, ZG<L>::smem, st>>>(a);
        return;
      }
    }
    dim3 blk(G::PS, G::T), grd(((2 * a.nx + G::PS - 1) / G::PS) * (2 * a.ny));
    k_z<L><<<grd, blk, G::smem_z, st>>>(a);
  }
  // persistent where the Green values live in registers: one wave of resident CTAs
  template <bool ALT>
  static void launch_zw(const ZParams& a, cudaStream_t st) {
    using W = ZW<L, ALT>;
    const int ntiles = (2 * a.nx / W::P) * (2 * a.ny);
    if constexpr (W::GREG) {
      if (a.persist == 1 && a.sms > 0) {
        k_zw<L, ALT, true><<<std::min(ntiles, a.sms * W::MINB), W::NT, W::smem, st>>>(a);
        return;
      }
    }
    k_zw<L, ALT, false><<<ntiles, W::NT, W::smem, st>>>(a);
  }
  template <bool ALT>
  static cudaError_t setup_zw() {
    using W = ZW<L, ALT>;
    cudaError_t e = cudaFuncSetAttribute(k_zw<L, ALT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::smem);
    if constexpr (W::GREG)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_zw<L, ALT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::smem);
    return e;
  }
  template <int DIR, int P>
  static cudaError_t set_strided_smem(int bytes) {
    if constexpr (StridedThree<L, P>::on)
      return cudaFuncSetAttribute(k_strided3<L, DIR, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    else
      return cudaFuncSetAttribute(k_strided<L, DIR, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  static cudaError_t setup() {
    cudaError_t e = cudaSuccess;
    {
      e = cudaFuncSetAttribute(k_fx<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_contig);
      if constexpr (FXB<L>::ok)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fxb<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FXB<L>::smem);
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ix<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_contig);
      if (e == cudaSuccess) e = set_strided_smem<-1, G::PS>((int)G::smem_strided);
      if (e == cudaSuccess) e = set_strided_smem<+1, G::PS>((int)G::smem_strided);
      if constexpr (G::T * 32 <= 1024) {
        constexpr int sw = (int)(L * 32 * sizeof(float2));
        if (e == cudaSuccess) e = set_strided_smem<-1, 32>(sw);
        if (e == cudaSuccess) e = set_strided_smem<+1, 32>(sw);
      }
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k_z<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_z);
      if constexpr (ZW<L>::ok)
        if (e == cudaSuccess) e = setup_zw<false>();
      if constexpr (ZW<L, true>::ok)
        if (e == cudaSuccess) e = setup_zw<true>();
      if constexpr (ZWD<L>::ok)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_zwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZWD<L>::smem);
      if constexpr (ZG<L>::ok) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_zg<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZG<L>::smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_zg<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ZG<L>::smem);
      }
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
    t.zalt_ok = ZW<L, true>::ok ? 1 : 0;
    t.zdyn_ok = ZWD<L>::ok ? 1 : 0;
    t.zauto_small = ZAuto<L>::small;
    t.zauto_large = ZAuto<L>::large;
    t.zr1b = ZRadixAlt<L>::R1;
    t.zr2b = ZRadixAlt<L>::R2;
    return t;
  }
};

// Defined in one translation unit per length (passes_L*.cu).
#define LS_DECLARE_LENGTH(L) \
  PassLaunch pass_table_##L(); \
  cudaError_t pass_setup_##L(); \
  unsigned bounds_site_##L(bool clear);
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
  cudaError_t pass_setup_##L() { return PassImpl<L>::setup(); } \
  LS_BOUNDS_READER(L)

}  // namespace lsgpu

// The z pass of the Green convolution: zero-padded FFT along z, Green multiply, inverse FFT, crop
// (the third of the five passes described in passes.cuh).  Two kernels: k_z stages each view with
// cp.async and exchanges through the whole CTA; k_zw is the TMA-staged, warp-specialised one.
#pragma once

#include "pass_common.cuh"

namespace lsgpu {

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
    if (!LS_IN_BOUNDS(slot < a.sel.nslots, BS_SLOT)) return;
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
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
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
template <> struct ZRadix<384> { static constexpr int R1 = 32, R2 = 12; };
template <> struct ZRadix<192> { static constexpr int R1 = 24, R2 = 8; };
// A second split of the same length for the autotuner: the transposed one where R1 != R2, else
// (2 R1, R2 / 2) (both factors even, thread count max(R1, R2) dividing 32 where it is usable)
template <int L> struct ZRadixAlt {
  static constexpr int R1 = ZRadix<L>::R1 != ZRadix<L>::R2 ? ZRadix<L>::R2 : 2 * ZRadix<L>::R1;
  static constexpr int R2 = ZRadix<L>::R1 != ZRadix<L>::R2 ? ZRadix<L>::R1 : ZRadix<L>::R2 / 2;
};
template <int L, bool ALT> struct ZSplit { static constexpr int R1 = ZRadix<L>::R1, R2 = ZRadix<L>::R2; };
template <int L> struct ZSplit<L, true> { static constexpr int R1 = ZRadixAlt<L>::R1, R2 = ZRadixAlt<L>::R2; };

// Threads per column of the TMA-staged z pass: max(R1, R2), except at L = 384, whose 32 x 12 split
// runs on 16 threads per column (two columns per warp, two stage-2 sub-transforms per thread) rather
// than 32 with 20 idle lanes in the 32-point stages.
template <int L, bool ALT> struct ZThreads { static constexpr int T = imax(ZSplit<L, ALT>::R1, ZSplit<L, ALT>::R2); };
template <> struct ZThreads<384, false> { static constexpr int T = 16; };
template <> struct ZThreads<128, false> { static constexpr int T = 8; };
template <> struct ZThreads<96, false> { static constexpr int T = 8; };
template <> struct ZThreads<192, false> { static constexpr int T = 8; };

// z-pass form untuned plans run (0: one CTA per tile, 1: persistent with tiles round-robin, 2: the
// dynamically scheduled form), for launches of at most kZSmallBatch views and above, as measured on
// GB300 with ls_matvec_batch (z pass GB/s): 128-point (64^3 grids) the round-robin persistent form is
// fastest from 1 to 60 views; 96-, 192- and 384-point (48^3, 96^3, 192^3) the dynamic form from 8 to 60
// views (and within 10% of the best at one view); 256-point (128^3) the dynamic form up to about 24
// views and one CTA per tile at 30-60.  A form a length does not have falls back to one CTA per tile.
constexpr int kZSmallBatch = 24;
template <int L> struct ZAuto { static constexpr int small = 2, large = 0; };
template <> struct ZAuto<96> { static constexpr int small = 2, large = 2; };
template <> struct ZAuto<128> { static constexpr int small = 1, large = 1; };
template <> struct ZAuto<192> { static constexpr int small = 2, large = 2; };
template <> struct ZAuto<384> { static constexpr int small = 2, large = 2; };

template <int L, bool ALT = false>
struct ZW {
  static constexpr int R1 = ZSplit<L, ALT>::R1, R2 = ZSplit<L, ALT>::R2;
  static constexpr int T = ZThreads<L, ALT>::T;
  static constexpr int S2 = (R1 + T - 1) / T;   // stage-2 sub-transforms per thread (k1 = t + T s)
  static constexpr bool ok = (32 % T) == 0 && R1 % 2 == 0 && R2 % 2 == 0 && R1 >= 2 && R2 >= 2 && T >= R2 &&
                             (S2 == 1 || R1 % T == 0);
  static constexpr int CPW = ok ? 32 / T : 1;   // whole columns per warp (lane = t * CPW + column)
  static constexpr int P = 16;                  // columns per CTA: one 128-byte TMA row
  static constexpr int NW = P / CPW;             // compute warps
  static constexpr int NT = 32 * NW + 32;        // + one producer warp (TMA loads and stores)
  static constexpr int NZ = L / 2;
  static constexpr int MINB0 = NT >= 512 ? 1 : NT >= 256 ? 2 : 512 / NT;
  // exchange pitch per column (in float2) congruent to 16/CPW mod 16: the CPW columns of a half-warp
  // then fall on disjoint banks; the Ghat rows [kz][P + CPW] are conflict-free for the same reason
  static constexpr int pitch(int n) { return n + (((16 / CPW) - n % 16) % 16 + 16) % 16; }
  static constexpr int GR = P + CPW;                                          // Ghat row [kz][GR], kz folded to [0, NZ]
  // exchange rows of R + 2 entries: a thread reads its row with 16-byte loads (two entries each)
  static constexpr int XP = pitch(imax(R1 * (R2 + 2), R2 * (R1 + 2)));
  static constexpr int TWA = R1 + 2, TWB = R2 + 2;                            // twiddle rows (16-byte aligned)
  static constexpr int NS = 4;                                                // view buffers (TMA pipeline depth)
  // each thread's Green values stay in registers across a tile's views where they fit (S2 R2 <= 24); the
  // Green tile is then dead once they are loaded and the exchange area reuses it, and the kernel can
  // also run persistent (Green values loaded per tile from the octant)
  static constexpr bool GREG = S2 * R2 <= 24;
  static_assert(GREG || S2 == 1, "stage-2 sub-transforms per thread need register-resident Green values");
  static constexpr size_t r16(size_t b) { return (b + 15) / 16 * 16; }       // every region 16-byte aligned
  static constexpr size_t stage_bytes = (size_t)NZ * P * sizeof(float2);
  static constexpr size_t g_bytes = r16((size_t)(NZ + 1) * GR * sizeof(float2));
  static constexpr size_t x_bytes = r16((size_t)P * XP * sizeof(float2));
  static constexpr size_t off_g = NS * stage_bytes;
  static constexpr size_t off_x = GREG ? off_g : off_g + g_bytes;   // with GREG the exchange overlays the Green tile
  static constexpr size_t off_twa = off_x + (GREG ? (g_bytes > x_bytes ? g_bytes : x_bytes) : x_bytes);
  static constexpr size_t off_twb = off_twa + r16((size_t)R2 * TWA * sizeof(float2));
  static constexpr size_t off_bar = off_twb + r16((size_t)R1 * TWB * sizeof(float2));
  static constexpr int NBAR = 2 * NS + 1;                                     // full[NS], done[NS], never
  static constexpr size_t smem = off_bar + NBAR * sizeof(uint64_t) + 1024;    // + room to align the base to 1024
  // resident CTAs asked of the launch: by threads, and no more than fit one SM's shared memory (with the
  // kernel's static arrays and the per-CTA reserve)
  static constexpr size_t cta_smem = smem + kMaxLaunchSlots * sizeof(int) + 32 * sizeof(int) + 16 + 1024;
  static constexpr int MINB = MINB0 * cta_smem <= 228 * 1024 ? MINB0 : (int)(228 * 1024 / cta_smem) > 0 ? (int)(228 * 1024 / cta_smem) : 1;
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

// Green values of one thread for one (ky, 16-column kx) tile, read from the stored octant: kz = t + R1 k2,
// folded into [0, L/2] (Ghat is even in every axis); column kx = kx0 + c folded into [0, nx].
template <int L, int R1, int R2>
__device__ __forceinline__ void load_green(float2 (&g)[R2], const ZParams& a, int ky, int kx, int t) {
  const int fy = ky <= a.ny ? ky : 2 * a.ny - ky;
  const int fx = kx <= a.nx ? kx : 2 * a.nx - kx;
  const float2* col = a.gocta + (size_t)fy * (a.nx + 1) + fx;
  const size_t plane = (size_t)(a.ny + 1) * (a.nx + 1);
#pragma unroll
  for (int k2 = 0; k2 < R2; ++k2) {
    const int kz = k2 < R2 / 2 ? t + R1 * k2 : L - R1 * k2 - t;
    g[k2] = LS_IN_BOUNDS(kz >= 0 && kz <= a.nz && fy >= 0 && fy <= a.ny && fx >= 0 && fx <= a.nx, BS_Z_GREEN)
                ? __ldg(col + (size_t)kz * plane)
                : make_float2(0.f, 0.f);
  }
}

// One view of one tile of the TMA-staged z pass, in place in its view buffer sb (TMA layout with the
// 128-byte swizzle): forward stage 1, warp-local exchange, forward stage 2, Green multiply (conjugate
// Green for the adjoint), inverse stage 1 (transposed split), exchange, inverse stage 2 with the crop.
// W is the shared-memory layout; the thread owns column c as sub-transform index t (lane = t CPW +
// column); g holds its Green values where W::GREG, else gc points at its column of the shared Green
// tile.  adj_of() gives the view's adjoint flag; after_green() runs right after the Green multiply.
template <class W, int L, class AdjF, class AfterF>
__device__ __forceinline__ void zw_view(unsigned char* sb, float2* xc, const float2* twa, const float2* twb,
                                        float2 (&g)[W::S2][W::GREG ? W::R2 : 1], const float2* gc, int t, int c,
                                        unsigned rb, AdjF&& adj_of, AfterF&& after_green) {
  constexpr int R1 = W::R1, R2 = W::R2, T = W::T, S2 = W::S2;
  constexpr bool GREG = W::GREG;
  if (R2 == T || t < R2) {
    // forward stage 1: inputs z = R2 n1 + t, n1 < R1/2 (z < nz)
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int n1 = 0; n1 < R1 / 2; ++n1) {
      const unsigned off = R2 % 8 == 0 ? rb + R2 * n1 * 128 : swz128(R2 * n1 + t, c);
      if (LS_IN_BOUNDS(off + sizeof(float2) <= W::stage_bytes, BS_Z_SMEM))
        v[n1] = *reinterpret_cast<const float2*>(sb + off);
    }
    Dft<R1, -1, R1 / 2, R1>::run(v);
    const float4* tw4 = reinterpret_cast<const float4*>(twa + t * W::TWA);
#pragma unroll
    for (int k = 0; k < R1 / 2; ++k) {
      const float4 w = tw4[k];
      if (k > 0) v[2 * k] = cmul(v[2 * k], make_float2(w.x, w.y));
      v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w.z, w.w));
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1)
      if (LS_IN_BOUNDS(c * W::XP + k1 * (R2 + 2) + t < W::P * W::XP, BS_Z_SMEM)) xc[k1 * (R2 + 2) + t] = v[k1];
  }
  __syncwarp();
  // forward stage 2, Green multiply and inverse stage 1 of sub-transforms k1 = t + T s; every row is
  // read before any thread writes the second exchange over the first
  float2 u[S2][R2];
#pragma unroll
  for (int s2 = 0; s2 < S2; ++s2) {
    const int k1 = t + T * s2;
    if (R1 == T * S2 || k1 < R1) {
#pragma unroll
      for (int q = 0; q < R2 / 2; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(xc + k1 * (R2 + 2) + 2 * q);
        u[s2][2 * q] = make_float2(x.x, x.y);
        u[s2][2 * q + 1] = make_float2(x.z, x.w);
      }
      Dft<R2, -1>::run(u[s2]);
      // the adjoint flag is read where it is used (not held across the stages)
      const bool adj = adj_of();
      if constexpr (GREG) {
        if (adj) {
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) u[s2][k2] = cmulc(u[s2][k2], g[s2][k2]);
        } else {
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) u[s2][k2] = cmul(u[s2][k2], g[s2][k2]);
        }
        if constexpr (S2 == 1) after_green();
      } else if (adj) {
        green_mul<true, R1, R2, L, W::GR>(u[s2], gc, k1);
      } else {
        green_mul<false, R1, R2, L, W::GR>(u[s2], gc, k1);
      }
      // inverse stage 1 (transposed split): DFT_R2 over k2, twiddle exp(+2 pi i j1 k1 / L)
      Dft<R2, +1>::run(u[s2]);
      const float4* tw4 = reinterpret_cast<const float4*>(twb + k1 * W::TWB);
#pragma unroll
      for (int k = 0; k < R2 / 2; ++k) {
        const float4 w = tw4[k];
        if (k > 0) u[s2][2 * k] = cmulc(u[s2][2 * k], make_float2(w.x, w.y));
        u[s2][2 * k + 1] = cmulc(u[s2][2 * k + 1], make_float2(w.z, w.w));
      }
    }
  }
  if constexpr (S2 > 1) after_green();
  __syncwarp();
#pragma unroll
  for (int s2 = 0; s2 < S2; ++s2) {
    const int k1 = t + T * s2;
    if (R1 == T * S2 || k1 < R1) {
#pragma unroll
      for (int j1 = 0; j1 < R2; ++j1) xc[j1 * (R1 + 2) + k1] = u[s2][j1];
    }
  }
  __syncwarp();
  if (R2 == T || t < R2) {
    float2 w[R1];
#pragma unroll
    for (int q = 0; q < R1 / 2; ++q) {
      const float4 x = *reinterpret_cast<const float4*>(xc + t * (R1 + 2) + 2 * q);
      w[2 * q] = make_float2(x.x, x.y);
      w[2 * q + 1] = make_float2(x.z, x.w);
    }
    Dft<R1, +1, R1, R1 / 2>::run(w);
    // outputs z = t + R2 j2 (j2 < R1/2: z < nz), in place
#pragma unroll
    for (int j2 = 0; j2 < R1 / 2; ++j2) {
      const unsigned off = R2 % 8 == 0 ? rb + R2 * j2 * 128 : swz128(t + R2 * j2, c);
      if (LS_IN_BOUNDS(off + sizeof(float2) <= W::stage_bytes, BS_Z_SMEM))
        *reinterpret_cast<float2*>(sb + off) = w[j2];
    }
  }
}

// One CTA per tile (PERSIST = false), or persistent (PERSIST = true, Green values in registers only):
// each CTA owns the tiles blockIdx.x, blockIdx.x + gridDim.x, ... and streams the (tile, view) items
// of all of them through its view buffers, so the per-CTA set-up (barriers, the active-view list,
// twiddles) is paid once per CTA rather than once per tile; each thread loads its next tile's Green
// values from the octant right after its last Green multiply of the current tile, and they land
// while the inverse transform of that view and the forward transform of the next item run.  Which
// form is faster depends on the views per launch (the autotuner times both).
template <int L, bool ALT, bool PERSIST>
__global__ void __launch_bounds__(ZW<L, ALT>::NT, ZW<L, ALT>::MINB) k_zw(const __grid_constant__ ZParams a) {
  using W = ZW<L, ALT>;
  static_assert(!PERSIST || W::GREG, "the persistent z pass keeps its Green values in registers");
  constexpr int R1 = W::R1, R2 = W::R2, P = W::P, NZ = W::NZ, CPW = W::CPW, T = W::T, NW = W::NW;
  static_assert(W::ok, "k_zw needs T | 32");
  static_assert(R1 % 2 == 0 && R2 % 2 == 0 && W::XP % 2 == 0, "16-byte exchange reads need even rows");
  constexpr bool GREG = W::GREG;
  extern __shared__ __align__(16) unsigned char zw_raw[];
  const unsigned raw = smem_addr(zw_raw);
  unsigned char* base = zw_raw + (((raw + 1023u) & ~1023u) - raw);
  float2* stage = reinterpret_cast<float2*>(base);
  float2* gs = reinterpret_cast<float2*>(base + W::off_g);
  float2* xs = reinterpret_cast<float2*>(base + W::off_x);
  float2* twa = reinterpret_cast<float2*>(base + W::off_twa);
  float2* twb = reinterpret_cast<float2*>(base + W::off_twb);
  constexpr int NS = W::NS;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + W::off_bar);   // [NS]: an item's tile has landed
  uint64_t* done = full + NS;                                         // [NS]: the compute warps are done with it
  uint64_t* never = done + NS;                                        // no thread arrives on it (stall test)
  __shared__ int s_list[kMaxLaunchSlots];
  __shared__ int s_ws[32];
  __shared__ int s_abort;
  const int nact = build_active(a.sel, s_list, s_ws);
  if (nact == 0) return;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles_c = 2 * a.nx / P;
  const int ntiles = tiles_c * 2 * a.ny;
  // tiles of this CTA: blockIdx.x + k gridDim.x, k < ntl; items i = k nact + view
  const int ntl = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int nitems = ntl * nact;
  const bool producer = warp == NW;
  // per-view wait limit (read from the parameter space where it is used, not held in a register)
#define LS_ZW_LIMIT (a.wait_ns ? a.wait_ns : 1000000000ull)
  // TMA coordinates of the item (view position iv, tile number kt of this CTA): (2 kx0 floats, ky, 0, slot)
  auto item_load = [&](int iv, int kt, int buf) {
    const int j = (int)blockIdx.x + kt * (int)gridDim.x;
    if (!LS_IN_BOUNDS(j < ntiles && iv < nact && active_slot(s_list[iv]) < a.sel.nslots, BS_Z_TILE)) {
      mbar_arrive(&full[buf]);   // nothing copied: the buffer's phase completes at once
      return;
    }
    mbar_expect_tx(&full[buf], (unsigned)W::stage_bytes);
    tma_load_4d(stage + (size_t)buf * NZ * P, &a.tmap, &full[buf], 2 * (j % tiles_c) * P, j / tiles_c, 0,
                a.slot0 + active_slot(s_list[iv]));
  };
  if (producer && lane == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&done[k], NW);
    }
    mbar_init(never, 1);
    mbar_init_fence();
    for (int k = 0; k < NS && k < nitems; ++k) item_load(k % nact, k / nact, k);
  }
  if constexpr (!PERSIST) {
    // one tile per CTA (the launch has one CTA per tile): its Green tile, kz folded into [0, NZ]
    const int ky = blockIdx.x / tiles_c, kx0 = (blockIdx.x % tiles_c) * P;
    const int fy = ky <= a.ny ? ky : 2 * a.ny - ky;
    // every load of the gather is issued before any store (one L2 round trip, not one per element)
    constexpr int GN = (NZ + 1) * P, GIT = (GN + W::NT - 1) / W::NT;
    float2 gv[GIT];
#pragma unroll
    for (int r = 0; r < GIT; ++r) {
      const int i = tid + r * W::NT;
      const int kz = i / P, cc = i % P, kx = kx0 + cc;
      const int fx = kx <= a.nx ? kx : 2 * a.nx - kx;
      if (i < GN && LS_IN_BOUNDS(kz <= a.nz && fy >= 0 && fy <= a.ny && fx >= 0 && fx <= a.nx, BS_Z_GREEN))
        gv[r] = __ldg(a.gocta + ((size_t)kz * (a.ny + 1) + fy) * (a.nx + 1) + fx);
    }
#pragma unroll
    for (int r = 0; r < GIT; ++r) {
      const int i = tid + r * W::NT;
      if (i < GN) gs[(i / P) * W::GR + i % P] = gv[r];
    }
  }
  for (int i = tid; i < R1 * R2; i += W::NT) {
    twa[(i / R1) * W::TWA + i % R1] = __ldg(a.zwa + i);
    twb[(i / R2) * W::TWB + i % R2] = __ldg(a.zwb + i);
  }
  __syncthreads();
  if (producer) {
    // producer: after the compute warps release an item's buffer, store it and refill it with the
    // item NS ahead
    if (lane != 0) return;
    // (view position, tile number) of the item being stored and of the one NS ahead, kept by counting
    int sv = 0, skt = 0, lv = NS % nact, lkt = NS / nact;
    int i = 0;
    for (; i < nitems; ++i) {
      const int buf = i % NS;
      if (!mbar_wait_abort(&done[buf], (unsigned)(i / NS) & 1u, &s_abort, LS_ZW_LIMIT)) break;
      const int j = (int)blockIdx.x + skt * (int)gridDim.x;
      if (LS_IN_BOUNDS(j < ntiles && active_slot(s_list[sv]) < a.sel.nslots, BS_Z_TILE))
        tma_store_4d(&a.tmap, stage + (size_t)buf * NZ * P, 2 * (j % tiles_c) * P, j / tiles_c, 0,
                     a.slot0 + active_slot(s_list[sv]));
      bulk_commit();
      if (i + NS < nitems) {
        bulk_wait_read_all();   // the store has read the buffer
        item_load(lv, lkt, buf);
      }
      if (++sv == nact) { sv = 0; ++skt; }
      if (++lv == nact) { lv = 0; ++lkt; }
    }
    bulk_wait_read_all();
    if (i < nitems) {
      // gave up at item i: flag it, and give the loads still in flight into this CTA's buffers
      // (items i .. i + NS - 1, all issued) a bounded time to land (one second each, whatever
      // the per-view limit)
      atomicExch(a.err, 1);
      for (int k = i; k < i + NS && k < nitems; ++k) mbar_wait(&full[k % NS], (unsigned)(k / NS) & 1u);
    }
    return;
  }
  // compute warps: each owns CPW whole columns (lane = t * CPW + column)
  const int t = lane / CPW;
  const int c = warp * CPW + lane % CPW;
  constexpr int S2 = W::S2;
  float2* xc = xs + c * W::XP;
  const float2* gc = gs + c;
  // byte offset of (z = t + R2 j, c) in a tile: row base for j = 0, plus j R2 rows
  const unsigned rb = swz128(t, c);
  // this thread's Green values (kz = k1 + R1 k2 for its stage-2 sub-transforms k1 = t + T s, the same
  // for every view of a tile) in registers where they fit (S2 R2 <= 24); longer splits read them from
  // the shared tile for every view
  float2 g[S2][GREG ? R2 : 1];
  if constexpr (GREG) {
#pragma unroll
    for (int s2 = 0; s2 < S2; ++s2) {
      const int k1 = t + T * s2;
      const bool has = R1 == T * S2 || k1 < R1;
      if (PERSIST && has) {
        load_green<L, R1, R2>(g[s2], a, blockIdx.x / tiles_c, (blockIdx.x % tiles_c) * P + c, k1);
      } else if (!PERSIST) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
          g[s2][k2] = has ? (k2 < R2 / 2 ? gc[(k1 + R1 * k2) * W::GR] : gc[(L - R1 * k2 - k1) * W::GR])
                          : make_float2(0.f, 0.f);
      }
    }
    // the exchange area overlays the Green tile: every compute warp has its values before any writes
    if constexpr (!PERSIST) asm volatile("bar.sync 1, %0;\n" ::"r"(NW * 32) : "memory");
  }
  int iv = 0, kt = 0;   // view position and tile number of item i, kept by counting
#pragma unroll 1
  for (int i = 0; i < nitems; ++i) {
    const int buf = i % NS;
    const bool ok = (a.stall && i == 0) ? mbar_wait_abort(never, 0u, &s_abort, LS_ZW_LIMIT)
                                        : mbar_wait_abort(&full[buf], (unsigned)(i / NS) & 1u, &s_abort, LS_ZW_LIMIT);
    if (!__all_sync(0xffffffffu, ok)) break;
    if (i < nact) count_run(a.sel);   // each view once per launch (by the first tile of CTA 0)
    unsigned char* sb = reinterpret_cast<unsigned char*>(stage + (size_t)buf * NZ * P);
    zw_view<W, L>(
        sb, xc, twa, twb, g, gc, t, c, rb, [&] { return active_adj(s_list[iv]); },
        [&] {
          // last view of this tile: the next tile's Green values, in flight during the rest of this
          // view and the forward transform of the next item
          if constexpr (PERSIST && W::GREG) {
            if (iv == nact - 1 && i + 1 < nitems) {
              const int j = (int)blockIdx.x + (kt + 1) * (int)gridDim.x;
#pragma unroll
              for (int s2 = 0; s2 < S2; ++s2)
                if (R1 == T * S2 || t + T * s2 < R1)
                  load_green<L, R1, R2>(g[s2], a, j / tiles_c, (j % tiles_c) * P + c, t + T * s2);
            }
          }
        });
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[buf]);
    if (++iv == nact) { iv = 0; ++kt; }
  }
#undef LS_ZW_LIMIT
}

// ------------------------------------------------------------------------- Z (TMA-staged, dynamic)
// Dynamically scheduled persistent form of the TMA-staged z pass, for the splits whose Green values
// fit in registers.  One wave of CTAs takes work units from a counter in device memory; a unit is
// one tile with a contiguous chunk of the active views (chunks sized so that every CTA gets many
// units: the last units finish close together).  The producer warp loads each unit's Green tile
// with one TMA copy from the x-unfolded Green array (rows kz = 0..nz of 16 columns, 128-byte
// swizzle) into a single shared buffer -- the compute warps copy it into registers at the unit's
// first view, after which the next unit's tile may be loaded -- and streams the unit's views through
// NS view buffers as k_zw does.  An item's view position and unit start are passed to the compute
// warps in a shared ring written before the item's copy is issued; a negative entry ends the loop.
template <int L, int NSB>
struct ZWDL {
  using B = ZW<L, false>;
  static constexpr bool ok = B::ok && B::GREG && (L / 2) % 8 == 0 && L / 2 + 1 <= 256;
  static constexpr int R1 = B::R1, R2 = B::R2, T = B::T, S2 = B::S2, CPW = B::CPW, P = B::P, NW = B::NW, NT = B::NT;
  static constexpr int NZ = B::NZ, MINB = B::MINB;
  static constexpr int XP = B::XP, TWA = B::TWA, TWB = B::TWB, GR = B::GR;
  static constexpr bool GREG = true;
  static constexpr int NS = NSB;
  static constexpr size_t r16(size_t b) { return (b + 15) / 16 * 16; }
  static constexpr size_t stage_bytes = B::stage_bytes;                // NZ rows of 128 bytes
  static constexpr size_t gtile_bytes = (size_t)(NZ + 1) * 128;        // Green rows kz = 0..NZ
  static constexpr size_t off_g = NS * stage_bytes;                    // a multiple of 1024 (NZ % 8 == 0)
  static constexpr size_t off_x = off_g + (gtile_bytes + 1023) / 1024 * 1024;
  static constexpr size_t x_bytes = B::x_bytes;
  static constexpr size_t off_twa = off_x + x_bytes;
  static constexpr size_t off_twb = off_twa + r16((size_t)R2 * TWA * sizeof(float2));
  static constexpr size_t off_bar = off_twb + r16((size_t)R1 * TWB * sizeof(float2));
  static constexpr int NBAR = 2 * NS + 3;                                // full[NS], done[NS], gfull, gdone, never
  static constexpr size_t smem = off_bar + NBAR * sizeof(uint64_t) + 1024;
  // static shared memory of the kernel (active-view list, warp sums, flags, item ring) and the SM's share
  static constexpr size_t static_smem = kMaxLaunchSlots * sizeof(int) + 32 * sizeof(int) + 16 + NS * sizeof(int);
  static constexpr bool fits = (size_t)MINB * (smem + static_smem + 1024) <= 228 * 1024;
};
// four view buffers where the resident CTAs still fit the SM's shared memory, else three
template <int L>
struct ZWD : ZWDL<L, ZWDL<L, 4>::fits ? 4 : 3> {};

template <int L>
__global__ void __launch_bounds__(ZWD<L>::NT, ZWD<L>::MINB) k_zwd(const __grid_constant__ ZParams a) {
  using W = ZWD<L>;
  constexpr int R1 = W::R1, R2 = W::R2, P = W::P, NZ = W::NZ, CPW = W::CPW, T = W::T, NW = W::NW, NS = W::NS;
  static_assert(W::ok, "k_zwd needs a register-resident Green split");
  extern __shared__ __align__(16) unsigned char zd_raw[];
  const unsigned raw = smem_addr(zd_raw);
  unsigned char* base = zd_raw + (((raw + 1023u) & ~1023u) - raw);
  float2* stage = reinterpret_cast<float2*>(base);
  unsigned char* gsm = base + W::off_g;
  float2* xs = reinterpret_cast<float2*>(base + W::off_x);
  float2* twa = reinterpret_cast<float2*>(base + W::off_twa);
  float2* twb = reinterpret_cast<float2*>(base + W::off_twb);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + W::off_bar);   // [NS]: an item's tile has landed
  uint64_t* done = full + NS;                                         // [NS]: the compute warps are done with it
  uint64_t* gfull = done + NS;                                        // a unit's Green tile has landed
  uint64_t* gdone = gfull + 1;                                        // the compute warps hold it in registers
  uint64_t* never = gdone + 1;                                        // no thread arrives on it (stall test)
  __shared__ int s_list[kMaxLaunchSlots];
  __shared__ int s_ws[32];
  __shared__ int s_abort;
  __shared__ int s_item[NS];   // item entry: view position | unit start << 16 | tile 0 << 17; -1 ends
  const int nact = build_active(a.sel, s_list, s_ws);
  if (nact == 0) return;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles_c = 2 * a.nx / P;
  const int ntiles = tiles_c * 2 * a.ny;
  // views per unit: about 16 units per CTA where the views allow, at least NS views per unit
  int nch = (16 * (int)gridDim.x + ntiles - 1) / ntiles;
  nch = max(1, min(nch, nact / NS));
  const int chunk = (nact + nch - 1) / nch;
  nch = (nact + chunk - 1) / chunk;
  const int nunits = ntiles * nch;
#define LS_ZD_LIMIT (a.wait_ns ? a.wait_ns : 1000000000ull)
  if (warp == NW && lane == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&done[k], NW);
    }
    mbar_init(gfull, 1);
    mbar_init(gdone, NW);
    mbar_init(never, 1);
    mbar_init_fence();
  }
  for (int i = tid; i < R1 * R2; i += W::NT) {
    twa[(i / R1) * W::TWA + i % R1] = __ldg(a.zwa + i);
    twb[(i / R2) * W::TWB + i % R2] = __ldg(a.zwb + i);
  }
  __syncthreads();
  if (warp == NW) {
    if (lane != 0) return;
    // producer: units from the counter (the next id fetched one unit ahead), items in order
    int u_next = (int)atomicAdd(a.ctr, 1u);
    int cu = -1, cv = 0, cv_end = 0;   // unit being issued, next view position, its end
    int ng = 0;                        // Green tiles issued
    int st_tile[NS], st_view[NS];      // tile and view position of the item in each buffer
    bool finished = false, failed = false;
    // issue the next item into buffer buf; false when no work is left (the end marker is then written)
    auto issue = [&](int buf) -> bool {
      bool start = false;
      if (cv >= cv_end) {
        cu = u_next;
        if (cu >= nunits) {
          s_item[buf] = -1;
          mbar_arrive(&full[buf]);   // nothing copied: the entry is visible once the phase completes
          return false;
        }
        u_next = (int)atomicAdd(a.ctr, 1u);
        const int j = cu / nch, ch = cu % nch;
        cv = ch * chunk;
        cv_end = min(nact, cv + chunk);
        // the single Green buffer is free once the compute warps hold the previous tile in registers
        if (ng > 0 && !mbar_wait_abort(gdone, (unsigned)(ng - 1) & 1u, &s_abort, LS_ZD_LIMIT)) {
          failed = true;
          return false;
        }
        const int ky = j / tiles_c;
        const int fy = ky <= a.ny ? ky : 2 * a.ny - ky;
        if (LS_IN_BOUNDS(j < ntiles && fy >= 0 && fy <= a.ny, BS_Z_TILE)) {
          mbar_expect_tx(gfull, (unsigned)W::gtile_bytes);
          tma_load_3d(gsm, &a.gmap, gfull, 2 * (j % tiles_c) * P, fy, 0);
        } else {
          mbar_arrive(gfull);
        }
        ++ng;
        start = true;
      }
      const int j = cu / nch;
      st_tile[buf] = j;
      st_view[buf] = cv;
      s_item[buf] = cv | (start ? 1 << 16 : 0) | (j == 0 ? 1 << 17 : 0);
      if (LS_IN_BOUNDS(cv < nact && active_slot(s_list[cv]) < a.sel.nslots, BS_Z_TILE)) {
        mbar_expect_tx(&full[buf], (unsigned)W::stage_bytes);
        tma_load_4d(stage + (size_t)buf * NZ * P, &a.tmap, &full[buf], 2 * (j % tiles_c) * P, j / tiles_c, 0,
                    a.slot0 + active_slot(s_list[cv]));
      } else {
        mbar_arrive(&full[buf]);
      }
      ++cv;
      return true;
    };
    int n_issued = 0;
    for (int k = 0; k < NS && !finished; ++k) {
      if (issue(k)) ++n_issued;
      else finished = true;
    }
    int i = 0;
    for (; i < n_issued && !failed; ++i) {
      const int buf = i % NS;
      if (!mbar_wait_abort(&done[buf], (unsigned)(i / NS) & 1u, &s_abort, LS_ZD_LIMIT)) {
        failed = true;
        break;
      }
      tma_store_4d(&a.tmap, stage + (size_t)buf * NZ * P, 2 * (st_tile[buf] % tiles_c) * P, st_tile[buf] / tiles_c,
                   0, a.slot0 + active_slot(s_list[st_view[buf]]));
      bulk_commit();
      if (!finished) {
        bulk_wait_read_all();   // the store has read the buffer
        if (issue(buf)) ++n_issued;
        else finished = true;
      }
    }
    bulk_wait_read_all();
    if (failed) {
      // flag the launch; give the copies still in flight into this CTA's buffers (the items from i
      // on, and the last Green tile) a bounded time to land
      atomicExch(a.err, 1);
      s_abort = 1;
      for (int k = i; k < n_issued; ++k) mbar_wait(&full[k % NS], (unsigned)(k / NS) & 1u);
      if (ng > 0) mbar_wait(gfull, (unsigned)(ng - 1) & 1u);
    }
    return;
  }
  // compute warps (as k_zw: each owns CPW whole columns, lane = t * CPW + column)
  const int t = lane / CPW;
  const int c = warp * CPW + lane % CPW;
  constexpr int S2 = W::S2;
  float2* xc = xs + c * W::XP;
  const unsigned rb = swz128(t, c);
  float2 g[S2][R2];
  int ngot = 0;   // Green tiles taken
#pragma unroll 1
  for (int i = 0;; ++i) {
    const int buf = i % NS;
    const bool ok = (a.stall && i == 0) ? mbar_wait_abort(never, 0u, &s_abort, LS_ZD_LIMIT)
                                        : mbar_wait_abort(&full[buf], (unsigned)(i / NS) & 1u, &s_abort, LS_ZD_LIMIT);
    if (!__all_sync(0xffffffffu, ok)) break;
    const int e = s_item[buf];
    if (e < 0) break;
    const int iv = e & 0xffff;
    if (e & (1 << 16)) {
      // first view of a unit: its Green values (kz = t + R1 k2 folded into [0, NZ]) into registers
      const bool gok = mbar_wait_abort(gfull, (unsigned)ngot & 1u, &s_abort, LS_ZD_LIMIT);
      if (!__all_sync(0xffffffffu, gok)) break;
      ++ngot;
#pragma unroll
      for (int s2 = 0; s2 < S2; ++s2) {
        const int k1 = t + T * s2;
        if (R1 == T * S2 || k1 < R1) {
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int kz = k2 < R2 / 2 ? k1 + R1 * k2 : L - R1 * k2 - k1;
            g[s2][k2] = *reinterpret_cast<const float2*>(gsm + swz128(kz, c));
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(gdone);
    }
    count_run_if(a.sel, (e & (1 << 17)) != 0);   // each view once per launch (with tile 0)
    unsigned char* sb = reinterpret_cast<unsigned char*>(stage + (size_t)buf * NZ * P);
    zw_view<W, L>(sb, xc, twa, twb, g, nullptr, t, c, rb, [&] { return active_adj(s_list[iv]); }, [] {});
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[buf]);
  }
#undef LS_ZD_LIMIT
}

// ------------------------------------------------------------------------- Z (TMA-staged, column groups)
// The TMA-staged z pass for lengths whose balanced split has a thread count that does not divide 32
// (the bead lengths 144 = 12 x 12 and 288 = 12 x 24).  T = R1 = 12 threads per column; a group of
// WG = 3 warps (96 threads) owns CG = 8 whole columns, so no lane idles; two groups per CTA cover the
// 16 columns of one TMA box.  A column's threads span the warps of its group, so its exchanges are
// ordered by a named barrier of the group, and the group agrees on every wait's outcome with a
// barrier reduction (no thread of a group can leave the view loop while another waits at a group
// barrier).  Stage 1 and the last inverse stage give each thread S1 = R2 / T sub-transforms of
// length R1; stage 2 and the first inverse stage one of length R2.  Producer warp, view buffers,
// Green values in registers and the waits' limits are those of k_zw.
template <int L> struct ZGRadix { static constexpr bool ok = false; static constexpr int R1 = 2, R2 = 2, NS = 1, MINB = 1; };
template <> struct ZGRadix<144> { static constexpr bool ok = true; static constexpr int R1 = 12, R2 = 12, NS = 4, MINB = 3; };
template <> struct ZGRadix<288> { static constexpr bool ok = true; static constexpr int R1 = 12, R2 = 24, NS = 3, MINB = 2; };

template <int L>
struct ZG {
  static constexpr bool ok = ZGRadix<L>::ok;
  static constexpr int R1 = ZGRadix<L>::R1, R2 = ZGRadix<L>::R2;
  static constexpr int T = R1;                   // threads per column
  static constexpr int S1 = R2 / T;              // stage-1 sub-transforms per thread
  static constexpr int CG = 8, WG = 3;           // columns and warps of a group: CG * T == 32 * WG
  static constexpr int P = 16;                   // columns per CTA: one 128-byte TMA row
  static constexpr int NGRP = P / CG;
  static constexpr int NW = NGRP * WG;           // compute warps
  static constexpr int NT = 32 * NW + 32;        // + one producer warp
  static constexpr int NZ = L / 2;
  static constexpr int NS = ZGRadix<L>::NS, MINB = ZGRadix<L>::MINB;
  // exchange rows of R + 2 entries, read with 16-byte loads; per-column pitch congruent to 2 mod 16
  // (float2 units): the 8 columns of a quarter-warp's 16-byte reads, and the two rows by eight
  // columns of a half-warp's 8-byte writes, fall on disjoint banks
  static constexpr int RA = R2 + 2, RB = R1 + 2;
  static constexpr int pitch(int n) { return n + ((2 - n % 16) % 16 + 16) % 16; }
  static constexpr int XP = pitch(imax(R1 * RA, R2 * RB));
  static constexpr int TWA = R1 + 2, TWB = R2 + 2;
  static constexpr size_t r16(size_t b) { return (b + 15) / 16 * 16; }
  static constexpr size_t stage_bytes = (size_t)NZ * P * sizeof(float2);
  // Green rows [kz][P + 8] of the non-persistent form: the two rows of a half-warp's reads are 8
  // words apart; the exchange area overlays the Green tile
  static constexpr int GR = P + 8;
  static constexpr size_t g_bytes = r16((size_t)(NZ + 1) * GR * sizeof(float2));
  static constexpr size_t x_bytes = r16((size_t)P * XP * sizeof(float2));
  static constexpr size_t off_x = NS * stage_bytes;
  static constexpr size_t off_g = off_x;
  static constexpr size_t off_twa = off_x + (g_bytes > x_bytes ? g_bytes : x_bytes);
  static constexpr size_t off_twb = off_twa + r16((size_t)R2 * TWA * sizeof(float2));
  static constexpr size_t off_bar = off_twb + r16((size_t)R1 * TWB * sizeof(float2));
  static constexpr int NBAR = 2 * NS + 1;                                     // full[NS], done[NS], never
  static constexpr size_t smem = off_bar + NBAR * sizeof(uint64_t) + 1024;    // + room to align the base to 1024
};

// Barrier of N threads on named barrier ID (N a multiple of 32, warp-uniform calls).
template <int ID, int N>
__device__ __forceinline__ void named_sync() {
  asm volatile("bar.sync %0, %1;\n" ::"n"(ID), "n"(N) : "memory");
}
// The same barrier, returning the AND of `v` over the participating threads.
template <int ID, int N>
__device__ __forceinline__ bool named_all(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.and.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r) : "r"((unsigned)v), "n"(ID), "n"(N) : "memory");
  return r != 0;
}
// Group barriers of the column-group z pass: named barriers 2 + group (0 is __syncthreads, 1 the
// compute warps' barrier).
template <int NGRP, int N>
__device__ __forceinline__ void group_sync(int gi) {
  static_assert(NGRP == 2, "two column groups per CTA");
  if (gi == 0) named_sync<2, N>();
  else named_sync<3, N>();
}
template <int NGRP, int N>
__device__ __forceinline__ bool group_all(int gi, bool v) {
  static_assert(NGRP == 2, "two column groups per CTA");
  return gi == 0 ? named_all<2, N>(v) : named_all<3, N>(v);
}

template <int L, bool PERSIST>
__global__ void __launch_bounds__(ZG<L>::NT, ZG<L>::MINB) k_zg(const __grid_constant__ ZParams a) {
  using W = ZG<L>;
  constexpr int R1 = W::R1, R2 = W::R2, P = W::P, NZ = W::NZ, T = W::T, S1 = W::S1, CG = W::CG, WG = W::WG,
                NW = W::NW, NS = W::NS, RA = W::RA, RB = W::RB;
  static_assert(W::ok && CG * T == 32 * WG && R2 % T == 0 && R1 == T, "k_zg split");
  static_assert(R1 % 2 == 0 && R2 % 2 == 0 && W::XP % 2 == 0, "16-byte exchange reads need even rows");
  extern __shared__ __align__(16) unsigned char zg_raw[];
  const unsigned raw = smem_addr(zg_raw);
  unsigned char* base = zg_raw + (((raw + 1023u) & ~1023u) - raw);
  float2* stage = reinterpret_cast<float2*>(base);
  float2* xs = reinterpret_cast<float2*>(base + W::off_x);
  float2* gs = reinterpret_cast<float2*>(base + W::off_g);
  float2* twa = reinterpret_cast<float2*>(base + W::off_twa);
  float2* twb = reinterpret_cast<float2*>(base + W::off_twb);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + W::off_bar);   // [NS]: an item's tile has landed
  uint64_t* done = full + NS;                                         // [NS]: the compute warps are done with it
  uint64_t* never = done + NS;                                        // no thread arrives on it (stall test)
  __shared__ int s_list[kMaxLaunchSlots];
  __shared__ int s_ws[32];
  __shared__ int s_abort;
  const int nact = build_active(a.sel, s_list, s_ws);
  if (nact == 0) return;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles_c = 2 * a.nx / P;
  const int ntiles = tiles_c * 2 * a.ny;
  // as k_zw: one tile per CTA, or persistent (tiles blockIdx.x + k gridDim.x), items i = k nact + view
  const int ntl = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int nitems = ntl * nact;
  const bool producer = warp == NW;
#define LS_ZG_LIMIT (a.wait_ns ? a.wait_ns : 1000000000ull)
  // TMA coordinates of the item (view position iv, tile number kt of this CTA): (2 kx0 floats, ky, 0, slot)
  auto item_load = [&](int iv, int kt, int buf) {
    const int j = (int)blockIdx.x + kt * (int)gridDim.x;
    if (!LS_IN_BOUNDS(j < ntiles && iv < nact && active_slot(s_list[iv]) < a.sel.nslots, BS_Z_TILE)) {
      mbar_arrive(&full[buf]);   // nothing copied: the buffer's phase completes at once
      return;
    }
    mbar_expect_tx(&full[buf], (unsigned)W::stage_bytes);
    tma_load_4d(stage + (size_t)buf * NZ * P, &a.tmap, &full[buf], 2 * (j % tiles_c) * P, j / tiles_c, 0,
                a.slot0 + active_slot(s_list[iv]));
  };
  if (producer && lane == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&done[k], NW);
    }
    mbar_init(never, 1);
    mbar_init_fence();
    for (int k = 0; k < NS && k < nitems; ++k) item_load(k % nact, k / nact, k);
  }
  if constexpr (!PERSIST) {
    // the CTA's one tile: its Green tile, kz folded into [0, NZ]
    const int ky = blockIdx.x / tiles_c, kx0 = (blockIdx.x % tiles_c) * P;
    const int fy = ky <= a.ny ? ky : 2 * a.ny - ky;
    // every load of the gather is issued before any store (one L2 round trip, not one per element)
    constexpr int GN = (NZ + 1) * P, GIT = (GN + W::NT - 1) / W::NT;
    float2 gv[GIT];
#pragma unroll
    for (int r = 0; r < GIT; ++r) {
      const int i = tid + r * W::NT;
      const int kz = i / P, c2 = i % P, kx = kx0 + c2;
      const int fx = kx <= a.nx ? kx : 2 * a.nx - kx;
      if (i < GN && LS_IN_BOUNDS(kz <= a.nz && fy >= 0 && fy <= a.ny && fx >= 0 && fx <= a.nx, BS_Z_GREEN))
        gv[r] = __ldg(a.gocta + ((size_t)kz * (a.ny + 1) + fy) * (a.nx + 1) + fx);
    }
#pragma unroll
    for (int r = 0; r < GIT; ++r) {
      const int i = tid + r * W::NT;
      if (i < GN) gs[(i / P) * W::GR + i % P] = gv[r];
    }
  }
  for (int i = tid; i < R1 * R2; i += W::NT) {
    twa[(i / R1) * W::TWA + i % R1] = __ldg(a.zwa + i);
    twb[(i / R2) * W::TWB + i % R2] = __ldg(a.zwb + i);
  }
  __syncthreads();
  if (producer) {
    if (lane != 0) return;
    // (view position, tile number) of the item being stored and of the one NS ahead, kept by counting
    int sv = 0, skt = 0, lv = NS % nact, lkt = NS / nact;
    int i = 0;
    for (; i < nitems; ++i) {
      const int buf = i % NS;
      if (!mbar_wait_abort(&done[buf], (unsigned)(i / NS) & 1u, &s_abort, LS_ZG_LIMIT)) break;
      const int j = (int)blockIdx.x + skt * (int)gridDim.x;
      if (LS_IN_BOUNDS(j < ntiles && active_slot(s_list[sv]) < a.sel.nslots, BS_Z_TILE))
        tma_store_4d(&a.tmap, stage + (size_t)buf * NZ * P, 2 * (j % tiles_c) * P, j / tiles_c, 0,
                     a.slot0 + active_slot(s_list[sv]));
      bulk_commit();
      if (i + NS < nitems) {
        bulk_wait_read_all();   // the store has read the buffer
        item_load(lv, lkt, buf);
      }
      if (++sv == nact) { sv = 0; ++skt; }
      if (++lv == nact) { lv = 0; ++lkt; }
    }
    bulk_wait_read_all();
    if (i < nitems) {
      // gave up at item i: flag it, and give the loads still in flight into this CTA's buffers
      // (items i .. i + NS - 1, all issued) a bounded time to land (one second each, whatever
      // the per-view limit)
      atomicExch(a.err, 1);
      for (int k = i; k < i + NS && k < nitems; ++k) mbar_wait(&full[k % NS], (unsigned)(k / NS) & 1u);
    }
    return;
  }
  // compute warps: group gi of WG warps owns columns [gi CG, gi CG + CG); thread (t, c) of the group
  const int gi = warp / WG;
  const int g = (warp % WG) * 32 + lane;
  const int t = g / CG, c = g % CG;
  const int cc = gi * CG + c;
  float2* xc = xs + cc * W::XP;
  // this thread's Green values (kz = t + R1 k2) for the current tile, in registers
  float2 gr[R2];
  if constexpr (PERSIST) {
    load_green<L, R1, R2>(gr, a, blockIdx.x / tiles_c, (blockIdx.x % tiles_c) * P + cc, t);
  } else {
    const float2* gc = gs + cc;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) gr[k2] = k2 < R2 / 2 ? gc[(t + R1 * k2) * W::GR] : gc[(L - R1 * k2 - t) * W::GR];
    // the exchange area overlays the Green tile: every compute warp has its values before any writes
    named_sync<1, NW * 32>();
  }
  int iv = 0, kt = 0;   // view position and tile number of item i, kept by counting
#pragma unroll 1
  for (int i = 0; i < nitems; ++i) {
    const int buf = i % NS;
    const bool ok = (a.stall && i == 0) ? mbar_wait_abort(never, 0u, &s_abort, LS_ZG_LIMIT)
                                        : mbar_wait_abort(&full[buf], (unsigned)(i / NS) & 1u, &s_abort, LS_ZG_LIMIT);
    // the group agrees (this is also the barrier that frees the exchange area of the previous item)
    if (!group_all<W::NGRP, WG * 32>(gi, ok)) break;
    if (i < nact) count_run(a.sel);   // each view once per launch (by the first tile of CTA 0)
    unsigned char* sb = reinterpret_cast<unsigned char*>(stage + (size_t)buf * NZ * P);
    // forward stage 1: sub-transforms n2 = t + T s, inputs z = R2 n1 + n2 (n1 < R1/2: z < nz)
#pragma unroll
    for (int s = 0; s < S1; ++s) {
      const int n2 = t + T * s;
      float2 v[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = make_float2(0.f, 0.f);
#pragma unroll
      for (int n1 = 0; n1 < R1 / 2; ++n1)
        if (LS_IN_BOUNDS(swz128(R2 * n1 + n2, cc) + sizeof(float2) <= W::stage_bytes, BS_Z_SMEM))
          v[n1] = *reinterpret_cast<const float2*>(sb + swz128(R2 * n1 + n2, cc));
      Dft<R1, -1, R1 / 2, R1>::run(v);
      const float4* tw4 = reinterpret_cast<const float4*>(twa + n2 * W::TWA);
#pragma unroll
      for (int k = 0; k < R1 / 2; ++k) {
        const float4 w = tw4[k];
        if (k > 0) v[2 * k] = cmul(v[2 * k], make_float2(w.x, w.y));
        v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w.z, w.w));
      }
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1)
        if (LS_IN_BOUNDS(cc * W::XP + k1 * RA + n2 < P * W::XP, BS_Z_SMEM)) xc[k1 * RA + n2] = v[k1];
    }
    group_sync<W::NGRP, WG * 32>(gi);
    // forward stage 2 (thread t = k1), Green multiply, inverse stage 1 (transposed split)
    float2 u[R2];
#pragma unroll
    for (int q = 0; q < R2 / 2; ++q) {
      const float4 x = *reinterpret_cast<const float4*>(xc + t * RA + 2 * q);
      u[2 * q] = make_float2(x.x, x.y);
      u[2 * q + 1] = make_float2(x.z, x.w);
    }
    Dft<R2, -1>::run(u);
    if (active_adj(s_list[iv])) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) u[k2] = cmulc(u[k2], gr[k2]);
    } else {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) u[k2] = cmul(u[k2], gr[k2]);
    }
    if (PERSIST && iv == nact - 1 && i + 1 < nitems) {
      // last view of this tile: the next tile's Green values, in flight while the transforms run
      const int j = (int)blockIdx.x + (kt + 1) * (int)gridDim.x;
      load_green<L, R1, R2>(gr, a, j / tiles_c, (j % tiles_c) * P + cc, t);
    }
    Dft<R2, +1>::run(u);
    {
      const float4* tw4 = reinterpret_cast<const float4*>(twb + t * W::TWB);
#pragma unroll
      for (int k = 0; k < R2 / 2; ++k) {
        const float4 w = tw4[k];
        if (k > 0) u[2 * k] = cmulc(u[2 * k], make_float2(w.x, w.y));
        u[2 * k + 1] = cmulc(u[2 * k + 1], make_float2(w.z, w.w));
      }
    }
    group_sync<W::NGRP, WG * 32>(gi);   // every thread of the group has read its stage-1 row
#pragma unroll
    for (int j1 = 0; j1 < R2; ++j1) xc[j1 * RB + t] = u[j1];
    group_sync<W::NGRP, WG * 32>(gi);
    // inverse stage 2: sub-transforms j1 = t + T s; outputs z = j1 + R2 j2 (j2 < R1/2: z < nz), in place
#pragma unroll
    for (int s = 0; s < S1; ++s) {
      const int j1 = t + T * s;
      float2 w[R1];
#pragma unroll
      for (int q = 0; q < R1 / 2; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(xc + j1 * RB + 2 * q);
        w[2 * q] = make_float2(x.x, x.y);
        w[2 * q + 1] = make_float2(x.z, x.w);
      }
      Dft<R1, +1, R1, R1 / 2>::run(w);
#pragma unroll
      for (int j2 = 0; j2 < R1 / 2; ++j2)
        if (LS_IN_BOUNDS(swz128(j1 + R2 * j2, cc) + sizeof(float2) <= W::stage_bytes, BS_Z_SMEM))
          *reinterpret_cast<float2*>(sb + swz128(j1 + R2 * j2, cc)) = w[j2];
    }
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&done[buf]);
    if (++iv == nact) { iv = 0; ++kt; }
  }
#undef LS_ZG_LIMIT
}

}  // namespace lsgpu

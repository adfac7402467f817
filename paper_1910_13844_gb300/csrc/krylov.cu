// BiCGStab scalar steps, fused vector update, and the element-wise kernels of
// the forward model and gradient (incident plane waves, far-field slice sum,
// adjoint far-field multiply, gradient accumulation, residuals).
//
// BiCGStab (van der Vorst 1992) for (I - G diag f) u = u_in (eq. lipp1, the
// solver the paper names in Sec. 2.2), complex with <a, b> = sum conj(a) b:
//   rho_i = <rh, r>;  beta = (rho_i / rho_{i-1}) (alpha / omega)
//   p = r + beta (p - omega v);  v = A p;  alpha = rho_i / <rh, v>
//   s = r - alpha v;  t = A s;  omega = <t, s> / <t, t>
//   x = x + alpha p + omega s;  r = s - omega t
// The p/s updates run inside the first FFT pass and v/t inside the last one
// (passes.cuh); this file holds the x/r update and the per-slot scalar logic.
// Dot products: float32 products and per-thread partial sums; every sum across threads in float64.
#include "krylov.cuh"
#include "passes.cuh"

#include <math.h>

namespace lsgpu {

// ------------------------------------------------------------------ update
// x += alpha p + omega s ; r = s - omega t ; partials <rh, r>, ||r||^2
__global__ void __launch_bounds__(256, 4) k_update(UpdParams a) {
  const int slot = blockIdx.y;
  if (!LS_IN_BOUNDS(slot < a.sel.nslots && (a.sel.nslots <= 1 || a.n <= a.vstride), BS_UPD_VEC)) return;
  if (!slot_runs(a.sel, slot)) return;
  count_run(a.sel);
  const SlotDev& sd = a.sel.slots[slot];
  const float2 al = sd.alpha_f;
  const float2 om = sd.omega_f;
  const size_t base = (size_t)slot * a.vstride;
  const float4* p = reinterpret_cast<const float4*>(a.p + base);
  const float4* s = reinterpret_cast<const float4*>(a.s + base);
  const float4* t = reinterpret_cast<const float4*>(a.t + base);
  const float4* rh = reinterpret_cast<const float4*>(a.rh + base);
  float4* x = reinterpret_cast<float4*>(a.x + base);
  float4* r = reinterpret_cast<float4*>(a.r + base);
  const size_t n4 = a.n / 2;
  float acc[3] = {0.f, 0.f, 0.f};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    float4 pv = __ldg(p + i), sv = __ldg(s + i), tv = __ldg(t + i), hv = __ldg(rh + i), xv = x[i];
    float2 p0 = make_float2(pv.x, pv.y), p1 = make_float2(pv.z, pv.w);
    float2 s0 = make_float2(sv.x, sv.y), s1 = make_float2(sv.z, sv.w);
    float2 t0 = make_float2(tv.x, tv.y), t1 = make_float2(tv.z, tv.w);
    float2 x0 = cadd(make_float2(xv.x, xv.y), cadd(cmul(al, p0), cmul(om, s0)));
    float2 x1 = cadd(make_float2(xv.z, xv.w), cadd(cmul(al, p1), cmul(om, s1)));
    float2 r0 = csub(s0, cmul(om, t0));
    float2 r1 = csub(s1, cmul(om, t1));
    x[i] = make_float4(x0.x, x0.y, x1.x, x1.y);
    r[i] = make_float4(r0.x, r0.y, r1.x, r1.y);
    float2 d0 = cdotterm(make_float2(hv.x, hv.y), r0);
    float2 d1 = cdotterm(make_float2(hv.z, hv.w), r1);
    acc[0] += d0.x + d1.x;
    acc[1] += d0.y + d1.y;
    acc[2] += r0.x * r0.x + r0.y * r0.y + r1.x * r1.x + r1.y * r1.y;
  }
  if (LS_IN_BOUNDS(a.maxparts == 0 || (int)gridDim.x <= a.maxparts, BS_UPD_PART))
    block_sum_store<3>(acc, a.partials + ((size_t)slot * gridDim.x + blockIdx.x) * 4);
}

// ------------------------------------------------------------------ scalar steps
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ bool zfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Relative breakdown threshold of BiCGStab's two inner products (the paper gives none).
constexpr double kBreakdownRel = 1e-30;

// One block per slot: sums the partials of the preceding kernel in a fixed
// order (float64), then thread 0 advances the slot's BiCGStab state.
__global__ void __launch_bounds__(256) k_scalar(ScalarParams a) {
  const int slot = blockIdx.x;
  SlotDev& sd = a.slots[slot];
  if (!(sd.flags & a.mask)) return;
  const double* part = a.partials + (size_t)slot * a.nparts * 4;
  // three partial sums per block (PH_RESID uses the first two)
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < a.nparts; i += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 3; ++j) v[j] += part[(size_t)i * 4 + j];
  }
  __shared__ double red[256][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) red[threadIdx.x][j] = v[j];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int j = 0; j < 3; ++j) red[threadIdx.x][j] += red[threadIdx.x + o][j];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double s0 = red[0][0], s1 = red[0][1], s2 = red[0][2];
  switch (a.phase) {
    case PH_RESID: {
      // partials: ||r||^2, ||b||^2 of r = b - A x
      sd.matvecs += 1;
      sd.bnorm2 = s1;
      sd.true_rnorm2 = s0;
      sd.flags &= ~SLOT_RESID;
      const bool initial = sd.checks == 0;
      sd.checks += 1;
      const double rel = s1 > 0.0 ? sqrt(s0 / s1) : 0.0;
      if (!isfinite(rel)) { sd.status = LS_BREAKDOWN; sd.flags &= ~SLOT_ITER; break; }
      const double accept = initial ? sd.tol : 10.0 * sd.tol;
      if (s1 == 0.0 || rel <= accept) {
        sd.rnorm2 = s0;
        if (sd.status == LS_BREAKDOWN && rel <= accept) sd.status = LS_OK;
        sd.flags &= ~SLOT_ITER;
        break;
      }
      if (sd.iters >= sd.max_iter || (!initial && sd.restarts >= sd.max_restarts)) {
        if (sd.status == LS_OK) sd.status = LS_NOT_CONVERGED;
        sd.flags &= ~SLOT_ITER;
        break;
      }
      if (!initial) sd.restarts += 1;
      // (re)start: rh = r (written by the pass), rho = <r, r>, alpha = omega = 1
      sd.status = LS_OK;
      sd.rho = make_double2(s0, 0.0);
      sd.rhnorm2 = s0;   // rh = r
      sd.alpha = make_double2(1.0, 0.0);
      sd.omega = make_double2(1.0, 0.0);
      sd.beta = make_double2(0.0, 0.0);
      sd.rnorm2 = s0;
      sd.first = 1;
      sd.flags |= SLOT_ITER;
    } break;
    case PH_ALPHA: {
      const double2 rv = make_double2(s0, s1);   // <rh, v>
      const double vv = s2;                      // ||v||^2
      sd.matvecs += 1;
      // breakdown when <rh, v> vanishes relative to ||rh|| ||v|| (or is not finite)
      if (!zfinite(rv) || !(hypot(rv.x, rv.y) > kBreakdownRel * sqrt(sd.rhnorm2 * vv))) {
        sd.status = LS_BREAKDOWN;
        sd.alpha = make_double2(0.0, 0.0);
        sd.flags = (sd.flags & ~SLOT_ITER) | SLOT_RESID;
        break;
      }
      sd.alpha = zdiv(sd.rho, rv);
    } break;
    case PH_OMEGA: {
      const double2 ts = make_double2(s0, s1);   // <t, s>
      const double tt = s2;                      // <t, t>
      sd.matvecs += 1;
      sd.omega = tt > 0.0 ? make_double2(ts.x / tt, ts.y / tt) : make_double2(0.0, 0.0);
    } break;
    case PH_RHO: {
      const double2 rho_new = make_double2(s0, s1);   // <rh, r>
      const double rr = s2;
      sd.iters += 1;
      sd.rnorm2 = rr;
      const double rel = sd.bnorm2 > 0.0 ? sqrt(rr / sd.bnorm2) : 0.0;
      if (!isfinite(rel)) {
        sd.status = LS_BREAKDOWN;
        sd.flags &= ~SLOT_ITER;
        break;
      }
      if (rel <= sd.tol) { sd.flags = (sd.flags & ~SLOT_ITER) | SLOT_RESID; break; }
      if (sd.iters >= sd.max_iter) {
        sd.status = LS_NOT_CONVERGED;
        sd.flags = (sd.flags & ~SLOT_ITER) | SLOT_RESID;
        break;
      }
      const double om = fabs(sd.omega.x) + fabs(sd.omega.y);
      // breakdown when rho = <rh, r> vanishes relative to ||rh|| ||r|| (or is not finite), or omega = 0
      if (om == 0.0 || !zfinite(rho_new) || !(hypot(rho_new.x, rho_new.y) > kBreakdownRel * sqrt(sd.rhnorm2 * rr))) {
        sd.status = LS_BREAKDOWN;
        sd.flags = (sd.flags & ~SLOT_ITER) | SLOT_RESID;
        break;
      }
      sd.beta = zmul(zdiv(rho_new, sd.rho), zdiv(sd.alpha, sd.omega));
      sd.rho = rho_new;
      sd.first = 0;
    } break;
  }
  sd.alpha_f = make_float2((float)sd.alpha.x, (float)sd.alpha.y);
  sd.omega_f = make_float2((float)sd.omega.x, (float)sd.omega.y);
  sd.beta_f = make_float2((float)sd.beta.x, (float)sd.beta.y);
}

// Test-only failure injection: zero the shadow residual of one slot at its initial residual
// evaluation, so that <rh, v> vanishes in the first iteration (a forced BiCGStab breakdown).
__global__ void k_zero_shadow(const SlotDev* slots, int slot, float2* rh, size_t n) {
  if (slots[slot].checks != 0 || !(slots[slot].flags & SLOT_RESID)) return;
  float2* v = rh + (size_t)slot * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v[i] = make_float2(0.f, 0.f);
}

// Count slots per flag so the host can decide what to run next.
__global__ void k_count(const SlotDev* slots, int nslots, int* out) {
  __shared__ int c[4];
  if (threadIdx.x < 4) c[threadIdx.x] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
    const unsigned f = slots[s].flags;
    if (f & SLOT_ITER) atomicAdd(&c[0], 1);
    if (f & SLOT_RESID) atomicAdd(&c[1], 1);
  }
  __syncthreads();
  if (threadIdx.x < 4) out[threadIdx.x] = c[threadIdx.x];
}

// ------------------------------------------------------------------ element-wise kernels

// u_in,q(x) = exp(i k_q . x) at voxel centres (Fig. 1) is separable: exp(i kx x) exp(i ky y) exp(i kz z).
// The three 1-D factors are evaluated per view with the phase reduced mod 2 pi in float64
// (tables [view][nx + ny + nz]); the volume is their complex64 product.
__global__ void k_plane_tables(PlaneWaveParams a) {
  const int q = blockIdx.y;
  const int m = a.nx + a.ny + a.nz;
  const double twopi = 6.283185307179586476925286766559;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    int axis = 0, idx = j, n = a.nx;
    if (j >= a.nx + a.ny) { axis = 2; idx = j - a.nx - a.ny; n = a.nz; }
    else if (j >= a.nx) { axis = 1; idx = j - a.nx; n = a.ny; }
    double ph = a.k[3 * q + axis] * (a.h * (idx - n / 2 + 1));
    ph -= twopi * rint(ph / twopi);
    double sn, cs;
    sincos(ph, &sn, &cs);
    a.tables[(size_t)q * m + j] = make_float2((float)cs, (float)sn);
  }
}

__global__ void k_plane_waves(PlaneWaveParams a) {
  const int q = blockIdx.y;
  const float2* ex = a.tables + (size_t)q * (a.nx + a.ny + a.nz);
  const float2* ey = ex + a.nx;
  const float2* ez = ey + a.ny;
  float2* out = a.out[q];
  const size_t plane = (size_t)a.nx * a.ny;
  const size_t n = plane * a.nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % a.nx);
    const int iy = (int)((i / a.nx) % a.ny);
    const int iz = (int)(i / plane);
    out[i] = cmul(__ldg(ez + iz), cmul(__ldg(ey + iy), __ldg(ex + ix)));
  }
}

// f = k_b^2 ((eta_b + dn)^2 / eta_b^2 - 1) (Sec. 2.1)
__global__ void k_potential(const float* dn, size_t count, double eta_b, double kb, float* f) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const double e = (eta_b + (double)dn[i]) / eta_b;
    f[i] = (float)(kb * kb * (e * e - 1.0));
  }
}

// Yhat[s][ky][kx] = sum_z K2hat[z][ky][kx] * A2[s][z][ky][kx]  (per-slice far-field kernels, eq. Gtild-1)
__global__ void k_far_reduce(FarParams a) {
  const int slot = blockIdx.y;
  if (!slot_runs(a.sel, slot)) return;
  const size_t plane = (size_t)(2 * a.ny) * (2 * a.nx);
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= plane) return;
  const float2* src = a.a2 + (size_t)slot * a.a2_stride + i;
  const float2* k = a.k2 + i;
  float2 acc = make_float2(0.f, 0.f);
  for (int z = 0; z < a.nz; ++z) acc = cadd(acc, cmul(__ldg(k + (size_t)z * plane), __ldg(src + (size_t)z * plane)));
  a.out[(size_t)slot * a.out_stride + i] = acc;
}

// A2[s][z][ky][kx] = conj(K2hat[z][ky][kx]) * Rhat[s][ky][kx]   (adjoint of the slice sum)
__global__ void k_far_adjoint_mul(FarParams a) {
  const int slot = blockIdx.y;
  if (!slot_runs(a.sel, slot)) return;
  const size_t plane = (size_t)(2 * a.ny) * (2 * a.nx);
  const size_t total = plane * a.nz;
  const float2* rhat = a.rhat + (size_t)slot * a.rhat_stride;
  float2* dst = a.a2 + (size_t)slot * a.a2_stride;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    dst[i] = cmulc(__ldg(rhat + (i % plane)), __ldg(a.k2 + i));
  }
}

// plane[s][y][x] = r[s][y - oy][x - ox] inside the detector window, 0 outside
__global__ void k_pad_detector(PadParams a) {
  const int slot = blockIdx.y;
  if (!slot_runs(a.sel, slot)) return;
  const size_t n = (size_t)a.ny * a.nx;
  const float2* r = a.src[slot];
  float2* dst = a.dst + (size_t)slot * a.dst_stride;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % a.nx), y = (int)(i / a.nx);
    const int xo = x - a.ox, yo = y - a.oy;
    dst[i] = (xo >= 0 && xo < a.mx && yo >= 0 && yo < a.my) ? r[(size_t)yo * a.mx + xo] : make_float2(0.f, 0.f);
  }
}

// grad[i] = sum_s c_s Re(conj(u_s[i]) w_s[i]), fixed slot order (Alg. 1 line 6)
__global__ void k_gradient(GradParams a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.n; i += (size_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int s = 0; s < a.nslots; ++s) {
      const float2 u = __ldg(a.u[s] + i);
      const float2 w = __ldg(a.w + (size_t)s * a.w_stride + i);
      acc += a.c[s] * (u.x * w.x + u.y * w.y);
    }
    a.grad[i] = acc;
  }
}

// res = pred - meas ; per-view partial ||res||^2
__global__ void __launch_bounds__(256) k_residual(ResidualParams a) {
  const int q = blockIdx.y;
  const float2* p = a.pred[q];
  const float2* m = a.meas[q];
  float2* r = a.res[q];
  float acc[2] = {0.f, 0.f};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 d = csub(__ldg(p + i), __ldg(m + i));
    r[i] = d;
    acc[0] += d.x * d.x + d.y * d.y;
    const float2 mm = __ldg(m + i);
    acc[1] += mm.x * mm.x + mm.y * mm.y;
  }
  block_sum_store<2>(acc, a.partials + ((size_t)q * gridDim.x + blockIdx.x) * 4);
}

// <a, b> = sum conj(a) b per view (the inner product of the solver's scalars): float32 products and
// per-thread partial sums, float64 from the warp shuffles up (the solver kernels' reduction)
__global__ void __launch_bounds__(256) k_inner(ResidualParams a) {
  const int q = blockIdx.y;
  const float2* x = a.pred[q];
  const float2* y = a.meas[q];
  float acc[2] = {0.f, 0.f};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.count; i += (size_t)gridDim.x * blockDim.x) {
    const float2 d = cdotterm(__ldg(x + i), __ldg(y + i));
    acc[0] += d.x;
    acc[1] += d.y;
  }
  block_sum_store<2>(acc, a.partials + ((size_t)q * gridDim.x + blockIdx.x) * 4);
}

// ------------------------------------------------------------------ launchers
void launch_update(const UpdParams& a0, int nblocks, int nslots, cudaStream_t st) {
  UpdParams a = a0;
  a.sel.nslots = nslots;
  k_update<<<dim3(nblocks, nslots), 256, 0, st>>>(a);
}
void launch_scalar(const ScalarParams& a, int nslots, cudaStream_t st) {
  k_scalar<<<nslots, 256, 0, st>>>(a);
}
void launch_zero_shadow(const SlotDev* slots, int slot, float2* rh, size_t n, cudaStream_t st) {
  k_zero_shadow<<<256, 256, 0, st>>>(slots, slot, rh, n);
}
void launch_count(const SlotDev* slots, int nslots, int* out, cudaStream_t st) {
  k_count<<<1, 256, 0, st>>>(slots, nslots, out);
}
cudaError_t launch_plane_waves(const PlaneWaveParams& a0, int nviews, cudaStream_t st) {
  PlaneWaveParams a = a0;
  const int m = a.nx + a.ny + a.nz;
  cudaError_t e = cudaMallocAsync((void**)&a.tables, (size_t)nviews * m * sizeof(float2), st);
  if (e != cudaSuccess) return e;
  k_plane_tables<<<dim3((m + 127) / 128, nviews), 128, 0, st>>>(a);
  const size_t n = (size_t)a.nx * a.ny * a.nz;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1216) blocks = 1216;
  k_plane_waves<<<dim3(blocks, nviews), 256, 0, st>>>(a);
  e = cudaGetLastError();
  cudaError_t f = cudaFreeAsync(a.tables, st);
  return e != cudaSuccess ? e : f;
}
void launch_potential(const float* dn, size_t count, double eta_b, double kb, float* f, cudaStream_t st) {
  int blocks = (int)((count + 255) / 256);
  if (blocks > 4864) blocks = 4864;
  if (blocks < 1) blocks = 1;
  k_potential<<<blocks, 256, 0, st>>>(dn, count, eta_b, kb, f);
}
void launch_far_reduce(const FarParams& a, int nslots, cudaStream_t st) {
  const size_t plane = (size_t)(2 * a.ny) * (2 * a.nx);
  k_far_reduce<<<dim3((unsigned)((plane + 255) / 256), nslots), 256, 0, st>>>(a);
}
void launch_far_adjoint_mul(const FarParams& a, int nslots, cudaStream_t st) {
  const size_t total = (size_t)(2 * a.ny) * (2 * a.nx) * a.nz;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 2432) blocks = 2432;
  k_far_adjoint_mul<<<dim3(blocks, nslots), 256, 0, st>>>(a);
}
void launch_pad_detector(const PadParams& a, int nslots, cudaStream_t st) {
  const size_t n = (size_t)a.ny * a.nx;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  k_pad_detector<<<dim3(blocks, nslots), 256, 0, st>>>(a);
}
void launch_gradient(const GradParams& a, cudaStream_t st) {
  int blocks = (int)((a.n + 255) / 256);
  if (blocks > 4864) blocks = 4864;
  k_gradient<<<blocks, 256, 0, st>>>(a);
}
void launch_inner(const ResidualParams& a, int nblocks, int nviews, cudaStream_t st) {
  k_inner<<<dim3(nblocks, nviews), 256, 0, st>>>(a);
}
void launch_residual(const ResidualParams& a, int nblocks, int nviews, cudaStream_t st) {
  k_residual<<<dim3(nblocks, nviews), 256, 0, st>>>(a);
}

LS_BOUNDS_READER(krylov)

}  // namespace lsgpu

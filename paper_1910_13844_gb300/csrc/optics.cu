// Detector-plane optics: the incident field propagated from its measurement on the detector
// (Sec. 3.4, eq. propUin with the tilt transfer of eq. propUin-2) and the pupil / refocus
// operator P (Sec. 3.3).  Both are 2-D convolutions on the detector grid applied through FFTs;
// they run once per view per call (not inside the solver iterations) and use the float64
// pencil FFT of the plan builder.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "engine.h"

namespace lsgpu {

__device__ __forceinline__ int centred_i(int q, int M) { return q > M / 2 ? q - M : q; }

// A[y][x] = y_in[y][x] exp(-i (kx x + ky y)) (tilt transfer; kx = ky = 0 without it), in float64
__global__ void k_demodulate(const float2* y_in, int nx, int ny, double h, double kx, double ky, double2* A) {
  const size_t n = (size_t)nx * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    const double ph = -(kx * h * (x - nx / 2 + 1) + ky * h * (y - ny / 2 + 1));
    double s, c;
    sincos(ph, &s, &c);
    const float2 v = y_in[i];
    A[i] = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// B[z][y][x] = A[y][x] p_hat_z(w + k) / (nx ny), p_hat_z(w) = exp(-i (x_gamma - z) sqrt(kb^2 - |w|^2)),
// evanescent components dropped
__global__ void k_spread_planes(const double2* A, int nx, int ny, int nz, double h, double kb, double x_gamma,
                                double kx, double ky, double2* B) {
  const size_t plane = (size_t)nx * ny;
  const size_t n = plane * nz;
  const double scale = 1.0 / (double)plane;
  const double twopi = 6.283185307179586476925286766559;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / plane);
    const double wx = twopi * centred_i(x, nx) / (nx * h) + kx;
    const double wy = twopi * centred_i(y, ny) / (ny * h) + ky;
    const double s = kb * kb - wx * wx - wy * wy;
    double2 out = make_double2(0.0, 0.0);
    if (s >= 0.0) {
      const double zc = h * (z - nz / 2 + 1);
      double sn, cs;
      sincos(-(x_gamma - zc) * sqrt(s), &sn, &cs);
      const double2 a = A[i % plane];
      out = make_double2((a.x * cs - a.y * sn) * scale, (a.x * sn + a.y * cs) * scale);
    }
    B[i] = out;
  }
}

// u_in[z][y][x] = B exp(+i (kx x + ky y)), rounded to complex64
__global__ void k_modulate_store(const double2* B, int nx, int ny, int nz, double h, double kx, double ky,
                                 float2* u) {
  const size_t plane = (size_t)nx * ny;
  const size_t n = plane * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny);
    const double ph = kx * h * (x - nx / 2 + 1) + ky * h * (y - ny / 2 + 1);
    double s, c;
    sincos(ph, &s, &c);
    const double2 b = B[i];
    u[i] = make_float2((float)(b.x * c - b.y * s), (float)(b.x * s + b.y * c));
  }
}

// H[y][x] on the 2my x 2mx padded detector: 1{|w| <= k_cut} exp(i d sqrt(kb^2 - |w|^2)), propagating only
__global__ void k_pupil_transfer(int Mx, int My, double h, double kb, double kcut, double d, double2* Hd) {
  const size_t n = (size_t)Mx * My;
  const double twopi = 6.283185307179586476925286766559;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Mx), y = (int)(i / Mx);
    const double wx = twopi * centred_i(x, Mx) / (Mx * h), wy = twopi * centred_i(y, My) / (My * h);
    const double w2 = wx * wx + wy * wy;
    const double s = kb * kb - w2;
    double2 v = make_double2(0.0, 0.0);
    if (s >= 0.0 && w2 <= kcut * kcut) {
      double sn, cs;
      sincos(d * sqrt(s), &sn, &cs);
      v = make_double2(cs, sn);
    }
    Hd[i] = v;
  }
}

// pad the my x mx field into the 2my x 2mx grid (offset 0), float64
__global__ void k_pad_c64(const float2* in, int mx, int my, double2* out) {
  const int Mx = 2 * mx, My = 2 * my;
  const size_t n = (size_t)Mx * My;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Mx), y = (int)(i / Mx);
    out[i] = (x < mx && y < my) ? make_double2(in[(size_t)y * mx + x].x, in[(size_t)y * mx + x].y)
                                : make_double2(0.0, 0.0);
  }
}

__global__ void k_mul_transfer(double2* d, const double2* Hd, size_t n, int conj, double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 hv = Hd[i];
    if (conj) hv.y = -hv.y;
    const double2 a = d[i];
    d[i] = make_double2((a.x * hv.x - a.y * hv.y) * scale, (a.x * hv.y + a.y * hv.x) * scale);
  }
}

__global__ void k_crop_c64(const double2* in, int mx, int my, float2* out) {
  const size_t n = (size_t)mx * my;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % mx), y = (int)(i / mx);
    const double2 v = in[(size_t)y * 2 * mx + x];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

static int blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b > 4864 ? 4864 : (b < 1 ? 1 : b));
}

// 2-D float64 FFT over `planes` stacked [planes][My][Mx] arrays (in place)
void fft64_2d_planes(double2* d, int Mx, int My, int planes, int dir, cudaStream_t st);

// lengths the float64 pencil FFT handles: 2^a 3^b, at most 1024
static bool fft64_length_ok(int L) {
  if (L < 1 || L > 1024) return false;
  while (L % 2 == 0) L /= 2;
  while (L % 3 == 0) L /= 3;
  return L == 1;
}

int apply_pupil_device(ls_plan* P, const float2* in, float2* out, int adjoint, double2* scratch, cudaStream_t st) {
  const int mx = P->mx, my = P->my, Mx = 2 * mx, My = 2 * my;
  const size_t n = (size_t)Mx * My;
  k_pad_c64<<<blocks_for(n), 256, 0, st>>>(in, mx, my, scratch);
  fft64_2d_planes(scratch, Mx, My, 1, -1, st);
  k_mul_transfer<<<blocks_for(n), 256, 0, st>>>(scratch, P->pupil_h, n, adjoint, 1.0 / (double)n);
  fft64_2d_planes(scratch, Mx, My, 1, +1, st);
  k_crop_c64<<<blocks_for((size_t)mx * my), 256, 0, st>>>(scratch, mx, my, out);
  LS_CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

}  // namespace lsgpu

using namespace lsgpu;

extern "C" {

int ls_incident_field(ls_plan* P, int n_views, const ls_c64* const* y_in, const double* k_in,
                      ls_c64* const* u_in, void* stream) {
  lsgpu::TraceRange trace_range("ls_incident_field");
  if (!P || n_views < 1 || !y_in || !u_in) { set_last_error("bad arguments"); return LS_EINVAL; }
  for (int q = 0; q < n_views; ++q)
    if (!y_in[q] || !u_in[q]) { set_last_error("null view pointer %d", q); return LS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const int nx = P->nx, ny = P->ny, nz = P->nz;
  if (!fft64_length_ok(nx) || !fft64_length_ok(ny)) {
    set_last_error("lateral grid %dx%d has no float64 FFT length", nx, ny);
    return LS_EUNSUPPORTED;
  }
  const size_t plane = (size_t)nx * ny, n = plane * nz;
  double2 *A = nullptr, *B = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&A, plane * sizeof(double2), st));
  LS_CUDA_TRY(cudaMallocAsync((void**)&B, n * sizeof(double2), st));
  for (int q = 0; q < n_views; ++q) {
    const double kx = k_in ? k_in[2 * q] : 0.0, ky = k_in ? k_in[2 * q + 1] : 0.0;
    k_demodulate<<<blocks_for(plane), 256, 0, st>>>((const float2*)y_in[q], nx, ny, P->h, kx, ky, A);
    fft64_2d_planes(A, nx, ny, 1, -1, st);
    k_spread_planes<<<blocks_for(n), 256, 0, st>>>(A, nx, ny, nz, P->h, P->kb, P->x_gamma, kx, ky, B);
    fft64_2d_planes(B, nx, ny, nz, +1, st);
    k_modulate_store<<<blocks_for(n), 256, 0, st>>>(B, nx, ny, nz, P->h, kx, ky, (float2*)u_in[q]);
  }
  LS_CUDA_TRY(cudaFreeAsync(A, st));
  LS_CUDA_TRY(cudaFreeAsync(B, st));
  LS_CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int ls_set_pupil(ls_plan* P, double k_cut, double distance) {
  if (!P) { set_last_error("null plan"); return LS_EINVAL; }
  if (k_cut <= 0) {
    cudaFree(P->pupil_h);
    P->pupil_h = nullptr;
    return LS_OK;
  }
  const int Mx = 2 * P->mx, My = 2 * P->my;
  if (!fft64_length_ok(Mx) || !fft64_length_ok(My)) {
    set_last_error("padded detector %dx%d has no float64 FFT length", My, Mx);
    return LS_EUNSUPPORTED;
  }
  if (!P->pupil_h) LS_CUDA_TRY(cudaMalloc(&P->pupil_h, (size_t)Mx * My * sizeof(double2)));
  k_pupil_transfer<<<blocks_for((size_t)Mx * My), 256>>>(Mx, My, P->h, P->kb, k_cut, distance, P->pupil_h);
  LS_CUDA_TRY(cudaDeviceSynchronize());
  return LS_OK;
}

int ls_apply_pupil(ls_plan* P, int n_views, const ls_c64* const* in, ls_c64* const* out, int adjoint, void* stream) {
  lsgpu::TraceRange trace_range("ls_apply_pupil");
  if (!P || n_views < 1 || !in || !out) { set_last_error("bad arguments"); return LS_EINVAL; }
  if (!P->pupil_h) { set_last_error("no pupil set (ls_set_pupil)"); return LS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  double2* scratch = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&scratch, (size_t)4 * P->mx * P->my * sizeof(double2), st));
  int rc = LS_OK;
  for (int q = 0; q < n_views && rc == LS_OK; ++q)
    rc = apply_pupil_device(P, (const float2*)in[q], (float2*)out[q], adjoint, scratch, st);
  LS_CUDA_TRY(cudaFreeAsync(scratch, st));
  return rc;
}

}  // extern "C"

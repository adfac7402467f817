// Proximal operator of lam TV + i_{>=0} (isotropic total variation, forward differences with a
// Neumann boundary) by the fast gradient projection method on the dual problem: the prox step of
// Alg. 1 (Sec. 4.2), evaluated with Beck and Teboulle's FGP as the paper does.  Each iteration is
// two element-wise stencil kernels over the [nz][ny][nx] grid:
//   primal:  x = max(z + lam div r, 0)
//   dual:    q = P_ball(r + step D x),  r = q + c_k (q - p),  p = q     (step = 1 / (12 lam))
// with p, r stored as three planes of N floats each and c_k = (t_k - 1) / t_{k+1} from the host.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "trace.h"

namespace lsgpu {

struct TvParams {
  int nx, ny, nz;
  size_t n;
  const float* z;
  float* x;
  const float* d;   // dual field read by the primal kernel: 3 planes of n
  float lam;
};

struct TvDualParams {
  int nx, ny, nz;
  size_t n;
  const float* x;
  float* p;         // 3 planes of n
  float* r;         // 3 planes of n
  float step, c;
};

__global__ void __launch_bounds__(256) k_tv_primal(TvParams a) {
  const size_t plane = (size_t)a.nx * a.ny;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < a.n; v += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(v % a.nx), iy = (int)((v / a.nx) % a.ny), iz = (int)(v / plane);
    const float* d0 = a.d;
    const float* d1 = a.d + a.n;
    const float* d2 = a.d + 2 * a.n;
    float div = 0.f;
    if (iz < a.nz - 1) div += d0[v];
    if (iz > 0) div -= d0[v - plane];
    if (iy < a.ny - 1) div += d1[v];
    if (iy > 0) div -= d1[v - a.nx];
    if (ix < a.nx - 1) div += d2[v];
    if (ix > 0) div -= d2[v - 1];
    a.x[v] = fmaxf(a.z[v] + a.lam * div, 0.f);
  }
}

__global__ void __launch_bounds__(256) k_tv_dual(TvDualParams a) {
  const size_t plane = (size_t)a.nx * a.ny;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < a.n; v += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(v % a.nx), iy = (int)((v / a.nx) % a.ny), iz = (int)(v / plane);
    const float xv = a.x[v];
    const float g0 = iz < a.nz - 1 ? a.x[v + plane] - xv : 0.f;
    const float g1 = iy < a.ny - 1 ? a.x[v + a.nx] - xv : 0.f;
    const float g2 = ix < a.nx - 1 ? a.x[v + 1] - xv : 0.f;
    float q0 = a.r[v] + a.step * g0;
    float q1 = a.r[v + a.n] + a.step * g1;
    float q2 = a.r[v + 2 * a.n] + a.step * g2;
    const float s = 1.f / fmaxf(sqrtf(q0 * q0 + q1 * q1 + q2 * q2), 1.f);
    q0 *= s; q1 *= s; q2 *= s;
    const float p0 = a.p[v], p1 = a.p[v + a.n], p2 = a.p[v + 2 * a.n];
    a.r[v] = q0 + a.c * (q0 - p0);
    a.r[v + a.n] = q1 + a.c * (q1 - p1);
    a.r[v + 2 * a.n] = q2 + a.c * (q2 - p2);
    a.p[v] = q0;
    a.p[v + a.n] = q1;
    a.p[v + 2 * a.n] = q2;
  }
}

static unsigned tv_blocks(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace lsgpu

using namespace lsgpu;

extern "C" int ls_prox_tv(const ls_grid* grid, const float* z, float* x, double lam, int iters, float* work,
                          void* stream) {
  lsgpu::TraceRange trace_range("ls_prox_tv");
  if (!grid || !z || !x || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || iters < 0) {
    set_last_error("bad arguments");
    return LS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)grid->nx * grid->ny * grid->nz;
  if (lam > 0 && iters > 0 && (const void*)z == (const void*)x) {
    set_last_error("z and x must not overlap (z is read in every iteration)");
    return LS_EINVAL;
  }
  TvParams pa{grid->nx, grid->ny, grid->nz, n, z, x, nullptr, (float)lam};
  if (!(lam > 0) || iters == 0) {
    // lam <= 0: the projection onto the non-negative orthant (div of a zero dual)
    float* zero = nullptr;
    if (lam > 0) {
      set_last_error("iters must be positive when lam > 0");
      return LS_EINVAL;
    }
    LS_CUDA_TRY(cudaMallocAsync((void**)&zero, 3 * n * sizeof(float), st));
    LS_CUDA_TRY(cudaMemsetAsync(zero, 0, 3 * n * sizeof(float), st));
    pa.d = zero;
    pa.lam = 0.f;
    k_tv_primal<<<tv_blocks(n), 256, 0, st>>>(pa);
    LS_CUDA_TRY(cudaGetLastError());
    LS_CUDA_TRY(cudaFreeAsync(zero, st));
    return LS_OK;
  }
  float* buf = work;
  if (!buf) LS_CUDA_TRY(cudaMallocAsync((void**)&buf, 6 * n * sizeof(float), st));
  float* p = buf;
  float* r = buf + 3 * n;
  LS_CUDA_TRY(cudaMemsetAsync(buf, 0, 6 * n * sizeof(float), st));
  TvDualParams da{grid->nx, grid->ny, grid->nz, n, x, p, r, (float)(1.0 / (12.0 * lam)), 0.f};
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    pa.d = r;
    k_tv_primal<<<tv_blocks(n), 256, 0, st>>>(pa);
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    da.c = (float)((t - 1.0) / tn);
    k_tv_dual<<<tv_blocks(n), 256, 0, st>>>(da);
    t = tn;
  }
  pa.d = p;
  k_tv_primal<<<tv_blocks(n), 256, 0, st>>>(pa);
  LS_CUDA_TRY(cudaGetLastError());
  if (!work) LS_CUDA_TRY(cudaFreeAsync(buf, st));
  return LS_OK;
}

// Proximal operator of lam sum_v ||H x (v)||_{S1} + i_{>=0}: the Hessian Schatten-norm regulariser
// named beside TV in Sec. 4.2, evaluated like the TV prox by the fast gradient projection method
// on the dual, whose variable is a field of symmetric 3 x 3 matrices constrained to the
// spectral-norm unit ball.  Per iteration two stencil kernels over the [nz][ny][nx] grid:
//   primal:  x = max(z - lam H^* W, 0)
//   dual:    Psi = P_ball(W + step H x),  W = Psi + c_k (Psi - Psi_prev),  Psi_prev = Psi
// with step = 1 / (144 lam) (||H||^2 <= 144) and c_k from the host.  H: D_aa = -D_a^T D_a (second
// difference, Neumann boundary), D_ab = D_b D_a for a != b, D_a the forward difference with zero on
// the last plane.  Matrix fields are six planes (zz, yy, xx, zy, zx, yx); the projection clips the
// eigenvalues of each voxel's matrix to [-1, 1] after a cyclic Jacobi eigen-decomposition (float32).
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "trace.h"

namespace lsgpu {

struct HsGeom {
  int n[3];        // extents of axes z, y, x
  size_t st[3];    // element strides of axes z, y, x
  size_t N;
};

__device__ __forceinline__ void hs_coords(const HsGeom& g, size_t v, int* c) {
  c[2] = (int)(v % g.n[2]);
  c[1] = (int)((v / g.n[2]) % g.n[1]);
  c[0] = (int)(v / ((size_t)g.n[2] * g.n[1]));
}

// (D_aa w)(v) = [v_a < n_a - 1] (w(v + e_a) - w(v)) - [v_a > 0] (w(v) - w(v - e_a))
__device__ __forceinline__ float hs_dd(const float* w, const HsGeom& g, size_t v, const int* c, int a) {
  const float wv = w[v];
  float r = 0.f;
  if (c[a] < g.n[a] - 1) r += w[v + g.st[a]] - wv;
  if (c[a] > 0) r -= wv - w[v - g.st[a]];
  return r;
}

// (D_b D_a x)(v), a != b
__device__ __forceinline__ float hs_dba(const float* x, const HsGeom& g, size_t v, const int* c, int a, int b) {
  if (c[a] >= g.n[a] - 1 || c[b] >= g.n[b] - 1) return 0.f;
  return x[v + g.st[a] + g.st[b]] - x[v + g.st[b]] - x[v + g.st[a]] + x[v];
}

// (D_a^T D_b^T w)(v), a != b: D^T p (u) = [u >= 1] p(u - e) - [u <= n - 2] p(u)
__device__ __forceinline__ float hs_dtt(const float* w, const HsGeom& g, size_t v, const int* c, int a, int b) {
  const bool am = c[a] >= 1, ak = c[a] <= g.n[a] - 2;
  const bool bm = c[b] >= 1, bk = c[b] <= g.n[b] - 2;
  float r = 0.f;
  if (am && bm) r += w[v - g.st[a] - g.st[b]];
  if (am && bk) r -= w[v - g.st[a]];
  if (ak && bm) r -= w[v - g.st[b]];
  if (ak && bk) r += w[v];
  return r;
}

__global__ void __launch_bounds__(256) k_hs_primal(HsGeom g, const float* z, const float* w, float lam, float* x) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < g.N; v += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    hs_coords(g, v, c);
    float hw = hs_dd(w, g, v, c, 0) + hs_dd(w + g.N, g, v, c, 1) + hs_dd(w + 2 * g.N, g, v, c, 2);
    hw += 2.f * (hs_dtt(w + 3 * g.N, g, v, c, 0, 1) + hs_dtt(w + 4 * g.N, g, v, c, 0, 2) +
                 hs_dtt(w + 5 * g.N, g, v, c, 1, 2));
    x[v] = fmaxf(z[v] - lam * hw, 0.f);
  }
}

// Eigen-decomposition of the symmetric matrix m (row-major 3 x 3) by cyclic Jacobi rotations
// (at most 10 sweeps); on return m's diagonal holds the eigenvalues and the columns of q the
// eigenvectors.
__device__ __forceinline__ void jacobi3(float (&m)[3][3], float (&q)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) q[i][j] = i == j ? 1.f : 0.f;
  for (int sweep = 0; sweep < 10; ++sweep) {
    const float off = fabsf(m[0][1]) + fabsf(m[0][2]) + fabsf(m[1][2]);
    const float dia = fabsf(m[0][0]) + fabsf(m[1][1]) + fabsf(m[2][2]);
    if (off <= 1e-7f * dia || off == 0.f) break;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int p = k == 2 ? 1 : 0, r = k == 0 ? 1 : 2;   // pairs (0,1), (0,2), (1,2)
      const float apq = m[p][r];
      if (fabsf(apq) <= 1e-12f * (fabsf(m[p][p]) + fabsf(m[r][r]))) continue;
      const float theta = (m[r][r] - m[p][p]) / (2.f * apq);
      const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
      const float cs = rsqrtf(fmaf(t, t, 1.f)), sn = t * cs;
      m[p][p] -= t * apq;
      m[r][r] += t * apq;
      m[p][r] = m[r][p] = 0.f;
      const int o = 3 - p - r;
      const float aop = m[o][p], aor = m[o][r];
      m[o][p] = m[p][o] = cs * aop - sn * aor;
      m[o][r] = m[r][o] = sn * aop + cs * aor;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float qp = q[i][p], qr = q[i][r];
        q[i][p] = cs * qp - sn * qr;
        q[i][r] = sn * qp + cs * qr;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_hs_dual(HsGeom g, const float* x, float* p, float* w, float step,
                                                 float cmom) {
  const size_t N = g.N;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
    int c[3];
    hs_coords(g, v, c);
    float h[6];
    h[0] = hs_dd(x, g, v, c, 0);
    h[1] = hs_dd(x, g, v, c, 1);
    h[2] = hs_dd(x, g, v, c, 2);
    h[3] = hs_dba(x, g, v, c, 0, 1);
    h[4] = hs_dba(x, g, v, c, 0, 2);
    h[5] = hs_dba(x, g, v, c, 1, 2);
    float m[3][3], q[3][3];
    float s[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k] = w[v + k * N] + step * h[k];
    m[0][0] = s[0]; m[1][1] = s[1]; m[2][2] = s[2];
    m[0][1] = m[1][0] = s[3];
    m[0][2] = m[2][0] = s[4];
    m[1][2] = m[2][1] = s[5];
    // spectral norm <= 1 already: a bound by the Frobenius norm skips the decomposition
    const float fro2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.f * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    if (fro2 > 1.f) {
      jacobi3(m, q);
      const float l0 = fminf(fmaxf(m[0][0], -1.f), 1.f), l1 = fminf(fmaxf(m[1][1], -1.f), 1.f),
                  l2 = fminf(fmaxf(m[2][2], -1.f), 1.f);
      // Q diag(l) Q^T
      s[0] = q[0][0] * q[0][0] * l0 + q[0][1] * q[0][1] * l1 + q[0][2] * q[0][2] * l2;
      s[1] = q[1][0] * q[1][0] * l0 + q[1][1] * q[1][1] * l1 + q[1][2] * q[1][2] * l2;
      s[2] = q[2][0] * q[2][0] * l0 + q[2][1] * q[2][1] * l1 + q[2][2] * q[2][2] * l2;
      s[3] = q[0][0] * q[1][0] * l0 + q[0][1] * q[1][1] * l1 + q[0][2] * q[1][2] * l2;
      s[4] = q[0][0] * q[2][0] * l0 + q[0][1] * q[2][1] * l1 + q[0][2] * q[2][2] * l2;
      s[5] = q[1][0] * q[2][0] * l0 + q[1][1] * q[2][1] * l1 + q[1][2] * q[2][2] * l2;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float prev = p[v + k * N];
      w[v + k * N] = s[k] + cmom * (s[k] - prev);
      p[v + k * N] = s[k];
    }
  }
}

static unsigned hs_blocks(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace lsgpu

using namespace lsgpu;

extern "C" int ls_prox_hs(const ls_grid* grid, const float* z, float* x, double lam, int iters, float* work,
                          void* stream) {
  lsgpu::TraceRange trace_range("ls_prox_hs");
  if (!grid || !z || !x || grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || iters < 0) {
    set_last_error("bad arguments");
    return LS_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  HsGeom g;
  g.n[0] = grid->nz; g.n[1] = grid->ny; g.n[2] = grid->nx;
  g.st[2] = 1; g.st[1] = (size_t)grid->nx; g.st[0] = (size_t)grid->nx * grid->ny;
  g.N = (size_t)grid->nx * grid->ny * grid->nz;
  const size_t n = g.N;
  if (!(lam > 0)) {
    float* zero = nullptr;
    LS_CUDA_TRY(cudaMallocAsync((void**)&zero, 6 * n * sizeof(float), st));
    LS_CUDA_TRY(cudaMemsetAsync(zero, 0, 6 * n * sizeof(float), st));
    k_hs_primal<<<hs_blocks(n), 256, 0, st>>>(g, z, zero, 0.f, x);
    LS_CUDA_TRY(cudaGetLastError());
    LS_CUDA_TRY(cudaFreeAsync(zero, st));
    return LS_OK;
  }
  if (iters == 0) { set_last_error("iters must be positive when lam > 0"); return LS_EINVAL; }
  if ((const void*)z == (const void*)x) {
    set_last_error("z and x must not overlap (z is read in every iteration)");
    return LS_EINVAL;
  }
  float* buf = work;
  if (!buf) LS_CUDA_TRY(cudaMallocAsync((void**)&buf, 12 * n * sizeof(float), st));
  float* p = buf;
  float* w = buf + 6 * n;
  LS_CUDA_TRY(cudaMemsetAsync(buf, 0, 12 * n * sizeof(float), st));
  const float step = (float)(1.0 / (144.0 * lam));
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    k_hs_primal<<<hs_blocks(n), 256, 0, st>>>(g, z, w, (float)lam, x);
    const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
    k_hs_dual<<<hs_blocks(n), 256, 0, st>>>(g, x, p, w, step, (float)((t - 1.0) / tn));
    t = tn;
  }
  k_hs_primal<<<hs_blocks(n), 256, 0, st>>>(g, z, p, (float)lam, x);
  LS_CUDA_TRY(cudaGetLastError());
  if (!work) LS_CUDA_TRY(cudaFreeAsync(buf, st));
  return LS_OK;
}

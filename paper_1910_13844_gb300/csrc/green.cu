// Plan-time construction (float64 on the GPU) of
//  * the Green spectrum Ghat = F_{2n}(g_t^m), g_t^m the reduced-padding kernel
//    of Proposition 1 built from samples of the closed-form spectrum of the
//    truncated Green function (Sec. 3.1, eqs. GreenL and GreenL2);
//  * the per-slice far-field kernels of eq. Gtild-1 and their 2-D spectra.
// Both are stored as complex64 for the hot path.
#include "green.cuh"

#include <math.h>

#include <map>
#include <mutex>
#include <utility>

namespace lsgpu {

// -------------------------------------------------------------- ghat_t
__device__ __forceinline__ double sinc_d(double x) {
  const double x2 = x * x;
  return fabs(x) < 1e-4 ? 1.0 - x2 / 6.0 + x2 * x2 / 120.0 : sin(x) / x;
}

// Spectrum of g_t (eq. GreenL, minus sign in front of the sinc term) at radial
// frequency w.  Written as
//   ghat_t(w) = R [sin(R d/2) sinc(R d/2) + i sinc(R d) - i e^{i k R} sinc(R w)] / (w + k),  d = w - k,
// which is the same function as eq. GreenL but has no 0/0 at w = k: there it
// gives eq. GreenL2, i (R/(2k) - e^{ikR} sin(kR)/(2k^2)).  With a = R d / 2 the first two terms
// need only sin a and cos a: sin(a) sinc(a) = sin(a)^2 / a and sinc(2a) = sinc(a) cos(a).
// skr, ckr = sin(kR), cos(kR).
__device__ double2 ghat_t(double w, double k, double R, double skr, double ckr) {
  const double a = 0.5 * R * (w - k);
  double sa, ca, sinc_a;
  if (fabs(a) < 1e-4) {
    const double a2 = a * a;
    sinc_a = 1.0 - a2 / 6.0 + a2 * a2 / 120.0;
    sa = a * sinc_a;
    ca = 1.0 - a2 / 2.0 + a2 * a2 / 24.0;
  } else {
    sincos(a, &sa, &ca);
    sinc_a = sa / a;
  }
  double re = R * sa * sinc_a;
  double im = R * sinc_a * ca;
  const double s = sinc_d(R * w);
  re += R * s * skr;
  im -= R * s * ckr;
  const double inv = 1.0 / (w + k);
  return make_double2(re * inv, im * inv);
}

__device__ __forceinline__ int centred(int q, int M) { return q > M / 2 ? q - M : q; }

// S[qz][qy][qx] = ghat_t(|delta .* ((p/2) c(q) - s)|), q on the 2n grid (Prop. 1 sub-lattice s)
__global__ void k_sample_sublattice(GreenBuildParams a, int sz, int sy, int sx, double2* S) {
  const size_t total = (size_t)a.Mx * a.My * a.Mz;
  const int half = a.p / 2;
  double skr, ckr;
  sincos(a.kb * a.R, &skr, &ckr);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int qx = (int)(i % a.Mx), qy = (int)((i / a.Mx) % a.My), qz = (int)(i / ((size_t)a.Mx * a.My));
    const double wx = a.dx * (half * centred(qx, a.Mx) - sx);
    const double wy = a.dy * (half * centred(qy, a.My) - sy);
    const double wz = a.dz * (half * centred(qz, a.Mz) - sz);
    S[i] = ghat_t(sqrt(wx * wx + wy * wy + wz * wz), a.kb, a.R, skr, ckr);
  }
}

// Phase factors of Prop. 1's sub-lattice shift s, one table per axis:
// ph[k] = exp(-2 pi i c(k) s / (n p)) for k < M on each axis (x, then y, then z), the turn count
// reduced exactly with integer arithmetic.
__global__ void k_prop1_phases(GreenBuildParams a, int sz, int sy, int sx, double2* ph) {
  const int m = a.Mx + a.My + a.Mz;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    int M = a.Mx, k = j, s = sx;
    if (j >= a.Mx + a.My) { M = a.Mz; k = j - a.Mx - a.My; s = sz; }
    else if (j >= a.Mx) { M = a.My; k = j - a.Mx; s = sy; }
    const int np = M / 2 * a.p;
    const double turns = (double)((long long)centred(k, M) * s % np) / np;
    double sn, cs;
    sincospi(-2.0 * turns, &sn, &cs);
    ph[j] = make_double2(cs, sn);
  }
}

// K[k] += scale * T[k] * ph_x[kx] ph_y[ky] ph_z[kz]
//   (= exp(-2 pi i (c(kx) sx/(nx p) + c(ky) sy/(ny p) + c(kz) sz/(nz p))), Prop. 1)
__global__ void k_prop1_accumulate(GreenBuildParams a, const double2* ph, const double2* T, double2* K,
                                   double scale) {
  const size_t total = (size_t)a.Mx * a.My * a.Mz;
  const double2* px = ph;
  const double2* py = ph + a.Mx;
  const double2* pz = ph + a.Mx + a.My;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % a.Mx), ky = (int)((i / a.Mx) % a.My), kz = (int)(i / ((size_t)a.Mx * a.My));
    const double2 e = zmul(pz[kz], zmul(py[ky], px[kx]));
    const double2 t = zmul(T[i], e);
    double2 acc = K[i];
    acc.x += scale * t.x;
    acc.y += scale * t.y;
    K[i] = acc;
  }
}

// Zero the Nyquist offset (storage index n) of each axis of the 2n grid.
__global__ void k_zero_nyquist(GreenBuildParams a, double2* K) {
  const size_t total = (size_t)a.Mx * a.My * a.Mz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % a.Mx), ky = (int)((i / a.Mx) % a.My), kz = (int)(i / ((size_t)a.Mx * a.My));
    if (kx == a.Mx / 2 || ky == a.My / 2 || kz == a.Mz / 2) K[i] = make_double2(0.0, 0.0);
  }
}

// Octant (kz <= nz, ky <= ny, kx <= nx) of Ghat, scaled by the hot path's 1/(8 nx ny nz).
__global__ void k_store_octant(GreenBuildParams a, const double2* Gh, float2* oct, double scale) {
  const int ox = a.Mx / 2 + 1, oy = a.My / 2 + 1, oz = a.Mz / 2 + 1;
  const size_t total = (size_t)ox * oy * oz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % ox), ky = (int)((i / ox) % oy), kz = (int)(i / ((size_t)ox * oy));
    const double2 g = Gh[((size_t)kz * a.My + ky) * a.Mx + kx];
    oct[i] = make_float2((float)(g.x * scale), (float)(g.y * scale));
  }
}

// Full (2nz)(2ny)(2nx) spectrum from the octant, undoing the hot-path scale.
__global__ void k_expand_octant(int nx, int ny, int nz, const float2* oct, float2* full, float unscale) {
  const int Mx = 2 * nx, My = 2 * ny, Mz = 2 * nz;
  const size_t total = (size_t)Mx * My * Mz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    int kx = (int)(i % Mx), ky = (int)((i / Mx) % My), kz = (int)(i / ((size_t)Mx * My));
    kx = kx <= nx ? kx : Mx - kx;
    ky = ky <= ny ? ky : My - ky;
    kz = kz <= nz ? kz : Mz - kz;
    const float2 g = oct[((size_t)kz * (ny + 1) + ky) * (nx + 1) + kx];
    full[i] = make_float2(g.x * unscale, g.y * unscale);
  }
}

// The octant unfolded along x for the dynamically scheduled z pass: gxz[kz][ky][kx] for kx in [0, 2nx)
// (Ghat is even in kx), kz in [0, nz], ky in [0, ny]: a tile of 16 consecutive kx of one (ky) row is
// contiguous in every kz plane, so one TMA copy fetches it.
__global__ void k_unfold_x(int nx, int ny, int nz, const float2* oct, float2* gxz) {
  const int Mx = 2 * nx;
  const size_t total = (size_t)Mx * (ny + 1) * (nz + 1);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % Mx);
    const size_t row = i / Mx;   // kz (ny + 1) + ky
    gxz[i] = oct[row * (nx + 1) + (kx <= nx ? kx : Mx - kx)];
  }
}

// -------------------------------------------------------------- far-field kernels
// K2[z][dy][dx] = h^3 g(h c(dx), h c(dy), x_gamma - z_c) with g = e^{i k r}/(4 pi r)
// (eq. def:Green, midpoint rule of eq. Gtild-1); zero at the Nyquist offsets.
__global__ void k_far_kernel(FarKernelParams a, double2* K2) {
  const int Mx = 2 * a.nx, My = 2 * a.ny;
  const size_t total = (size_t)Mx * My * a.nz;
  const double inv4pi = 0.079577471545947667884441881686257;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int dx = (int)(i % Mx), dy = (int)((i / Mx) % My), z = (int)(i / ((size_t)Mx * My));
    if (dx == a.nx || dy == a.ny) { K2[i] = make_double2(0.0, 0.0); continue; }
    const double X = a.h * centred(dx, Mx), Y = a.h * centred(dy, My);
    const double Z = a.x_gamma - a.h * (z - a.nz / 2 + 1);
    const double r = sqrt(X * X + Y * Y + Z * Z);
    double sn, cs;
    sincos(a.kb * r, &sn, &cs);
    const double m = a.h * a.h * a.h * inv4pi / r;
    K2[i] = make_double2(m * cs, m * sn);
  }
}

__global__ void k_to_c64(const double2* src, float2* dst, size_t n, double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)(src[i].x * scale), (float)(src[i].y * scale));
}

// -------------------------------------------------------------- float64 FFT (plan time)
// One CTA per pencil; the pencil (length L = 2^a 3^b, L <= 1024) is staged in
// shared memory and transformed in place by Stockham autosort stages of radix
// 4, 2 and 3.  dir = -1 forward, +1 inverse (unnormalised).
__device__ __forceinline__ void zdft(double2* v, int r, int dir) {
  if (r == 2) {
    double2 t = v[1];
    v[1] = zsub(v[0], t);
    v[0] = zadd(v[0], t);
  } else if (r == 4) {
    double2 s0 = zadd(v[0], v[2]), d0 = zsub(v[0], v[2]);
    double2 s1 = zadd(v[1], v[3]), d1 = zsub(v[1], v[3]);
    double2 d1r = dir < 0 ? make_double2(d1.y, -d1.x) : make_double2(-d1.y, d1.x);
    v[0] = zadd(s0, s1);
    v[2] = zsub(s0, s1);
    v[1] = zadd(d0, d1r);
    v[3] = zsub(d0, d1r);
  } else {  // 3
    const double h = 0.86602540378443864676;
    double2 s = zadd(v[1], v[2]), d = zsub(v[1], v[2]);
    double2 m = make_double2(v[0].x - 0.5 * s.x, v[0].y - 0.5 * s.y);
    double2 rr = dir < 0 ? make_double2(h * d.y, -h * d.x) : make_double2(-h * d.y, h * d.x);
    v[0] = zadd(v[0], s);
    v[1] = zadd(m, rr);
    v[2] = zsub(m, rr);
  }
}

__global__ void k_fft64(double2* data, int L, size_t elem_stride, int ninner, size_t inner_stride,
                        size_t outer_stride, int dir, const double2* __restrict__ tw) {
  extern __shared__ double2 zb[];
  double2* b0 = zb;
  double2* b1 = zb + L;
  const size_t pencil = blockIdx.x;
  const size_t base = (pencil / ninner) * outer_stride + (pencil % ninner) * inner_stride;
  for (int i = threadIdx.x; i < L; i += blockDim.x) b0[i] = data[base + (size_t)i * elem_stride];
  __syncthreads();
  int rest = L, Ns = 1;
  double2* src = b0;
  double2* dst = b1;
  while (rest > 1) {
    const int r = (rest % 4 == 0) ? 4 : (rest % 2 == 0 ? 2 : 3);
    const int m = L / r;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const int k = j % Ns;
      double2 v[4];
      for (int q = 0; q < r; ++q) {
        v[q] = src[j + q * m];
        if (q > 0) {
          // exp(dir 2 pi i k q / (Ns r)) = tw[k q L / (Ns r)] (conjugated for dir = +1)
          double2 w = tw[(size_t)k * q * (L / (Ns * r)) % L];
          if (dir > 0) w.y = -w.y;
          v[q] = zmul(v[q], w);
        }
      }
      zdft(v, r, dir);
      const int o = (j / Ns) * Ns * r + k;
      for (int q = 0; q < r; ++q) dst[o + q * Ns] = v[q];
    }
    __syncthreads();
    double2* tmp = src; src = dst; dst = tmp;
    Ns *= r;
    rest /= r;
  }
  for (int i = threadIdx.x; i < L; i += blockDim.x) data[base + (size_t)i * elem_stride] = src[i];
}

// exp(-2 pi i j / L), j < L, in float64
__global__ void k_twiddle64(int L, double2* w) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < L; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)j / (double)L, &sn, &cs);
    w[j] = make_double2(cs, sn);
  }
}

// Twiddle table of length L on the current device, built on first use and kept for the process
// (a few KB per length); the first build is synchronous so every stream may read it.
static const double2* twiddle64(int L, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, double2*> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({dev, L});
  if (it != cache.end()) return it->second;
  double2* w = nullptr;
  if (cudaMalloc((void**)&w, (size_t)L * sizeof(double2)) != cudaSuccess) return nullptr;
  k_twiddle64<<<(L + 127) / 128, 128, 0, st>>>(L, w);
  if (cudaStreamSynchronize(st) != cudaSuccess) { cudaFree(w); return nullptr; }
  cache[{dev, L}] = w;
  return w;
}

static void fft64_pass(double2* d, int L, size_t pencils, size_t elem_stride, int ninner, size_t inner_stride,
                       size_t outer_stride, int dir, cudaStream_t st) {
  const double2* tw = twiddle64(L, st);
  if (!tw) return;   // the allocation error is left for the caller's cudaGetLastError
  k_fft64<<<(unsigned)pencils, 128, 2 * L * sizeof(double2), st>>>(d, L, elem_stride, ninner, inner_stride,
                                                                    outer_stride, dir, tw);
}

// 3-D (or 2-D when Mz == 1) in-place float64 FFT of a [Mz][My][Mx] array.
void fft64_3d(double2* d, int Mx, int My, int Mz, int dir, cudaStream_t st) {
  // x: pencils are rows
  fft64_pass(d, Mx, (size_t)My * Mz, 1, 1, 0, Mx, dir, st);
  // y: pencils (z, x)
  fft64_pass(d, My, (size_t)Mx * Mz, Mx, Mx, 1, (size_t)Mx * My, dir, st);
  if (Mz > 1) fft64_pass(d, Mz, (size_t)Mx * My, (size_t)Mx * My, Mx * My, 1, 0, dir, st);
}

// 2-D in-place float64 FFT of `planes` stacked [My][Mx] arrays.
void fft64_2d_planes(double2* d, int Mx, int My, int planes, int dir, cudaStream_t st) {
  fft64_pass(d, Mx, (size_t)My * planes, 1, 1, 0, Mx, dir, st);
  fft64_pass(d, My, (size_t)Mx * planes, Mx, Mx, 1, (size_t)Mx * My, dir, st);
}

static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 9728 ? 9728 : (b < 1 ? 1 : b));
}

cudaError_t build_green_octant(const GreenBuildParams& a, double2* S, double2* K, float2* oct, cudaStream_t st) {
  const size_t total = (size_t)a.Mx * a.My * a.Mz;
  cudaError_t e = cudaMemsetAsync(K, 0, total * sizeof(double2), st);
  if (e != cudaSuccess) return e;
  const int half = a.p / 2;
  const int nx = a.Mx / 2, ny = a.My / 2, nz = a.Mz / 2;
  // (np)^{-3} = (8/p^3) * 1/((2nx)(2ny)(2nz)) folds F^{-1}_{2n}'s normalisation and Prop. 1's factor
  const double scale = 1.0 / ((double)a.p * a.p * a.p * (double)nx * ny * nz);
  double2* ph = nullptr;
  e = cudaMallocAsync((void**)&ph, (size_t)(a.Mx + a.My + a.Mz) * sizeof(double2), st);
  if (e != cudaSuccess) return e;
  for (int sz = 0; sz < half; ++sz)
    for (int sy = 0; sy < half; ++sy)
      for (int sx = 0; sx < half; ++sx) {
        k_sample_sublattice<<<grid_for(total), 256, 0, st>>>(a, sz, sy, sx, S);
        fft64_3d(S, a.Mx, a.My, a.Mz, +1, st);
        k_prop1_phases<<<(a.Mx + a.My + a.Mz + 127) / 128, 128, 0, st>>>(a, sz, sy, sx, ph);
        k_prop1_accumulate<<<grid_for(total), 256, 0, st>>>(a, ph, S, K, scale);
      }
  e = cudaFreeAsync(ph, st);
  if (e != cudaSuccess) return e;
  k_zero_nyquist<<<grid_for(total), 256, 0, st>>>(a, K);
  fft64_3d(K, a.Mx, a.My, a.Mz, -1, st);
  const size_t oct_n = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  k_store_octant<<<grid_for(oct_n), 256, 0, st>>>(a, K, oct, 1.0 / (8.0 * nx * ny * nz));
  return cudaGetLastError();
}

cudaError_t expand_octant(int nx, int ny, int nz, const float2* oct, float2* full, cudaStream_t st) {
  const size_t total = (size_t)8 * nx * ny * nz;
  k_expand_octant<<<grid_for(total), 256, 0, st>>>(nx, ny, nz, oct, full, (float)(8.0 * nx * ny * nz));
  return cudaGetLastError();
}

cudaError_t unfold_octant_x(int nx, int ny, int nz, const float2* oct, float2* gxz, cudaStream_t st) {
  const size_t total = (size_t)2 * nx * (ny + 1) * (nz + 1);
  k_unfold_x<<<grid_for(total), 256, 0, st>>>(nx, ny, nz, oct, gxz);
  return cudaGetLastError();
}

cudaError_t build_far_kernels(const FarKernelParams& a, double2* K2, float2* out, cudaStream_t st) {
  const size_t total = (size_t)4 * a.nx * a.ny * a.nz;
  k_far_kernel<<<grid_for(total), 256, 0, st>>>(a, K2);
  // 2-D FFT of every slice: x then y pencils, z stays
  fft64_2d_planes(K2, 2 * a.nx, 2 * a.ny, a.nz, -1, st);
  k_to_c64<<<grid_for(total), 256, 0, st>>>(K2, out, total, 1.0 / (4.0 * a.nx * a.ny));
  return cudaGetLastError();
}

}  // namespace lsgpu

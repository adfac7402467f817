// Plan-time builders (float64 on the GPU): Green spectrum octant and far-field kernel spectra.
#pragma once

#include "common.cuh"

namespace lsgpu {

struct GreenBuildParams {
  int Mx, My, Mz;      // 2n per axis
  int p;               // oversampling of Theorem 1 (even)
  double dx, dy, dz;   // delta_i = 2 pi / (p L_i)
  double kb, R;        // wavenumber, truncation radius (diagonal of Omega)
};

struct FarKernelParams {
  int nx, ny, nz;
  double h, kb, x_gamma;
};

// S, K: (2nz)(2ny)(2nx) double2 scratch; oct: (nz+1)(ny+1)(nx+1) float2 output scaled by 1/(8 nx ny nz).
cudaError_t build_green_octant(const GreenBuildParams& a, double2* S, double2* K, float2* oct, cudaStream_t st);
// full[(2nz)(2ny)(2nx)] = unscaled spectrum from the octant
cudaError_t expand_octant(int nx, int ny, int nz, const float2* oct, float2* full, cudaStream_t st);
// gxz[kz][ky][kx] = oct[kz][ky][fold(kx)] for kx < 2nx (the octant unfolded along x)
cudaError_t unfold_octant_x(int nx, int ny, int nz, const float2* oct, float2* gxz, cudaStream_t st);
// K2: nz (2ny)(2nx) double2 scratch; out: spectra scaled by 1/(4 nx ny)
cudaError_t build_far_kernels(const FarKernelParams& a, double2* K2, float2* out, cudaStream_t st);
void fft64_3d(double2* d, int Mx, int My, int Mz, int dir, cudaStream_t st);

}  // namespace lsgpu

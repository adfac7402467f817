// Parameter blocks and launchers of the solver and element-wise kernels (krylov.cu).
#pragma once

#include "common.cuh"
#include "passes.cuh"

namespace lsgpu {

enum ScalarPhase : int { PH_RESID = 0, PH_ALPHA = 1, PH_OMEGA = 2, PH_RHO = 3 };

// debug build: the index-check record of krylov.cu (debug_bounds.cuh)
unsigned bounds_site_krylov(bool clear);

struct UpdParams {
  SlotSel sel;
  size_t n, vstride;
  float2 *x, *r;
  const float2 *p, *s, *t, *rh;
  double* partials;
  int maxparts = 0;   // partial-sum blocks allocated per slot (0: not checked)
};

struct ScalarParams {
  SlotDev* slots;
  unsigned mask;
  int phase;
  const double* partials;   // [slot][nparts][4]
  int nparts;
};

struct PlaneWaveParams {
  int nx, ny, nz;
  double h;
  const double* k;          // device, 3 per view
  float2* const* out;       // device array of device pointers
  float2* tables = nullptr; // per-view 1-D phase factors (allocated by the launcher)
};

struct FarParams {
  SlotSel sel;
  int nx, ny, nz;
  float2* a2; size_t a2_stride;           // reduce: input slices; adjoint: output
  const float2* k2;                       // [nz][2ny][2nx], scaled by 1/(4 nx ny)
  float2* out; size_t out_stride;         // reduce output [2ny][2nx] per slot
  const float2* rhat; size_t rhat_stride; // adjoint input [2ny][2nx] per slot
};

struct PadParams {
  SlotSel sel;
  int nx, ny, mx, my, ox, oy;
  const float2* const* src;   // device array of per-slot detector arrays
  float2* dst; size_t dst_stride;
};

struct GradParams {
  size_t n;
  int nslots;
  const float2* const* u;     // device array of forward fields
  const float2* w; size_t w_stride;
  const float* c;             // device, per-slot weights
  float* grad;
};

struct ResidualParams {
  size_t count;
  const float2* const* pred;
  const float2* const* meas;
  float2* const* res;
  double* partials;           // [view][nblocks][4]
};

void launch_update(const UpdParams& a, int nblocks, int nslots, cudaStream_t st);
void launch_scalar(const ScalarParams& a, int nslots, cudaStream_t st);
void launch_count(const SlotDev* slots, int nslots, int* out, cudaStream_t st);
void launch_zero_shadow(const SlotDev* slots, int slot, float2* rh, size_t n, cudaStream_t st);
void launch_inner(const ResidualParams& a, int nblocks, int nviews, cudaStream_t st);
cudaError_t launch_plane_waves(const PlaneWaveParams& a, int nviews, cudaStream_t st);
void launch_potential(const float* dn, size_t count, double eta_b, double kb, float* f, cudaStream_t st);
void launch_far_reduce(const FarParams& a, int nslots, cudaStream_t st);
void launch_far_adjoint_mul(const FarParams& a, int nslots, cudaStream_t st);
void launch_pad_detector(const PadParams& a, int nslots, cudaStream_t st);
void launch_gradient(const GradParams& a, cudaStream_t st);
void launch_residual(const ResidualParams& a, int nblocks, int nviews, cudaStream_t st);

}  // namespace lsgpu

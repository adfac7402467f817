// ls_matvec_noalloc: the operator y = x - G (f .* x) for callers that must
// not allocate device memory.
//
// ls_matvec keeps its FFT intermediates in the plan's workspace, which the
// plan allocates (cudaMalloc) the first time it is needed.  Some callers
// cannot let that happen: a process that has handed all of its device memory
// to its own pool at start-up, or a latency-bound loop in which a cudaMalloc
// or cudaFree (both may synchronise the device) would stall other work.  This
// entry point uses instead one static device array that is part of the
// library image; every GPU that loads the library's module for it holds it
// until the process exits.
//
// With lazy module loading the array is only reserved when its module is
// first touched.  ls_plan_create does that (noalloc_setup below, on the
// plan's device, while it allocates its own memory anyway) and keeps the
// array's device address in the plan, so this call neither loads a module nor
// looks anything up.  A plan belongs to the CUDA context it was created in;
// after a context is destroyed (cudaDeviceReset), plans from before are
// invalid and a new plan repeats the set-up.
#include "engine.h"

using namespace lsgpu;

namespace {

// Size of the static scratch: the two FFT intermediates of one operator
// application, 2N + 4N complex64 values (48 N bytes) for an N-voxel grid.
constexpr size_t kNoallocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(float2)];

}  // namespace

namespace lsgpu {

// Device address of the static scratch on the current device.  The name
// g_noalloc_scratch is only a host-side stand-in for the array; the address a
// kernel can use is the one the runtime reports for the current device.
int noalloc_setup(void** addr) {
  *addr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(addr, g_noalloc_scratch);
  if (e != cudaSuccess) {
    *addr = nullptr;
    set_last_error("static scratch of ls_matvec_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LS_ENOMEM : LS_ECUDA;
  }
  return LS_OK;
}

}  // namespace lsgpu

extern "C" int ls_matvec_noalloc(const ls_plan* P, const float* f, const ls_c64* x, ls_c64* y, int adjoint,
                                 void* stream) {
  if (!P || !f || !x || !y) {
    set_last_error("ls_matvec_noalloc: null argument");
    return LS_EINVAL;
  }
  const size_t a1n = (size_t)2 * P->nx * P->ny * P->nz;   // [nz][ny][2nx]
  const size_t a2n = (size_t)4 * P->nx * P->ny * P->nz;   // [nz][2ny][2nx]
  const size_t need = (a1n + a2n) * sizeof(float2);
  if (need > kNoallocScratchBytes) {
    set_last_error("ls_matvec_noalloc: a %dx%dx%d grid needs %zu bytes of scratch, the static scratch holds %zu "
                   "(48 bytes per voxel: at most %zu voxels)", P->nx, P->ny, P->nz, need, kNoallocScratchBytes,
                   kNoallocScratchBytes / 48);
    return LS_EINVAL;
  }
  if (!P->noalloc_scratch) {
    set_last_error("ls_matvec_noalloc: the static scratch could not be set up when the plan was created (%s)",
                   ls_status_string(P->noalloc_rc));
    return P->noalloc_rc ? P->noalloc_rc : LS_ECUDA;
  }
  int dev = -1;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != P->device) {
    set_last_error("ls_matvec_noalloc: the current device is %d, the plan was created on device %d", dev, P->device);
    return LS_EINVAL;
  }
  float2* a1 = static_cast<float2*>(P->noalloc_scratch);
  float2* a2 = a1 + a1n;
  cudaStream_t st = (cudaStream_t)stream;

  // Every scratch element that a pass reads is written earlier in the same
  // call, so nothing has to be cleared between calls.
  SlotSel sel;
  sel.slots = nullptr;
  sel.mask = 0;
  sel.f_default = f;
  sel.adj_default = adjoint ? 1 : 0;
  sel.runs = nullptr;
  sel.nslots = 1;

  FxParams fx = {};
  fx.sel = sel;
  fx.nx = P->nx;
  fx.rows = P->ny * P->nz;
  fx.mode = FX_F_TIMES;
  fx.src = (const float2*)x;
  fx.vstride = P->N;
  fx.dst = a1;
  fx.dst_stride = a1n;
  fx.tw2 = P->tw2_x;
  P->px.fx(fx, 1, st);

  StridedParams fy = {};
  fy.sel = sel;
  fy.ncont = 2 * P->nx;
  fy.planes = P->nz;
  fy.out_o = 0;
  fy.out_m = P->ny;
  fy.src = a1; fy.src_stride = a1n;
  fy.dst = a2; fy.dst_stride = a2n;
  fy.src_plane = (size_t)P->ny * 2 * P->nx;
  fy.dst_plane = (size_t)2 * P->ny * 2 * P->nx;
  fy.tw = P->tw_y;
  P->py.fy(fy, 1, st);

  ZParams z = {};
  z.sel = sel;
  z.nx = P->nx; z.ny = P->ny; z.nz = P->nz;
  z.a2 = a2; z.a2_stride = a2n;
  z.gocta = P->gocta;
  z.twa = P->twa_z;
  z.twb = P->twb_z;
  z.zwa = P->zwa_z;
  z.zwb = P->zwb_z;
  P->pz.z(z, 1, st);

  StridedParams iy = fy;
  iy.src = a2; iy.src_stride = a2n;
  iy.dst = a1; iy.dst_stride = a1n;
  iy.src_plane = (size_t)2 * P->ny * 2 * P->nx;
  iy.dst_plane = (size_t)P->ny * 2 * P->nx;
  P->py.iy(iy, 1, st);

  IxParams ix = {};
  ix.sel = sel;
  ix.nx = P->nx;
  ix.rows = P->ny * P->nz;
  ix.mode = IX_MATVEC;
  ix.src = a1; ix.src_stride = a1n;
  ix.in0 = (const float2*)x;
  ix.out0 = (float2*)y;
  ix.vstride = 0;
  ix.out_o = 0; ix.out_m = P->nx;
  ix.tw2 = P->tw2_x;
  P->px.ix(ix, 1, st);

  LS_CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

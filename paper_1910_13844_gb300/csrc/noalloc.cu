// ls_matvec_noalloc: the operator y = x - G (f .* x) for callers that must
// not allocate device memory.
//
// ls_matvec keeps its FFT intermediates in the plan's workspace, which the
// plan allocates (cudaMalloc) the first time it is needed.  Some callers
// cannot let that happen: a process that has handed all of its device memory
// to its own pool at start-up, or a latency-bound loop in which a cudaMalloc
// or cudaFree (both may synchronise the device) would stall other work.  This
// entry point uses instead one static device array that is part of the
// library image; every GPU that loads the library holds it until the process
// exits.
#include <mutex>

#include "engine.h"

using namespace lsgpu;

namespace {

// Size of the static scratch: the two FFT intermediates of one operator
// application, 2N + 4N complex64 values (48 N bytes) for an N-voxel grid.
constexpr size_t kNoallocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchBytes / sizeof(float2)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device, looked up once
// per device (the name g_noalloc_scratch is only a host-side stand-in).
int scratch_on_current_device(float2** out) {
  int dev = -1;
  LS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("device ordinal %d out of range for the static scratch table", dev);
    return LS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    LS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = static_cast<float2*>(p);
  }
  *out = g_scratch_addr[dev];
  return LS_OK;
}

}  // namespace

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
  float2* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc != LS_OK) return rc;
  float2* a1 = scratch;
  float2* a2 = scratch + a1n;
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

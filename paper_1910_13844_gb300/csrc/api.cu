// C ABI of the LS library: plans, the batched BiCGStab engine and the
// forward / far-field / gradient entry points (see include/ls.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "engine.h"

namespace lsgpu {

static const double kPi = 3.14159265358979323846;

static thread_local char g_last_error[512] = "";

void set_last_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
}

static bool fft_length_ok(int L) {
  switch (L) {
    case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 144: case 192: case 256: case 288: case 384:
      return true;
    default: return false;
  }
}

static bool pass_for_length(int L, PassLaunch* t, cudaError_t* setup_err) {
  switch (L) {
#define LS_CASE(LL) case LL: *t = pass_table_##LL(); *setup_err = pass_setup_##LL(); return true;
    LS_CASE(16) LS_CASE(24) LS_CASE(32) LS_CASE(48) LS_CASE(64)
    LS_CASE(96) LS_CASE(128) LS_CASE(144) LS_CASE(192) LS_CASE(256) LS_CASE(288) LS_CASE(384)
#undef LS_CASE
    default: return false;
  }
}

// Per-thread twiddle rows of the z pass: twa[t*R1 + k1] (t < R2) and twb[t*R2 + j1] (t < R1),
// both exp(-2 pi i t k / L).
static int make_z_twiddles(int L, int R1, int R2, float2** twa, float2** twb) {
  const double pi = 3.14159265358979323846;
  std::vector<float2> a(L), b(L);
  for (int t = 0; t < R2; ++t)
    for (int k = 0; k < R1; ++k) {
      const int j = (t * k) % L;
      a[t * R1 + k] = make_float2((float)cos(-2.0 * pi * j / L), (float)sin(-2.0 * pi * j / L));
    }
  for (int t = 0; t < R1; ++t)
    for (int k = 0; k < R2; ++k) {
      const int j = (t * k) % L;
      b[t * R2 + k] = make_float2((float)cos(-2.0 * pi * j / L), (float)sin(-2.0 * pi * j / L));
    }
  LS_CUDA_TRY(cudaMalloc(twa, L * sizeof(float2)));
  LS_CUDA_TRY(cudaMemcpy(*twa, a.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
  LS_CUDA_TRY(cudaMalloc(twb, L * sizeof(float2)));
  LS_CUDA_TRY(cudaMemcpy(*twb, b.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
  return LS_OK;
}

// Twiddles computed in double on the host, rounded once to float.
static int make_twiddles(int L, int R1, int R2, float2** tw, float2** tw2) {
  std::vector<float2> a(L), b(L);
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < L; ++j) a[j] = make_float2((float)cos(-2.0 * pi * j / L), (float)sin(-2.0 * pi * j / L));
  for (int k1 = 0; k1 < R1; ++k1)
    for (int n2 = 0; n2 < R2; ++n2) {
      const int j = (k1 * n2) % L;
      b[k1 * R2 + n2] = a[j];
    }
  if (tw) {
    LS_CUDA_TRY(cudaMalloc(tw, L * sizeof(float2)));
    LS_CUDA_TRY(cudaMemcpy(*tw, a.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
  }
  if (tw2) {
    LS_CUDA_TRY(cudaMalloc(tw2, L * sizeof(float2)));
    LS_CUDA_TRY(cudaMemcpy(*tw2, b.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
  }
  return LS_OK;
}

void slot_defaults(const ls_plan* P, SlotDev& s, const float* f, int adjoint) {
  memset(&s, 0, sizeof(s));
  s.f = f;
  s.flags = SLOT_RESID;
  s.adjoint = adjoint;
  s.first = 1;
  s.status = LS_OK;
  s.max_iter = P->opt.max_iter;
  s.max_restarts = P->opt.max_restarts;
  s.tol = P->opt.tol;
  s.alpha = s.omega = s.rho = make_double2(1.0, 0.0);
  s.alpha_f = s.omega_f = make_float2(1.f, 0.f);
  s.beta_f = make_float2(0.f, 0.f);
}

void engine_release(Engine& e) {
  if (e.iter_graph) cudaGraphExecDestroy(e.iter_graph);
  if (e.cap_stream) cudaStreamDestroy(e.cap_stream);
  cudaFree(e.vec); cudaFree(e.a1); cudaFree(e.a2); cudaFree(e.far); cudaFree(e.ucache);
  cudaFree(e.partials); cudaFree(e.slots_d); cudaFreeHost(e.slots_h);
  cudaFree(e.counts_d); cudaFreeHost(e.counts_h); cudaFree(e.ptrs_d); cudaFree(e.kvec_d); cudaFree(e.weights_d);
  e = Engine();
}

// The driver's tensor-map encoder, looked up once through the runtime (null if unavailable).
using TmapEncode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static TmapEncode tmap_encoder() {
  static TmapEncode encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<TmapEncode>(fn);
  }();
  return encode;
}

// TMA map of the x-unfolded Green array for the dynamically scheduled z pass: floats [nz+1][ny+1][4nx],
// box of 16 complex columns x 1 row x (nz+1) planes, 128-byte swizzle.
static bool encode_gxz_map(ls_plan* P) {
  TmapEncode encode = tmap_encoder();
  if (!encode || !P->gxz || P->nz + 1 > 256 || (2 * P->nx) % 16 != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)4 * P->nx, (cuuint64_t)P->ny + 1, (cuuint64_t)P->nz + 1};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * P->nx * sizeof(float2),
                                 (cuuint64_t)2 * P->nx * (P->ny + 1) * sizeof(float2)};
  const cuuint32_t box[3] = {32, 1, (cuuint32_t)P->nz + 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(&P->gxz_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, P->gxz, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA map of the engine's A2 buffers for the z pass: floats [slot][nz][2ny][4nx], box of 16 complex
// columns x 1 row x nz planes of one slot, 128-byte swizzle.  Returns false when the driver entry
// point is unavailable or the shape does not fit a box (the z pass then stages with cp.async).
static bool encode_a2_map(const ls_plan* P, Engine& e) {
  TmapEncode encode = tmap_encoder();
  if (!encode || P->nz > 256 || (2 * P->nx) % 16 != 0) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)4 * P->nx, (cuuint64_t)2 * P->ny, (cuuint64_t)P->nz, (cuuint64_t)e.cap};
  const cuuint64_t strides[3] = {(cuuint64_t)2 * P->nx * sizeof(float2),
                                 (cuuint64_t)2 * P->nx * 2 * P->ny * sizeof(float2),
                                 (cuuint64_t)e.a2_stride * sizeof(float2)};
  const cuuint32_t box[4] = {32, 1, (cuuint32_t)P->nz, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return encode(&e.a2_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, e.a2, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int max_parts(const ls_plan* P) {
  const int rows = P->ny * P->nz;
  const int ix_blocks = (rows + P->px.rows_per_cta_contig - 1) / P->px.rows_per_cta_contig;
  return std::max(ix_blocks, 512);
}

// Test-only failure injection: the next g_fail_allocs engine allocations fail (ls_debug_inject).
static std::atomic<long long> g_fail_allocs{0};

static bool injected_alloc_failure() {
  long long n = g_fail_allocs.load();
  while (n > 0)
    if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
  return false;
}

// Allocates the per-slot arrays of a workspace for nslots slots into e (which must be empty).
// On failure everything allocated so far is released and e is left empty.
static int engine_alloc(ls_plan* P, Engine& e, int nslots) {
  if (injected_alloc_failure()) {
    set_last_error("workspace allocation for %d views failed (injected)", nslots);
    return LS_ENOMEM;
  }
  const int cap = nslots;
  e.cap = cap;
  e.N = P->N;
  e.a1_stride = (size_t)2 * P->nx * P->ny * P->nz;
  e.a2_stride = (size_t)4 * P->nx * P->ny * P->nz;
  e.maxparts = max_parts(P);
  int rc = LS_OK;
  auto dev = [&](void** p, size_t bytes) {
    if (rc != LS_OK) return;
    const cudaError_t err = cudaMalloc(p, bytes);
    if (err != cudaSuccess) {
      *p = nullptr;
      set_last_error("workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(err));
      rc = err == cudaErrorMemoryAllocation ? LS_ENOMEM : LS_ECUDA;
    }
  };
  auto host = [&](void** p, size_t bytes) {
    if (rc != LS_OK) return;
    const cudaError_t err = cudaMallocHost(p, bytes);
    if (err != cudaSuccess) {
      *p = nullptr;
      set_last_error("pinned allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(err));
      rc = err == cudaErrorMemoryAllocation ? LS_ENOMEM : LS_ECUDA;
    }
  };
  dev((void**)&e.vec, (size_t)NVEC * cap * e.N * sizeof(float2));
  dev((void**)&e.a1, (size_t)cap * e.a1_stride * sizeof(float2));
  dev((void**)&e.a2, (size_t)cap * e.a2_stride * sizeof(float2));
  dev((void**)&e.far, (size_t)cap * P->mx * P->my * sizeof(float2));
  dev((void**)&e.partials, (size_t)cap * e.maxparts * 4 * sizeof(double));
  dev((void**)&e.slots_d, (size_t)cap * sizeof(SlotDev));
  host((void**)&e.slots_h, (size_t)cap * sizeof(SlotDev));
  dev((void**)&e.counts_d, 8 * sizeof(int));
  host((void**)&e.counts_h, 8 * sizeof(int));
  dev((void**)&e.ptrs_d, (size_t)4 * cap * sizeof(void*));
  dev((void**)&e.kvec_d, (size_t)6 * cap * sizeof(double));   // 3 per view, twice (built-in plane waves)
  dev((void**)&e.weights_d, (size_t)cap * sizeof(float));
  if (rc == LS_OK && cudaMemset(e.counts_d, 0, 8 * sizeof(int)) != cudaSuccess) rc = LS_ECUDA;
  if (rc == LS_OK && cudaMemset(e.slots_d, 0, (size_t)cap * sizeof(SlotDev)) != cudaSuccess) rc = LS_ECUDA;
  if (rc != LS_OK) {
    engine_release(e);
    return rc;
  }
  memset(e.slots_h, 0, (size_t)cap * sizeof(SlotDev));
  memset(e.counts_h, 0, 8 * sizeof(int));
  e.a2_map_ok = encode_a2_map(P, e) ? 1 : 0;
  return LS_OK;
}

int engine_reserve(ls_plan* P, int nslots) {
  Engine& e = P->eng;
  if (nslots > kMaxLaunchSlots) {
    set_last_error("at most %d views per call (got %d)", kMaxLaunchSlots, nslots);
    return LS_EINVAL;
  }
  if (nslots <= e.cap) return LS_OK;
  // keep the slot-independent pieces; reallocate the per-slot arrays (the old ones are freed first,
  // so that the new ones can use their memory)
  cudaStream_t cs = e.cap_stream;
  e.cap_stream = nullptr;
  engine_release(e);
  int rc = engine_alloc(P, e, nslots);
  e.cap_stream = cs;
  if (rc != LS_OK) return rc;
  if (!e.cap_stream) LS_CUDA_TRY(cudaStreamCreateWithFlags(&e.cap_stream, cudaStreamNonBlocking));
  return LS_OK;
}

int engine_reserve_ucache(ls_plan* P, int nslots) {
  Engine& e = P->eng;
  if (e.ucache && e.ucache_cap >= nslots) return LS_OK;
  cudaFree(e.ucache);
  e.ucache = nullptr;
  LS_CUDA_TRY(cudaMalloc(&e.ucache, (size_t)nslots * e.N * sizeof(float2)));
  e.ucache_cap = nslots;
  return LS_OK;
}

void** engine_ptr_table(ls_plan* P, int table) { return P->eng.ptrs_d + (size_t)table * P->eng.cap; }

int engine_upload_ptrs(ls_plan* P, int table, const void* const* host_ptrs, int n, cudaStream_t st) {
  LS_CUDA_TRY(cudaMemcpyAsync(engine_ptr_table(P, table), host_ptrs, (size_t)n * sizeof(void*),
                              cudaMemcpyHostToDevice, st));
  return LS_OK;
}

// ------------------------------------------------------------------ pass parameter helpers
static SlotSel sel_slots(ls_plan* P, unsigned mask) {
  SlotSel s;
  s.slots = P->eng.slots_d;
  s.mask = mask;
  s.f_default = nullptr;
  s.adj_default = 0;
  s.runs = nullptr;
  s.nslots = 0;
  return s;
}

static FxParams fx_base(ls_plan* P, SlotSel sel, int rows) {
  FxParams a;
  memset(&a, 0, sizeof(a));
  a.sel = sel;
  a.nx = P->nx;
  a.rows = rows;
  a.vstride = P->eng.N;
  a.dst = P->eng.a1;
  a.dst_stride = P->eng.a1_stride;
  a.tw2 = P->tw2_x;
  a.views_fastest = P->tune_fx_views_fastest;
  a.bulk = P->tune_fx_bulk;
  a.sms = P->sms;
  a.err = P->eng.counts_d + 4;
  return a;
}

static StridedParams fy_base(ls_plan* P, SlotSel sel, const float2* src, size_t sstride, float2* dst,
                             size_t dstride, int planes) {
  StridedParams a;
  memset(&a, 0, sizeof(a));
  a.sel = sel;
  a.ncont = 2 * P->nx;
  a.planes = planes;
  a.out_o = 0;
  a.out_m = P->ny;
  a.src = src; a.src_stride = sstride;
  a.dst = dst; a.dst_stride = dstride;
  a.src_plane = (size_t)P->ny * 2 * P->nx;        // FY input plane [ny][2nx]
  a.dst_plane = (size_t)2 * P->ny * 2 * P->nx;    // FY output plane [2ny][2nx]
  a.tw = P->tw_y;
  a.wide = P->tune_strided_wide;
  return a;
}

static SlotSel counted(ls_plan* P, SlotSel s, int kind) {
  ls_plan* o = prof_owner(P);
  s.runs = o->prof.runs_d ? o->prof.runs_d + kind : nullptr;
  return s;
}

static void matvec_core(ls_plan* P, SlotSel sel, int nslots, const FxParams& fx_in, IxParams ix, cudaStream_t st) {
  Engine& e = P->eng;
  FxParams fx = fx_in;
  fx.sel = counted(P, fx.sel, LS_K_FX);
  fx.dbg_probe = P->inj_bounds_probe;
  timed(P, LS_K_FX, nslots, st, [&] { P->px.fx(fx, nslots, st); });
  StridedParams fy = fy_base(P, counted(P, sel, LS_K_FY), e.a1, e.a1_stride, e.a2, e.a2_stride, P->nz);
  timed(P, LS_K_FY, nslots, st, [&] { P->py.fy(fy, nslots, st); });
  ZParams z = {};
  z.tmap = e.a2_map;
  z.use_tma = e.a2_map_ok && P->tune_z_tma;
  z.slot0 = e.slot0;
  z.err = e.counts_d + 4;
  z.sel = counted(P, sel, LS_K_Z);
  z.nx = P->nx; z.ny = P->ny; z.nz = P->nz;
  z.a2 = e.a2; z.a2_stride = e.a2_stride;
  z.gocta = P->gocta;
  z.twa = P->twa_z;
  z.twb = P->twb_z;
  z.alt = P->tune_z_split && P->zwa2_z ? 1 : 0;
  z.zwa = z.alt ? P->zwa2_z : P->zwa_z;
  z.zwb = z.alt ? P->zwb2_z : P->zwb_z;
  z.wait_ns = (unsigned long long)P->inj_z_wait_ns;
  z.sms = P->sms;
  if (P->tune_z_persist >= 0 && 2 * nslots > P->tune_views) {
    z.persist = P->tune_z_persist;
  } else {
    const int form = nslots <= kZSmallBatch ? P->pz.zauto_small : P->pz.zauto_large;
    z.persist = form == 2 && !P->gxz_ok ? 0 : form;
  }
  z.gmap = P->gxz_map;
  z.gmap_ok = P->gxz_ok;
  z.ctr = reinterpret_cast<unsigned*>(e.counts_d + 6);
  z.stall = P->inj_z_stall;
  timed(P, LS_K_Z, nslots, st, [&] { P->pz.z(z, nslots, st); });
  StridedParams iy = fy_base(P, counted(P, sel, LS_K_IY), e.a2, e.a2_stride, e.a1, e.a1_stride, P->nz);
  iy.src_plane = (size_t)2 * P->ny * 2 * P->nx;
  iy.dst_plane = (size_t)P->ny * 2 * P->nx;
  timed(P, LS_K_IY, nslots, st, [&] { P->py.iy(iy, nslots, st); });
  ix.sel = counted(P, sel, LS_K_IX);
  ix.nx = P->nx;
  ix.rows = P->ny * P->nz;
  ix.src = e.a1; ix.src_stride = e.a1_stride;
  ix.tw2 = P->tw2_x;
  ix.prefetch = P->tune_ix_prefetch;
  ix.maxparts = e.maxparts;
  timed(P, LS_K_IX, nslots, st, [&] { P->px.ix(ix, nslots, st); });
}

static int ix_blocks(const ls_plan* P) {
  const int rows = P->ny * P->nz;
  return (rows + P->px.rows_per_cta_contig - 1) / P->px.rows_per_cta_contig;
}

static int upd_blocks(const ls_plan* P, int nslots) {
  // enough blocks to fill the GPU for a single slot, fewer per slot when many run together
  const size_t n4 = P->N / 2;
  int want = nslots >= 8 ? 128 : 512;
  const int max_useful = (int)((n4 + 255) / 256);
  return std::max(1, std::min(want, max_useful));
}

void seq_resid(ls_plan* P, int nslots, cudaStream_t st) {
  Engine& e = P->eng;
  SlotSel sel = sel_slots(P, SLOT_RESID);
  FxParams fx = fx_base(P, sel, P->ny * P->nz);
  fx.mode = FX_F_TIMES;
  fx.src = e.vptr(V_X);
  IxParams ix;
  memset(&ix, 0, sizeof(ix));
  ix.mode = IX_RESID;
  ix.in0 = e.vptr(V_X);
  ix.in1 = e.vptr(V_B);
  ix.out0 = e.vptr(V_R);
  ix.out1 = e.vptr(V_RH);
  ix.vstride = e.N;
  ix.partials = e.partials;
  matvec_core(P, sel, nslots, fx, ix, st);
  if (P->inj_zero_shadow_view >= 0 && P->inj_zero_shadow_view < nslots)
    launch_zero_shadow(e.slots_d, P->inj_zero_shadow_view, e.vptr(V_RH), e.N, st);
  ScalarParams sc{e.slots_d, SLOT_RESID, PH_RESID, e.partials, ix_blocks(P)};
  timed(P, LS_K_SCALAR, nslots, st, [&] { launch_scalar(sc, nslots, st); });
}

void seq_iter(ls_plan* P, int nslots, cudaStream_t st) {
  Engine& e = P->eng;
  SlotSel sel = sel_slots(P, SLOT_ITER);
  // v = A p with p = r + beta (p - omega v)
  {
    FxParams fx = fx_base(P, sel, P->ny * P->nz);
    fx.mode = FX_BICG_P;
    fx.src = e.vptr(V_R);
    fx.vp = e.vptr(V_P);
    fx.vv = e.vptr(V_V);
    IxParams ix;
    memset(&ix, 0, sizeof(ix));
    ix.mode = IX_BICG_V;
    ix.in0 = e.vptr(V_P);
    ix.in1 = e.vptr(V_RH);
    ix.out0 = e.vptr(V_V);
    ix.vstride = e.N;
    ix.partials = e.partials;
    matvec_core(P, sel, nslots, fx, ix, st);
    ScalarParams sc{e.slots_d, SLOT_ITER, PH_ALPHA, e.partials, ix_blocks(P)};
    timed(P, LS_K_SCALAR, nslots, st, [&] { launch_scalar(sc, nslots, st); });
  }
  // t = A s with s = r - alpha v
  {
    FxParams fx = fx_base(P, sel, P->ny * P->nz);
    fx.mode = FX_BICG_S;
    fx.src = e.vptr(V_R);
    fx.vv = e.vptr(V_V);
    fx.vs = e.vptr(V_S);
    IxParams ix;
    memset(&ix, 0, sizeof(ix));
    ix.mode = IX_BICG_T;
    ix.in0 = e.vptr(V_S);
    ix.out0 = e.vptr(V_T);
    ix.vstride = e.N;
    ix.partials = e.partials;
    matvec_core(P, sel, nslots, fx, ix, st);
    ScalarParams sc{e.slots_d, SLOT_ITER, PH_OMEGA, e.partials, ix_blocks(P)};
    timed(P, LS_K_SCALAR, nslots, st, [&] { launch_scalar(sc, nslots, st); });
  }
  // x += alpha p + omega s ; r = s - omega t
  {
    UpdParams u;
    u.sel = counted(P, sel, LS_K_UPDATE);
    u.n = e.N;
    u.vstride = e.N;
    u.x = e.vptr(V_X); u.r = e.vptr(V_R);
    u.p = e.vptr(V_P); u.s = e.vptr(V_S); u.t = e.vptr(V_T); u.rh = e.vptr(V_RH);
    u.partials = e.partials;
    u.maxparts = e.maxparts;
    const int nb = upd_blocks(P, nslots);
    timed(P, LS_K_UPDATE, nslots, st, [&] { launch_update(u, nb, nslots, st); });
    ScalarParams sc{e.slots_d, SLOT_ITER, PH_RHO, e.partials, nb};
    timed(P, LS_K_SCALAR, nslots, st, [&] { launch_scalar(sc, nslots, st); });
  }
}

void seq_iter_chunked(ls_plan* P, int nslots, cudaStream_t st) {
  const int c = P->tune_views_per_launch;
  if (c <= 0 || c >= nslots) {
    seq_iter(P, nslots, st);
    return;
  }
  for (int s0 = 0; s0 < nslots; s0 += c) {
    ls_plan v = plan_slot_view(P, s0);
    seq_iter(&v, std::min(c, nslots - s0), st);
  }
}

// far[s] = G~ (f x_s) for the selected slots (eq. Gtild-1)
void seq_far(ls_plan* P, int nslots, unsigned mask, cudaStream_t st) {
  Engine& e = P->eng;
  SlotSel sel = sel_slots(P, mask);
  FxParams fx = fx_base(P, sel, P->ny * P->nz);
  fx.mode = FX_F_TIMES;
  fx.src = e.vptr(V_X);
  timed(P, LS_K_FX, nslots, st, [&] { P->px.fx(fx, nslots, st); });
  StridedParams fy = fy_base(P, sel, e.a1, e.a1_stride, e.a2, e.a2_stride, P->nz);
  timed(P, LS_K_FY, nslots, st, [&] { P->py.fy(fy, nslots, st); });
  FarParams fr;
  memset(&fr, 0, sizeof(fr));
  fr.sel = sel;
  fr.nx = P->nx; fr.ny = P->ny; fr.nz = P->nz;
  fr.a2 = e.a2; fr.a2_stride = e.a2_stride;
  fr.k2 = P->k2hat;
  fr.out = e.a1; fr.out_stride = e.a1_stride;
  timed(P, LS_K_FAR, nslots, st, [&] { launch_far_reduce(fr, nslots, st); });
  // 2-D inverse transform of the single plane, cropped to the detector window
  StridedParams iy = fy_base(P, sel, e.a1, e.a1_stride, e.a2, e.a2_stride, 1);
  iy.src_plane = 0; iy.dst_plane = 0;
  iy.out_o = P->oy; iy.out_m = P->my;
  timed(P, LS_K_FAR, nslots, st, [&] { P->py.iy(iy, nslots, st); });
  IxParams ix;
  memset(&ix, 0, sizeof(ix));
  ix.sel = sel;
  ix.mode = IX_STORE;
  ix.nx = P->nx;
  ix.rows = P->my;
  ix.src = e.a2; ix.src_stride = e.a2_stride;
  ix.out0 = e.far;
  ix.vstride = (size_t)P->mx * P->my;
  ix.out_o = P->ox; ix.out_m = P->mx;
  ix.tw2 = P->tw2_x;
  timed(P, LS_K_FAR, nslots, st, [&] { P->px.ix(ix, nslots, st); });
}

// b_s = G~^H r_s for the selected slots; r_dev_table holds one device pointer per slot
void seq_far_adjoint(ls_plan* P, int nslots, const float2* const* r_dev_table, unsigned mask, cudaStream_t st) {
  Engine& e = P->eng;
  SlotSel sel = sel_slots(P, mask);
  PadParams pd;
  pd.sel = sel;
  pd.nx = P->nx; pd.ny = P->ny; pd.mx = P->mx; pd.my = P->my; pd.ox = P->ox; pd.oy = P->oy;
  pd.src = r_dev_table;
  pd.dst = e.vptr(V_V);
  pd.dst_stride = e.N;
  timed(P, LS_K_FAR, nslots, st, [&] { launch_pad_detector(pd, nslots, st); });
  FxParams fx = fx_base(P, sel, P->ny);
  fx.mode = FX_COPY;
  fx.src = e.vptr(V_V);
  fx.dst = e.a2;
  fx.dst_stride = e.a2_stride;
  timed(P, LS_K_FAR, nslots, st, [&] { P->px.fx(fx, nslots, st); });
  StridedParams fy = fy_base(P, sel, e.a2, e.a2_stride, e.a1, e.a1_stride, 1);
  timed(P, LS_K_FAR, nslots, st, [&] { P->py.fy(fy, nslots, st); });
  FarParams fr;
  memset(&fr, 0, sizeof(fr));
  fr.sel = sel;
  fr.nx = P->nx; fr.ny = P->ny; fr.nz = P->nz;
  fr.a2 = e.a2; fr.a2_stride = e.a2_stride;
  fr.k2 = P->k2hat;
  fr.rhat = e.a1; fr.rhat_stride = e.a1_stride;
  timed(P, LS_K_FAR, nslots, st, [&] { launch_far_adjoint_mul(fr, nslots, st); });
  StridedParams iy = fy_base(P, sel, e.a2, e.a2_stride, e.a1, e.a1_stride, P->nz);
  iy.src_plane = (size_t)2 * P->ny * 2 * P->nx;
  iy.dst_plane = (size_t)P->ny * 2 * P->nx;
  timed(P, LS_K_IY, nslots, st, [&] { P->py.iy(iy, nslots, st); });
  IxParams ix;
  memset(&ix, 0, sizeof(ix));
  ix.sel = sel;
  ix.mode = IX_STORE;
  ix.nx = P->nx;
  ix.rows = P->ny * P->nz;
  ix.src = e.a1; ix.src_stride = e.a1_stride;
  ix.out0 = e.vptr(V_B);
  ix.vstride = e.N;
  ix.out_o = 0; ix.out_m = P->nx;
  ix.tw2 = P->tw2_x;
  ix.prefetch = P->tune_ix_prefetch;
  timed(P, LS_K_IX, nslots, st, [&] { P->px.ix(ix, nslots, st); });
}

int ensure_iter_graph(ls_plan* P, int nslots) {
  Engine& e = P->eng;
  // the captured launches carry the plan's launch variants: recapture when ls_autotune changed them
  const int variant = P->tune_z_tma | P->tune_ix_prefetch << 1 | P->tune_fx_views_fastest << 2 |
                      (P->inj_z_stall || P->inj_z_wait_ns ? 1 << 3 : 0) | P->tune_z_split << 4 |
                      P->tune_strided_wide << 5 | (P->tune_z_persist & 3) << 6 | P->tune_fx_bulk << 8 |
                      (P->tune_views_per_launch & 0x7ff) << 9 | (P->tune_views & 0x7ff) << 20;
  if (e.iter_graph && e.iter_graph_slots == nslots && e.iter_graph_variant == variant) return LS_OK;
  if (e.iter_graph) {
    cudaGraphExecDestroy(e.iter_graph);
    e.iter_graph = nullptr;
  }
  cudaGraph_t g;
  LS_CUDA_TRY(cudaStreamBeginCapture(e.cap_stream, cudaStreamCaptureModeThreadLocal));
  seq_iter_chunked(P, nslots, e.cap_stream);
  LS_CUDA_TRY(cudaStreamEndCapture(e.cap_stream, &g));
  cudaError_t err = cudaGraphInstantiate(&e.iter_graph, g, 0);
  cudaGraphDestroy(g);
  LS_CUDA_TRY(err);
  e.iter_graph_slots = nslots;
  e.iter_graph_variant = variant;
  return LS_OK;
}

ls_plan plan_slot_view(const ls_plan* P, int s0) {
  ls_plan v;
  v.nx = P->nx; v.ny = P->ny; v.nz = P->nz; v.N = P->N; v.kb = P->kb; v.h = P->h; v.opt = P->opt;
  v.mx = P->mx; v.my = P->my; v.ox = P->ox; v.oy = P->oy; v.x_gamma = P->x_gamma;
  v.px = P->px; v.py = P->py; v.pz = P->pz;
  v.tw2_x = P->tw2_x; v.tw_y = P->tw_y;
  v.twa_z = P->twa_z; v.twb_z = P->twb_z; v.zwa_z = P->zwa_z; v.zwb_z = P->zwb_z;
  v.zwa2_z = P->zwa2_z; v.zwb2_z = P->zwb2_z;
  v.tune_z_split = P->tune_z_split; v.tune_strided_wide = P->tune_strided_wide; v.tune_z_persist = P->tune_z_persist;
  v.tune_fx_bulk = P->tune_fx_bulk;
  v.tune_views_per_launch = P->tune_views_per_launch;
  v.tune_views = P->tune_views;
  v.gocta = P->gocta; v.k2hat = P->k2hat; v.p_built = P->p_built;
  v.gxz = P->gxz; v.gxz_map = P->gxz_map; v.gxz_ok = P->gxz_ok;
  v.device = P->device; v.sms = P->sms;
  v.tune_z_tma = P->tune_z_tma; v.tune_ix_prefetch = P->tune_ix_prefetch;
  v.tune_fx_views_fastest = P->tune_fx_views_fastest;
  v.inj_z_stall = P->inj_z_stall; v.inj_z_wait_ns = P->inj_z_wait_ns; v.inj_bounds_probe = P->inj_bounds_probe;
  const Engine& e = P->eng;
  Engine& w = v.eng;
  w = e;
  w.vec = e.vec + (size_t)s0 * e.N;
  w.a1 = e.a1 + (size_t)s0 * e.a1_stride;
  w.a2 = e.a2 + (size_t)s0 * e.a2_stride;
  w.far = e.far + (size_t)s0 * P->mx * P->my;
  w.ucache = e.ucache ? e.ucache + (size_t)s0 * e.N : nullptr;
  w.partials = e.partials + (size_t)s0 * e.maxparts * 4;
  w.slots_d = e.slots_d + s0;
  w.slots_h = e.slots_h + s0;
  w.ptrs_d = e.ptrs_d + s0;
  w.kvec_d = e.kvec_d + 3 * (size_t)s0;
  w.weights_d = e.weights_d + s0;
  w.slot0 = e.slot0 + s0;
  w.iter_graph = nullptr;
  w.cap_stream = nullptr;
  v.prof_parent = const_cast<ls_plan*>(prof_owner(const_cast<ls_plan*>(P)));
  return v;
}

ls_plan* plan_clone_shared(const ls_plan* P) {
  ls_plan* c = new ls_plan();
  c->nx = P->nx; c->ny = P->ny; c->nz = P->nz; c->N = P->N; c->kb = P->kb; c->h = P->h; c->opt = P->opt;
  c->mx = P->mx; c->my = P->my; c->ox = P->ox; c->oy = P->oy; c->x_gamma = P->x_gamma;
  c->px = P->px; c->py = P->py; c->pz = P->pz;
  c->tw2_x = P->tw2_x; c->tw_y = P->tw_y;
  c->twa_z = P->twa_z; c->twb_z = P->twb_z; c->zwa_z = P->zwa_z; c->zwb_z = P->zwb_z;
  c->zwa2_z = P->zwa2_z; c->zwb2_z = P->zwb2_z;
  c->tune_z_split = P->tune_z_split; c->tune_strided_wide = P->tune_strided_wide; c->tune_z_persist = P->tune_z_persist;
  c->tune_fx_bulk = P->tune_fx_bulk;
  c->tune_views_per_launch = P->tune_views_per_launch;
  c->tune_views = P->tune_views;
  c->gocta = P->gocta; c->k2hat = P->k2hat; c->p_built = P->p_built;
  c->gxz = P->gxz; c->gxz_map = P->gxz_map; c->gxz_ok = P->gxz_ok;
  c->device = P->device; c->sms = P->sms;
  c->tune_z_tma = P->tune_z_tma; c->tune_ix_prefetch = P->tune_ix_prefetch;
  c->tune_fx_views_fastest = P->tune_fx_views_fastest;
  c->owns_shared = false;
  return c;
}

int tune_matvec(ls_plan* P, const float* f, int n, cudaStream_t st) {
  Engine& e = P->eng;
  for (int q = 0; q < n; ++q) {
    slot_defaults(P, e.slots_h[q], f, 0);
    e.slots_h[q].flags = SLOT_AUX;
  }
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_d, e.slots_h, (size_t)n * sizeof(SlotDev), cudaMemcpyHostToDevice, st));
  SlotSel sel = sel_slots(P, SLOT_AUX);
  FxParams fx = fx_base(P, sel, P->ny * P->nz);
  fx.mode = FX_F_TIMES;
  fx.src = e.vptr(V_X);
  IxParams ix;
  memset(&ix, 0, sizeof(ix));
  ix.mode = IX_MATVEC;
  ix.in0 = e.vptr(V_X);
  ix.out0 = e.vptr(V_R);
  ix.vstride = e.N;
  matvec_core(P, sel, n, fx, ix, st);
  LS_CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int tune_forward(ls_plan* P, const float* f, int n, cudaStream_t st) {
  Engine& e = P->eng;
  LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_X), e.vptr(V_B), (size_t)n * e.N * sizeof(float2), cudaMemcpyDeviceToDevice,
                              st));
  for (int q = 0; q < n; ++q) slot_defaults(P, e.slots_h[q], f, 0);
  return engine_solve(P, n, st);
}

int engine_solve(ls_plan* P, int nslots, cudaStream_t st) {
  TraceRange range("solve");
  Engine& e = P->eng;
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_d, e.slots_h, (size_t)nslots * sizeof(SlotDev), cudaMemcpyHostToDevice, st));
  // the z pass's error word (a TMA wait that gave up) covers this solve only
  LS_CUDA_TRY(cudaMemsetAsync(e.counts_d + 4, 0, sizeof(int), st));
  const bool graphs = P->opt.use_graphs != 0 && !P->prof.on;
  if (graphs) {
    int rc = ensure_iter_graph(P, nslots);
    if (rc != LS_OK) return rc;
  }
  const int chunk = P->opt.check_every > 0 ? P->opt.check_every : 2;
  long long max_rounds = (long long)P->opt.max_iter * (P->opt.max_restarts + 2) / chunk + 16;
  if (P->inj_max_rounds >= 0) max_rounds = std::min(max_rounds, P->inj_max_rounds);
  for (long long round = 0; round < max_rounds; ++round) {
    timed(P, LS_K_OTHER, nslots, st, [&] { launch_count(e.slots_d, nslots, e.counts_d, st); });
    LS_CUDA_TRY(cudaMemcpyAsync(e.counts_h, e.counts_d, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
    prof_resolve(P, false);
    if (e.counts_h[4]) {
      set_last_error("a TMA copy of the z pass or a bulk copy of the first pass did not complete within its time limit");
      return LS_ECUDA;
    }
    const int n_iter = e.counts_h[0], n_resid = e.counts_h[1];
    if (n_iter == 0 && n_resid == 0) break;
    if (n_resid > 0) {
      seq_resid(P, nslots, st);
      continue;
    }
    for (int k = 0; k < chunk; ++k) {
      if (graphs) {
        LS_CUDA_TRY(cudaGraphLaunch(e.iter_graph, st));
      } else {
        seq_iter_chunked(P, nslots, st);
      }
    }
    LS_CUDA_TRY(cudaGetLastError());
  }
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_h, e.slots_d, (size_t)nslots * sizeof(SlotDev), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  return LS_OK;
}

cudaEvent_t prof_event(ls_plan* P) {
  if (P->prof.pool.empty()) {
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    return ev;
  }
  cudaEvent_t ev = P->prof.pool.back();
  P->prof.pool.pop_back();
  return ev;
}

void prof_resolve(ls_plan* P, bool wait) {
  Profiler& pr = P->prof;
  size_t keep = 0;
  for (size_t i = 0; i < pr.pending.size(); ++i) {
    Profiler::Pending& q = pr.pending[i];
    if (wait) cudaEventSynchronize(q.b);
    if (cudaEventQuery(q.b) == cudaSuccess) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, q.a, q.b);
      pr.ms[q.kind] += ms;
      pr.launches[q.kind] += 1;
      pr.slot_passes[q.kind] += q.slots;
      pr.pool.push_back(q.a);
      pr.pool.push_back(q.b);
    } else {
      pr.pending[keep++] = q;
    }
  }
  pr.pending.resize(keep);
}

// far[q] <- P far[q] for the engine's detector buffers of slots [0, n) (no-op without a pupil)
static int pupil_on_far(ls_plan* P, int n, cudaStream_t st) {
  if (!P->pupil_h) return LS_OK;
  double2* scratch = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&scratch, (size_t)4 * P->mx * P->my * sizeof(double2), st));
  const size_t M = (size_t)P->mx * P->my;
  int rc = LS_OK;
  for (int q = 0; q < n && rc == LS_OK; ++q)
    rc = apply_pupil_device(P, P->eng.far + q * M, P->eng.far + q * M, 0, scratch, st);
  LS_CUDA_TRY(cudaFreeAsync(scratch, st));
  return rc;
}

// r'_q = P^H r_q into the engine's detector buffers (returns a host table of their pointers in tab)
static int pupil_adjoint_residuals(ls_plan* P, int n, const ls_c64* const* r, std::vector<const void*>& tab,
                                   cudaStream_t st) {
  tab.assign(n, nullptr);
  const size_t M = (size_t)P->mx * P->my;
  if (!P->pupil_h) {
    for (int q = 0; q < n; ++q) tab[q] = r[q];
    return LS_OK;
  }
  double2* scratch = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&scratch, (size_t)4 * M * sizeof(double2), st));
  int rc = LS_OK;
  for (int q = 0; q < n && rc == LS_OK; ++q) {
    rc = apply_pupil_device(P, (const float2*)r[q], P->eng.far + q * M, 1, scratch, st);
    tab[q] = P->eng.far + q * M;
  }
  LS_CUDA_TRY(cudaFreeAsync(scratch, st));
  return rc;
}

static int worst_status(const Engine& e, int nslots, ls_stats* stats) {
  int worst = LS_OK;
  for (int s = 0; s < nslots; ++s) {
    const SlotDev& sd = e.slots_h[s];
    int st = sd.status;
    if (sd.flags & (SLOT_ITER | SLOT_RESID)) st = LS_TIMEOUT;
    if (stats) {
      stats[s].status = st;
      stats[s].iterations = sd.iters;
      stats[s].restarts = sd.restarts;
      stats[s].matvecs = sd.matvecs;
      stats[s].rel_residual = sd.bnorm2 > 0 ? sqrt(sd.rnorm2 / sd.bnorm2) : 0.0;
      stats[s].true_rel_residual = sd.bnorm2 > 0 ? sqrt(sd.true_rnorm2 / sd.bnorm2) : 0.0;
    }
    if (st != LS_OK && (worst == LS_OK || st == LS_BREAKDOWN || st == LS_TIMEOUT)) worst = st;
  }
  return worst;
}

}  // namespace lsgpu

using namespace lsgpu;

// ====================================================================== C ABI
extern "C" {

void ls_default_options(ls_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->tol = 1e-6;
  opt->max_iter = 1000;
  opt->oversample_p = 4;
  opt->det_mx = 0;
  opt->det_my = 0;
  opt->x_gamma = 0.0;
  opt->max_restarts = 4;
  opt->check_every = 0;
  opt->use_graphs = 1;
  opt->cone_sin_theta = 0.0;
}

const char* ls_status_string(int status) {
  switch (status) {
    case LS_OK: return "LS_OK";
    case LS_EINVAL: return "LS_EINVAL: invalid argument";
    case LS_ENOMEM: return "LS_ENOMEM: device allocation failed";
    case LS_ECUDA: return "LS_ECUDA: CUDA runtime error";
    case LS_NOT_CONVERGED: return "LS_NOT_CONVERGED: max_iter reached";
    case LS_BREAKDOWN: return "LS_BREAKDOWN: BiCGStab breakdown";
    case LS_TIMEOUT: return "LS_TIMEOUT: the solve loop ended with views still running";
    case LS_PENDING: return "LS_PENDING: request still running";
    case LS_EAGAIN: return "LS_EAGAIN: request cannot fit the memory budget";
    case LS_ENOTFOUND: return "LS_ENOTFOUND: unknown ticket";
    case LS_EUNSUPPORTED: return "LS_EUNSUPPORTED: grid size without an FFT length";
    default: return "unknown status";
  }
}

const char* ls_last_error(void) { return g_last_error; }

int ls_profile(ls_plan* P, int enable, ls_kernel_times* out) {
  if (!P) { set_last_error("null plan"); return LS_EINVAL; }
  prof_resolve(P, true);
  if (!P->prof.runs_d) {
    LS_CUDA_TRY(cudaMalloc(&P->prof.runs_d, LS_K_COUNT * sizeof(unsigned long long)));
    LS_CUDA_TRY(cudaMemset(P->prof.runs_d, 0, LS_K_COUNT * sizeof(unsigned long long)));
  }
  unsigned long long runs[LS_K_COUNT];
  LS_CUDA_TRY(cudaDeviceSynchronize());
  LS_CUDA_TRY(cudaMemcpy(runs, P->prof.runs_d, sizeof(runs), cudaMemcpyDeviceToHost));
  if (out) {
    for (int k = 0; k < LS_K_COUNT; ++k) {
      out->ms[k] = P->prof.ms[k];
      out->launches[k] = P->prof.launches[k];
      out->slot_passes[k] = P->prof.slot_passes[k];
      out->active_slot_passes[k] = (long long)runs[k];
    }
  }
  if (enable) {
    for (int k = 0; k < LS_K_COUNT; ++k) P->prof.ms[k] = 0, P->prof.launches[k] = 0, P->prof.slot_passes[k] = 0;
    LS_CUDA_TRY(cudaMemset(P->prof.runs_d, 0, LS_K_COUNT * sizeof(unsigned long long)));
  }
  P->prof.on = enable != 0;
  return LS_OK;
}

size_t ls_workspace_bytes(const ls_grid* g, int n_views) {
  if (!g || n_views < 1) return 0;
  const size_t N = (size_t)g->nx * g->ny * g->nz;
  const size_t per_slot = (NVEC + 2 + 4) * N * sizeof(float2) + (size_t)g->nx * g->ny * sizeof(float2);
  const size_t shared = (size_t)(g->nx + 1) * (g->ny + 1) * (g->nz + 1) * sizeof(float2) +
                        (size_t)4 * N * sizeof(float2);
  return shared + per_slot * (size_t)n_views;
}

int ls_plan_create(const ls_grid* grid, int padding, double k_b, double voxel, const ls_options* opt,
                   ls_plan** out) {
  lsgpu::TraceRange trace_range("ls_plan_create");
  if (!grid || !out) { set_last_error("null argument"); return LS_EINVAL; }
  *out = nullptr;
  if (padding != 2) { set_last_error("storage padding must be 2 (Prop. 1)"); return LS_EINVAL; }
  if (!(k_b > 0) || !(voxel > 0)) { set_last_error("k_b and voxel must be positive"); return LS_EINVAL; }
  if (!(k_b * voxel < kPi)) { set_last_error("Theorem 1 needs k_b h < pi"); return LS_EINVAL; }
  const int L[3] = {2 * grid->nx, 2 * grid->ny, 2 * grid->nz};
  for (int i = 0; i < 3; ++i)
    if (!fft_length_ok(L[i])) {
      set_last_error("grid %dx%dx%d: 2n = %d has no FFT length", grid->nx, grid->ny, grid->nz, L[i]);
      return LS_EUNSUPPORTED;
    }
  ls_plan* P = new ls_plan();
  P->nx = grid->nx; P->ny = grid->ny; P->nz = grid->nz;
  P->N = (size_t)P->nx * P->ny * P->nz;
  P->kb = k_b;
  P->h = voxel;
  if (opt) P->opt = *opt; else ls_default_options(&P->opt);
  if (P->opt.tol <= 0) P->opt.tol = 1e-6;
  if (P->opt.max_iter <= 0) P->opt.max_iter = 1000;
  if (P->opt.oversample_p <= 0) P->opt.oversample_p = 4;
  if (P->opt.max_restarts < 0) P->opt.max_restarts = 0;
  if (!(P->opt.cone_sin_theta >= 0.0 && P->opt.cone_sin_theta <= 1.0)) {
    set_last_error("cone_sin_theta must lie in [0, 1]");
    delete P;
    return LS_EINVAL;
  }
  P->mx = P->opt.det_mx > 0 ? P->opt.det_mx : P->nx;
  P->my = P->opt.det_my > 0 ? P->opt.det_my : P->ny;
  if (P->mx > P->nx || P->my > P->ny || ((P->nx - P->mx) & 1) || ((P->ny - P->my) & 1)) {
    set_last_error("detector must satisfy m <= n with n - m even");
    delete P;
    return LS_EINVAL;
  }
  P->ox = (P->nx - P->mx) / 2;
  P->oy = (P->ny - P->my) / 2;
  P->x_gamma = P->opt.x_gamma > 0 ? P->opt.x_gamma : 0.75 * P->nz * P->h;
  int rc = LS_OK;
  cudaError_t se = cudaSuccess;
  if (cudaGetDevice(&P->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess) {
    set_last_error("no current CUDA device");
    delete P;
    return LS_ECUDA;
  }
  // ls_matvec_noalloc's static scratch: its address is looked up (and its module loaded) here,
  // while creating a plan allocates anyway, so that the no-allocation entry point never does
  P->noalloc_rc = noalloc_setup(&P->noalloc_scratch);
  if (!pass_for_length(L[0], &P->px, &se) || se != cudaSuccess ||
      !pass_for_length(L[1], &P->py, &se) || se != cudaSuccess ||
      !pass_for_length(L[2], &P->pz, &se) || se != cudaSuccess) {
    set_last_error("pass setup failed: %s", cudaGetErrorString(se));
    delete P;
    return LS_ECUDA;
  }
  rc = make_twiddles(L[0], P->px.r1, P->px.r2, nullptr, &P->tw2_x);
  if (rc == LS_OK) rc = make_twiddles(L[1], P->py.r1, P->py.r2, &P->tw_y, nullptr);
  if (rc == LS_OK) rc = make_z_twiddles(L[2], P->pz.r1, P->pz.r2, &P->twa_z, &P->twb_z);
  if (rc == LS_OK && P->pz.zalt_ok)
    rc = make_z_twiddles(L[2], P->pz.zr1b, P->pz.zr2b, &P->zwa2_z, &P->zwb2_z);
  if (rc == LS_OK) {
    if (P->pz.zr1 == P->pz.r1 && P->pz.zr2 == P->pz.r2) {
      P->zwa_z = P->twa_z;
      P->zwb_z = P->twb_z;
    } else {
      rc = make_z_twiddles(L[2], P->pz.zr1, P->pz.zr2, &P->zwa_z, &P->zwb_z);
    }
  }
  if (rc == LS_OK) {
    if (cudaMalloc(&P->gocta, (size_t)(P->nx + 1) * (P->ny + 1) * (P->nz + 1) * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&P->k2hat, (size_t)4 * P->N * sizeof(float2)) != cudaSuccess) {
      set_last_error("allocation of the Green spectrum failed");
      rc = LS_ENOMEM;
    }
  }
  // the x-unfolded Green array of the dynamically scheduled z pass (where that pass exists); without
  // it the z pass runs in its other forms
  if (rc == LS_OK && P->pz.zdyn_ok && P->nz + 1 <= 256 && (2 * P->nx) % 16 == 0) {
    if (cudaMalloc(&P->gxz, (size_t)2 * P->nx * (P->ny + 1) * (P->nz + 1) * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      P->gxz = nullptr;
    }
    P->gxz_ok = encode_gxz_map(P) ? 1 : 0;
  }
  if (rc == LS_OK) rc = ls_green_spectrum(P, P->opt.oversample_p, nullptr, nullptr);
  if (rc == LS_OK) {
    double2* scratch = nullptr;
    if (cudaMalloc(&scratch, (size_t)4 * P->N * sizeof(double2)) != cudaSuccess) {
      set_last_error("far-field scratch allocation failed");
      rc = LS_ENOMEM;
    } else {
      FarKernelParams fk{P->nx, P->ny, P->nz, P->h, P->kb, P->x_gamma};
      cudaError_t e = build_far_kernels(fk, scratch, P->k2hat, nullptr);
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
      cudaFree(scratch);
      if (e != cudaSuccess) { set_last_error("far-field kernels: %s", cudaGetErrorString(e)); rc = LS_ECUDA; }
    }
  }
  if (rc != LS_OK) {
    ls_plan_destroy(P);
    return rc;
  }
  *out = P;
  return LS_OK;
}

void ls_plan_destroy(ls_plan* P) {
  if (!P) return;
  prof_resolve(P, true);
  for (cudaEvent_t ev : P->prof.pool) cudaEventDestroy(ev);
  cudaFree(P->prof.runs_d);
  engine_release(P->eng);
  cudaFree(P->pupil_h);
  if (P->owns_shared) {
    cudaFree(P->tw2_x); cudaFree(P->tw_y);
    if (P->zwa_z != P->twa_z) { cudaFree(P->zwa_z); cudaFree(P->zwb_z); }
    cudaFree(P->zwa2_z); cudaFree(P->zwb2_z);
    cudaFree(P->twa_z); cudaFree(P->twb_z);
    cudaFree(P->gocta); cudaFree(P->k2hat); cudaFree(P->gxz);
  }
  delete P;
}

int ls_green_spectrum(ls_plan* P, int p, ls_c64* out_full, void* stream) {
  lsgpu::TraceRange trace_range("ls_green_spectrum");
  if (!P) { set_last_error("null plan"); return LS_EINVAL; }
  if (p < 2 || (p & 1)) { set_last_error("oversampling p must be even and >= 2"); return LS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  if (p != P->p_built) {
    GreenBuildParams g;
    g.Mx = 2 * P->nx; g.My = 2 * P->ny; g.Mz = 2 * P->nz;
    g.p = p;
    const double Lx = P->nx * P->h, Ly = P->ny * P->h, Lz = P->nz * P->h;
    g.dx = 2.0 * kPi / (p * Lx);
    g.dy = 2.0 * kPi / (p * Ly);
    g.dz = 2.0 * kPi / (p * Lz);
    g.kb = P->kb;
    g.R = sqrt(Lx * Lx + Ly * Ly + Lz * Lz);
    double2 *S = nullptr, *K = nullptr;
    const size_t total = (size_t)8 * P->N;
    if (cudaMalloc(&S, total * sizeof(double2)) != cudaSuccess || cudaMalloc(&K, total * sizeof(double2)) != cudaSuccess) {
      cudaFree(S);
      set_last_error("Green build scratch allocation failed");
      return LS_ENOMEM;
    }
    cudaError_t e = build_green_octant(g, S, K, P->gocta, st);
    if (e == cudaSuccess && P->gxz) e = unfold_octant_x(P->nx, P->ny, P->nz, P->gocta, P->gxz, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(S);
    cudaFree(K);
    if (e != cudaSuccess) { set_last_error("Green build: %s", cudaGetErrorString(e)); return LS_ECUDA; }
    P->p_built = p;
  }
  if (out_full) {
    cudaError_t e = expand_octant(P->nx, P->ny, P->nz, P->gocta, (float2*)out_full, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_last_error("expand: %s", cudaGetErrorString(e)); return LS_ECUDA; }
  }
  return LS_OK;
}

int ls_scattering_potential(const float* dn, size_t count, double eta_b, double k_b, float* f, void* stream) {
  if ((!dn || !f) && count) { set_last_error("null pointer"); return LS_EINVAL; }
  if (!(eta_b > 0) || !(k_b > 0)) { set_last_error("eta_b and k_b must be positive"); return LS_EINVAL; }
  if (count == 0) return LS_OK;
  launch_potential(dn, count, eta_b, k_b, f, (cudaStream_t)stream);
  LS_CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int ls_plane_waves(ls_plan* P, int n_views, const double* kvec, ls_c64* const* u_in, void* stream) {
  lsgpu::TraceRange trace_range("ls_plane_waves");
  if (!P || !kvec || !u_in || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  for (int q = 0; q < n_views; ++q) if (!u_in[q]) { set_last_error("u_in[%d] is null", q); return LS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = engine_reserve(P, n_views);
  if (rc) return rc;
  LS_CUDA_TRY(cudaMemcpyAsync(P->eng.kvec_d, kvec, (size_t)3 * n_views * sizeof(double), cudaMemcpyHostToDevice, st));
  rc = engine_upload_ptrs(P, 0, (const void* const*)u_in, n_views, st);
  if (rc) return rc;
  PlaneWaveParams a{P->nx, P->ny, P->nz, P->h, P->eng.kvec_d, (float2* const*)engine_ptr_table(P, 0)};
  LS_CUDA_TRY(launch_plane_waves(a, n_views, st));
  return LS_OK;
}

static int single_op(ls_plan* P, const float* f, const ls_c64* x, ls_c64* y, int adjoint, int matvec, cudaStream_t st) {
  int rc = engine_reserve(P, 1);
  if (rc) return rc;
  SlotSel sel;
  sel.slots = nullptr; sel.mask = 0; sel.f_default = f; sel.adj_default = adjoint ? 1 : 0;
  sel.runs = nullptr;
  sel.nslots = 1;
  FxParams fx = fx_base(P, sel, P->ny * P->nz);
  fx.mode = matvec ? FX_F_TIMES : FX_COPY;
  fx.src = (const float2*)x;
  IxParams ix;
  memset(&ix, 0, sizeof(ix));
  ix.mode = matvec ? IX_MATVEC : IX_STORE;
  ix.in0 = (const float2*)x;
  ix.out0 = (float2*)y;
  ix.vstride = 0;
  ix.out_o = 0; ix.out_m = P->nx;
  matvec_core(P, sel, 1, fx, ix, st);
  LS_CUDA_TRY(cudaGetLastError());
  return LS_OK;
}

int ls_apply_green(ls_plan* P, const ls_c64* v, ls_c64* out, int adjoint, void* stream) {
  lsgpu::TraceRange trace_range("ls_apply_green");
  if (!P || !v || !out) { set_last_error("bad arguments"); return LS_EINVAL; }
  return single_op(P, nullptr, v, out, adjoint, 0, (cudaStream_t)stream);
}

int ls_matvec(ls_plan* P, const float* f, const ls_c64* x, ls_c64* y, int adjoint, void* stream) {
  lsgpu::TraceRange trace_range("ls_matvec");
  if (!P || !f || !x || !y) { set_last_error("bad arguments"); return LS_EINVAL; }
  return single_op(P, f, x, y, adjoint, 1, (cudaStream_t)stream);
}

static int check_views(int n, const void* const* a, const char* what, bool allow_null_array) {
  if (!a) {
    if (allow_null_array) return LS_OK;
    set_last_error("%s is null", what);
    return LS_EINVAL;
  }
  for (int q = 0; q < n; ++q)
    if (!a[q]) { set_last_error("%s[%d] is null", what, q); return LS_EINVAL; }
  return LS_OK;
}

int ls_matvec_batch(ls_plan* P, const float* f, int n_views, const ls_c64* const* x, ls_c64* const* y, int adjoint,
                    void* stream) {
  lsgpu::TraceRange trace_range("ls_matvec_batch");
  if (!P || !f || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)x, "x", false);
  if (!rc) rc = check_views(n_views, (const void* const*)y, "y", false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = engine_reserve(P, n_views);
  if (rc) return rc;
  Engine& e = P->eng;
  for (int q = 0; q < n_views; ++q) {
    LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_X, q), x[q], e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    slot_defaults(P, e.slots_h[q], f, adjoint ? 1 : 0);
    e.slots_h[q].flags = SLOT_AUX;
  }
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_d, e.slots_h, (size_t)n_views * sizeof(SlotDev), cudaMemcpyHostToDevice, st));
  SlotSel sel = sel_slots(P, SLOT_AUX);
  FxParams fx = fx_base(P, sel, P->ny * P->nz);
  fx.mode = FX_F_TIMES;
  fx.src = e.vptr(V_X);
  IxParams ix;
  memset(&ix, 0, sizeof(ix));
  ix.mode = IX_MATVEC;
  ix.in0 = e.vptr(V_X);
  ix.out0 = e.vptr(V_R);
  ix.vstride = e.N;
  matvec_core(P, sel, n_views, fx, ix, st);
  for (int q = 0; q < n_views; ++q)
    LS_CUDA_TRY(cudaMemcpyAsync(y[q], e.vptr(V_R, q), e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  LS_CUDA_TRY(cudaGetLastError());
  prof_resolve(P, false);
  return LS_OK;
}

// Wave vectors of the plan's built-in illumination for n views: a cone of half-angle theta around
// +z (sin theta = opt.cone_sin_theta), azimuths 2 pi q / n (the set-up of Fig. 1).
static void builtin_kvec(const ls_plan* P, int n, std::vector<double>& k) {
  const double s = P->opt.cone_sin_theta, c = sqrt(std::max(0.0, 1.0 - s * s));
  k.assign(3 * (size_t)n, 0.0);
  for (int q = 0; q < n; ++q) {
    const double phi = 2.0 * kPi * q / n;
    k[3 * q] = P->kb * s * cos(phi);
    k[3 * q + 1] = P->kb * s * sin(phi);
    k[3 * q + 2] = P->kb * c;
  }
}

// Built-in plane waves for slots [0, n), written straight into b and (unless initial guesses are
// given) x0 = b: one launch over a pointer table of 2n (or n) vectors.
static int builtin_plane_waves(ls_plan* P, int n, bool also_x, cudaStream_t st) {
  Engine& e = P->eng;
  std::vector<double> k;
  builtin_kvec(P, n, k);
  const int m = also_x ? 2 * n : n;
  if (also_x) k.insert(k.end(), k.begin(), k.end());
  std::vector<void*> ptrs(m);
  for (int q = 0; q < n; ++q) {
    ptrs[q] = e.vptr(V_B, q);
    if (also_x) ptrs[n + q] = e.vptr(V_X, q);
  }
  // the kvec table holds 6 * cap doubles and the pointer tables 4 * cap pointers: tables 0 and 1 carry 2n
  LS_CUDA_TRY(cudaMemcpyAsync(e.kvec_d, k.data(), k.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = engine_upload_ptrs(P, 0, (const void* const*)ptrs.data(), m, st);
  if (rc) return rc;
  PlaneWaveParams a{P->nx, P->ny, P->nz, P->h, e.kvec_d, (float2* const*)engine_ptr_table(P, 0)};
  LS_CUDA_TRY(launch_plane_waves(a, m, st));
  return LS_OK;
}

// Copy the caller's right-hand sides into slots [0, n) (b, and x0 = b unless initial guesses are given)
// and set the slot states.  rhs == NULL: the plan's built-in plane waves.
static int load_rhs(ls_plan* P, const float* f, int n, const ls_c64* const* rhs, int adjoint, cudaStream_t st,
                    const ls_c64* const* x0 = nullptr) {
  Engine& e = P->eng;
  if (!rhs) {
    int rc = builtin_plane_waves(P, n, x0 == nullptr, st);
    if (rc) return rc;
  }
  for (int q = 0; q < n; ++q) {
    if (rhs) LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_B, q), rhs[q], e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (rhs || x0)
      LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_X, q), x0 ? x0[q] : rhs[q], e.N * sizeof(float2),
                                  cudaMemcpyDeviceToDevice, st));
  }
  for (int q = 0; q < n; ++q) slot_defaults(P, e.slots_h[q], f, adjoint);
  return LS_OK;
}

static int forward_impl(ls_plan* P, const float* f, int n_views, const ls_c64* const* u_in,
                        const ls_c64* const* x0, ls_c64* const* u_out, ls_c64* const* far, ls_stats* stats,
                        void* stream) {
  if (!P || !f || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)u_in, "u_in", true);
  if (!rc && x0) rc = check_views(n_views, (const void* const*)x0, "x0", false);
  if (!rc) rc = check_views(n_views, (const void* const*)u_out, "u_out", true);
  if (!rc) rc = check_views(n_views, (const void* const*)far, "far", true);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = engine_reserve(P, n_views);
  if (rc) return rc;
  Engine& e = P->eng;
  rc = load_rhs(P, f, n_views, u_in, 0, st, x0);
  if (rc) return rc;
  rc = engine_solve(P, n_views, st);
  if (rc) return rc;
  const int status = worst_status(e, n_views, stats);
  if (far) {
    seq_far(P, n_views, 0, st);
    rc = pupil_on_far(P, n_views, st);
    if (rc) return rc;
    for (int q = 0; q < n_views; ++q)
      LS_CUDA_TRY(cudaMemcpyAsync(far[q], e.far + (size_t)q * P->mx * P->my, (size_t)P->mx * P->my * sizeof(float2),
                                  cudaMemcpyDeviceToDevice, st));
  }
  if (u_out)
    for (int q = 0; q < n_views; ++q)
      LS_CUDA_TRY(cudaMemcpyAsync(u_out[q], e.vptr(V_X, q), e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  LS_CUDA_TRY(cudaGetLastError());
  return status;
}

int ls_forward(ls_plan* P, const float* f, int n_views, const ls_c64* const* u_in, ls_c64* const* u_out,
               ls_c64* const* far, ls_stats* stats, void* stream) {
  lsgpu::TraceRange trace_range("ls_forward");
  return forward_impl(P, f, n_views, u_in, nullptr, u_out, far, stats, stream);
}

int ls_forward_warm(ls_plan* P, const float* f, int n_views, const ls_c64* const* u_in, const ls_c64* const* x0,
                    ls_c64* const* u_out, ls_c64* const* far, ls_stats* stats, void* stream) {
  lsgpu::TraceRange trace_range("ls_forward_warm");
  if (!x0) { set_last_error("x0 is null (use ls_forward)"); return LS_EINVAL; }
  return forward_impl(P, f, n_views, u_in, x0, u_out, far, stats, stream);
}

int ls_farfield(ls_plan* P, const float* f, int n_views, const ls_c64* const* u, ls_c64* const* far, void* stream) {
  lsgpu::TraceRange trace_range("ls_farfield");
  if (!P || !f || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)u, "u", false);
  if (!rc) rc = check_views(n_views, (const void* const*)far, "far", false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = engine_reserve(P, n_views);
  if (rc) return rc;
  Engine& e = P->eng;
  for (int q = 0; q < n_views; ++q) {
    LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_X, q), u[q], e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    slot_defaults(P, e.slots_h[q], f, 0);
  }
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_d, e.slots_h, (size_t)n_views * sizeof(SlotDev), cudaMemcpyHostToDevice, st));
  seq_far(P, n_views, 0, st);
  rc = pupil_on_far(P, n_views, st);
  if (rc) return rc;
  for (int q = 0; q < n_views; ++q)
    LS_CUDA_TRY(cudaMemcpyAsync(far[q], e.far + (size_t)q * P->mx * P->my, (size_t)P->mx * P->my * sizeof(float2),
                                cudaMemcpyDeviceToDevice, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  return LS_OK;
}

int ls_farfield_adjoint(ls_plan* P, int n_views, const ls_c64* const* r, ls_c64* const* out, void* stream) {
  lsgpu::TraceRange trace_range("ls_farfield_adjoint");
  if (!P || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)r, "r", false);
  if (!rc) rc = check_views(n_views, (const void* const*)out, "out", false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = engine_reserve(P, n_views);
  if (rc) return rc;
  Engine& e = P->eng;
  std::vector<const void*> rt;
  rc = pupil_adjoint_residuals(P, n_views, r, rt, st);
  if (rc) return rc;
  rc = engine_upload_ptrs(P, 1, rt.data(), n_views, st);
  if (rc) return rc;
  for (int q = 0; q < n_views; ++q) slot_defaults(P, e.slots_h[q], nullptr, 1);
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_d, e.slots_h, (size_t)n_views * sizeof(SlotDev), cudaMemcpyHostToDevice, st));
  seq_far_adjoint(P, n_views, (const float2* const*)engine_ptr_table(P, 1), 0, st);
  for (int q = 0; q < n_views; ++q)
    LS_CUDA_TRY(cudaMemcpyAsync(out[q], e.vptr(V_B, q), e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  return LS_OK;
}

int ls_residual(int n_views, size_t count, const ls_c64* const* pred, const ls_c64* const* meas, ls_c64* const* res,
                double* loss_out, void* stream) {
  lsgpu::TraceRange trace_range("ls_residual");
  if (n_views < 1 || count == 0) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)pred, "pred", false);
  if (!rc) rc = check_views(n_views, (const void* const*)meas, "meas", false);
  if (!rc) rc = check_views(n_views, (const void* const*)res, "res", false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)std::min<size_t>(64, (count + 255) / 256);
  void** tab = nullptr;
  double* part = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&tab, (size_t)3 * n_views * sizeof(void*), st));
  LS_CUDA_TRY(cudaMallocAsync((void**)&part, (size_t)n_views * nb * 4 * sizeof(double), st));
  std::vector<void*> h(3 * n_views);
  for (int q = 0; q < n_views; ++q) {
    h[q] = (void*)pred[q];
    h[n_views + q] = (void*)meas[q];
    h[2 * n_views + q] = (void*)res[q];
  }
  LS_CUDA_TRY(cudaMemcpyAsync(tab, h.data(), h.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
  ResidualParams a{count, (const float2* const*)tab, (const float2* const*)(tab + n_views),
                   (float2* const*)(tab + 2 * n_views), part};
  launch_residual(a, nb, n_views, st);
  std::vector<double> hp((size_t)n_views * nb * 4);
  if (loss_out) {
    LS_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  LS_CUDA_TRY(cudaFreeAsync(tab, st));
  LS_CUDA_TRY(cudaFreeAsync(part, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss_out)
    for (int q = 0; q < n_views; ++q) {
      double s = 0;
      for (int b = 0; b < nb; ++b) s += hp[((size_t)q * nb + b) * 4];
      loss_out[q] = s;
    }
  return LS_OK;
}

int ls_inner_products(int n_views, size_t count, const ls_c64* const* a, const ls_c64* const* b, double* out,
                      void* stream) {
  lsgpu::TraceRange trace_range("ls_inner_products");
  if (n_views < 1 || count == 0 || !out) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)a, "a", false);
  if (!rc) rc = check_views(n_views, (const void* const*)b, "b", false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (int)std::min<size_t>(64, (count + 255) / 256);
  void** tab = nullptr;
  double* part = nullptr;
  LS_CUDA_TRY(cudaMallocAsync((void**)&tab, (size_t)2 * n_views * sizeof(void*), st));
  LS_CUDA_TRY(cudaMallocAsync((void**)&part, (size_t)n_views * nb * 4 * sizeof(double), st));
  std::vector<void*> h(2 * n_views);
  for (int q = 0; q < n_views; ++q) {
    h[q] = (void*)a[q];
    h[n_views + q] = (void*)b[q];
  }
  LS_CUDA_TRY(cudaMemcpyAsync(tab, h.data(), h.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
  ResidualParams p{count, (const float2* const*)tab, (const float2* const*)(tab + n_views), nullptr, part};
  launch_inner(p, nb, n_views, st);
  LS_CUDA_TRY(cudaGetLastError());
  std::vector<double> hp((size_t)n_views * nb * 4);
  LS_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  LS_CUDA_TRY(cudaFreeAsync(tab, st));
  LS_CUDA_TRY(cudaFreeAsync(part, st));
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  for (int q = 0; q < n_views; ++q) {
    double re = 0, im = 0;
    for (int k = 0; k < nb; ++k) {
      re += hp[((size_t)q * nb + k) * 4];
      im += hp[((size_t)q * nb + k) * 4 + 1];
    }
    out[2 * q] = re;
    out[2 * q + 1] = im;
  }
  return LS_OK;
}

int ls_gradient(ls_plan* P, const float* f, int n_views, const ls_c64* const* u_in, const ls_c64* const* u_fwd,
                const ls_c64* const* residuals, const double* view_weights, float* grad, ls_stats* stats,
                void* stream) {
  lsgpu::TraceRange trace_range("ls_gradient");
  if (!P || !f || !grad || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  int rc = check_views(n_views, (const void* const*)residuals, "residuals", false);
  if (!rc && !u_fwd) rc = check_views(n_views, (const void* const*)u_in, "u_in", true);
  if (!rc && u_fwd) rc = check_views(n_views, (const void* const*)u_fwd, "u_fwd", false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = engine_reserve(P, n_views);
  if (rc) return rc;
  Engine& e = P->eng;
  std::vector<const void*> uptr(n_views);
  int fwd_status = LS_OK;
  if (!u_fwd) {
    // recompute the forward fields and keep them
    rc = engine_reserve_ucache(P, n_views);
    if (rc) return rc;
    rc = load_rhs(P, f, n_views, u_in, 0, st);
    if (rc) return rc;
    rc = engine_solve(P, n_views, st);
    if (rc) return rc;
    fwd_status = worst_status(e, n_views, nullptr);
    for (int q = 0; q < n_views; ++q) {
      LS_CUDA_TRY(cudaMemcpyAsync(e.ucache + (size_t)q * e.N, e.vptr(V_X, q), e.N * sizeof(float2),
                                  cudaMemcpyDeviceToDevice, st));
      uptr[q] = e.ucache + (size_t)q * e.N;
    }
  } else {
    for (int q = 0; q < n_views; ++q) uptr[q] = u_fwd[q];
  }
  // adjoint right-hand sides b_q = G~^H P^H r_q
  std::vector<const void*> rt;
  rc = pupil_adjoint_residuals(P, n_views, residuals, rt, st);
  if (rc) return rc;
  rc = engine_upload_ptrs(P, 1, rt.data(), n_views, st);
  if (rc) return rc;
  for (int q = 0; q < n_views; ++q) slot_defaults(P, e.slots_h[q], f, 1);
  LS_CUDA_TRY(cudaMemcpyAsync(e.slots_d, e.slots_h, (size_t)n_views * sizeof(SlotDev), cudaMemcpyHostToDevice, st));
  seq_far_adjoint(P, n_views, (const float2* const*)engine_ptr_table(P, 1), 0, st);
  for (int q = 0; q < n_views; ++q)
    LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_X, q), e.vptr(V_B, q), e.N * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  rc = engine_solve(P, n_views, st);
  if (rc) return rc;
  const int adj_status = worst_status(e, n_views, stats);
  // grad = sum_q c_q Re(conj(u_q) w_q)
  rc = engine_upload_ptrs(P, 2, (const void* const*)uptr.data(), n_views, st);
  if (rc) return rc;
  std::vector<float> w(n_views);
  for (int q = 0; q < n_views; ++q) w[q] = view_weights ? (float)view_weights[q] : 1.0f;
  LS_CUDA_TRY(cudaMemcpyAsync(e.weights_d, w.data(), n_views * sizeof(float), cudaMemcpyHostToDevice, st));
  GradParams g{e.N, n_views, (const float2* const*)engine_ptr_table(P, 2), e.vptr(V_X), e.N, e.weights_d, grad};
  launch_gradient(g, st);
  LS_CUDA_TRY(cudaGetLastError());
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (fwd_status != LS_OK) return fwd_status;
  return adj_status;
}

int ls_debug_bounds(unsigned* site, int clear) {
  if (site) *site = 0;
#ifdef LS_DEBUG_BOUNDS
  unsigned (*const readers[])(bool) = {bounds_site_16,  bounds_site_24,  bounds_site_32,  bounds_site_48,
                                       bounds_site_64,  bounds_site_96,  bounds_site_128, bounds_site_144,
                                       bounds_site_192, bounds_site_256, bounds_site_288, bounds_site_384,
                                       bounds_site_krylov};
  unsigned first = 0;
  for (auto rd : readers) {
    const unsigned v = rd(clear != 0);
    if (v == 0xffffffffu) {
      set_last_error("ls_debug_bounds: an index-check record could not be read");
      return LS_ECUDA;
    }
    if (first == 0) first = v;
  }
  if (site) *site = first;
  return 1;
#else
  (void)clear;
  return 0;
#endif
}

int ls_debug_inject(ls_plan* P, int kind, long long value) {
  switch (kind) {
    case LS_INJECT_NONE:
      if (!P) { set_last_error("null plan"); return LS_EINVAL; }
      P->inj_zero_shadow_view = -1;
      P->inj_max_rounds = -1;
      P->inj_z_stall = 0;
      P->inj_z_wait_ns = 0;
      P->inj_bounds_probe = 0;
      g_fail_allocs.store(0);
      return LS_OK;
    case LS_INJECT_ZERO_SHADOW:
      if (!P) { set_last_error("null plan"); return LS_EINVAL; }
      P->inj_zero_shadow_view = value >= 0 && value < kMaxLaunchSlots ? (int)value : -1;
      return LS_OK;
    case LS_INJECT_MAX_ROUNDS:
      if (!P) { set_last_error("null plan"); return LS_EINVAL; }
      P->inj_max_rounds = value >= 0 ? value : -1;
      return LS_OK;
    case LS_INJECT_ALLOC_FAIL:
      g_fail_allocs.store(value > 0 ? value : 0);
      return LS_OK;
    case LS_INJECT_Z_STALL:
      if (!P) { set_last_error("null plan"); return LS_EINVAL; }
      if (value < 0) { set_last_error("wait limit must be >= 0"); return LS_EINVAL; }
      P->inj_z_stall = value > 0 ? 1 : 0;
      P->inj_z_wait_ns = value;
      return LS_OK;
    case LS_INJECT_BOUNDS_PROBE:
      if (!P) { set_last_error("null plan"); return LS_EINVAL; }
      P->inj_bounds_probe = value != 0 ? 1 : 0;
      return LS_OK;
    default:
      set_last_error("unknown injection kind %d", kind);
      return LS_EINVAL;
  }
}

}  // extern "C"

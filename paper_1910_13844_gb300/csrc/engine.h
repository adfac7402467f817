// Host-side plan and batched solver engine shared by the C ABI and the server.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "green.cuh"
#include "krylov.cuh"
#include "passes.cuh"
#include "trace.h"

namespace lsgpu {

enum Vec : int { V_B = 0, V_X = 1, V_R = 2, V_RH = 3, V_P = 4, V_V = 5, V_S = 6, V_T = 7, NVEC = 8 };

struct Engine {
  CUtensorMap a2_map;           // TMA map of a2 for the z pass (valid if a2_map_ok)
  int a2_map_ok = 0;
  int slot0 = 0;                // slot coordinate of this engine's slot 0 in a2_map (server lanes view a range)
  int cap = 0;                  // slots allocated
  size_t N = 0;
  float2* vec = nullptr;        // [NVEC][cap][N]
  float2* a1 = nullptr;         // [cap][nz][ny][2nx]
  float2* a2 = nullptr;         // [cap][nz][2ny][2nx]
  size_t a1_stride = 0, a2_stride = 0;
  float2* far = nullptr;        // [cap][my*mx]
  float2* ucache = nullptr;     // [cap][N] forward fields kept for a gradient (lazy)
  int ucache_cap = 0;
  double* partials = nullptr;   // [cap][maxparts][4]
  int maxparts = 0;
  SlotDev* slots_d = nullptr;
  SlotDev* slots_h = nullptr;   // pinned mirror
  int* counts_d = nullptr;      // [0..3] slot counts (k_count), [4] device error flag (a wait gave up)
  int* counts_h = nullptr;      // pinned
  void** ptrs_d = nullptr;      // pointer tables: [4][cap]
  double* kvec_d = nullptr;     // [cap*6]: wave vectors, 3 per view (twice for the built-in plane waves)
  float* weights_d = nullptr;   // [cap]
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t iter_graph = nullptr;
  int iter_graph_slots = 0;
  int iter_graph_variant = 0;   // launch variants the graph was captured with
  float2* vptr(int v, int slot = 0) const { return vec + ((size_t)v * cap + slot) * N; }
};

struct Profiler {
  bool on = false;
  struct Pending { int kind; int slots; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  unsigned long long* runs_d = nullptr;   // [LS_K_COUNT] slots that ran, counted by the kernels
  double ms[LS_K_COUNT] = {};
  long long launches[LS_K_COUNT] = {};
  long long slot_passes[LS_K_COUNT] = {};
};

}  // namespace lsgpu

struct ls_plan {
  int nx = 0, ny = 0, nz = 0;
  size_t N = 0;
  double kb = 0, h = 0;
  ls_options opt{};
  int mx = 0, my = 0, ox = 0, oy = 0;
  double x_gamma = 0;
  lsgpu::PassLaunch px{}, py{}, pz{};
  float2 *tw2_x = nullptr, *tw_y = nullptr;   // x-pass stage twiddles [k1*R2 + n2]; y-pass exp(-2 pi i j / L)
  float2 *twa_z = nullptr, *twb_z = nullptr;
  float2 *zwa_z = nullptr, *zwb_z = nullptr;   // z tables for the TMA-staged split (alias twa_z/twb_z if equal)
  float2 *zwa2_z = nullptr, *zwb2_z = nullptr; // z tables for its second split (null if the length has none)
  float2* gocta = nullptr;
  float2* gxz = nullptr;        // the octant unfolded along x (dynamically scheduled z pass), if that pass exists
  CUtensorMap gxz_map;          // TMA map of gxz (valid if gxz_ok)
  int gxz_ok = 0;
  float2* k2hat = nullptr;
  int p_built = 0;
  bool owns_shared = true;   // false for clones that borrow another plan's spectra and twiddles
  double2* pupil_h = nullptr; // pupil / refocus transfer function on the 2my x 2mx detector grid (ls_set_pupil)
  // launch variants chosen by ls_autotune (defaults: the best measured at 128^3 x 60 views)
  int tune_z_tma = 1;           // TMA-staged z pass where available (else the cp.async-staged one)
  int tune_ix_prefetch = 1;     // IX asks L2 for its epilogue operands at kernel start
  int tune_fx_views_fastest = 0;  // FX grid with views fastest (else row blocks fastest)
  int tune_z_split = 0;           // TMA-staged z pass with its second radix split
  int tune_z_persist = -1;        // persistent TMA-staged z pass (0: one CTA per tile, 1: tiles round-robin,
                                  // 2: work units from a counter; -1, untuned: the length's ZAuto form)
  int tune_views = 0;             // batch size ls_autotune tuned for: its z form applies to launches of
                                  // more than tune_views / 2 views, smaller launches take the ZAuto form
  int tune_fx_bulk = 0;           // bulk-copy-staged persistent first pass
  int tune_strided_wide = 0;      // FY/IY with 32 pencils per CTA (else 16)
  int tune_views_per_launch = 0;  // BiCGStab iteration launched over chunks of this many views (0: all)
  // test-only failure injection (ls_debug_inject); the defaults inject nothing
  int inj_zero_shadow_view = -1;  // this view's shadow residual is zeroed at the start of a solve
  long long inj_max_rounds = -1;  // host rounds a solve may take (-1: the normal bound)
  int inj_z_stall = 0;            // the TMA-staged z pass waits on a barrier nothing completes
  long long inj_z_wait_ns = 0;    // per-view wait limit of the TMA-staged z pass (0: one second)
  int inj_bounds_probe = 0;       // debug build: the first pass treats its last view as out of range
  // ls_matvec_noalloc: device address of the library's static scratch array on this plan's device,
  // looked up when the plan is created (null, with noalloc_rc set, if that failed)
  int device = 0;
  int sms = 0;                   // SMs of the plan's device (grid size of the persistent z passes)
  void* noalloc_scratch = nullptr;
  int noalloc_rc = 0;
  lsgpu::Engine eng;
  lsgpu::Profiler prof;
  ls_plan* prof_parent = nullptr;   // slot views time their launches in the viewed plan's profiler
};

namespace lsgpu {

int engine_reserve(ls_plan* P, int nslots);
int engine_reserve_ucache(ls_plan* P, int nslots);
void engine_release(Engine& e);

// Upload host slot states [0, nslots) and run BiCGStab until every slot has
// left SLOT_ITER/SLOT_RESID.  Vectors b and x must be set.
int engine_solve(ls_plan* P, int nslots, cudaStream_t st);
// Sequences of kernel launches (no synchronisation).
void seq_resid(ls_plan* P, int nslots, cudaStream_t st);
void seq_iter(ls_plan* P, int nslots, cudaStream_t st);
// seq_iter over chunks of P->tune_views_per_launch slots (one launch per pass and chunk)
void seq_iter_chunked(ls_plan* P, int nslots, cudaStream_t st);
void seq_far(ls_plan* P, int nslots, unsigned mask, cudaStream_t st);
void seq_far_adjoint(ls_plan* P, int nslots, const float2* const* r_dev_table, unsigned mask, cudaStream_t st);
int engine_upload_ptrs(ls_plan* P, int table, const void* const* host_ptrs, int n, cudaStream_t st);
void** engine_ptr_table(ls_plan* P, int table);
void slot_defaults(const ls_plan* P, SlotDev& s, const float* f, int adjoint);
int ensure_iter_graph(ls_plan* P, int nslots);
// Shallow view of slots [s0, s0 + n) of P's engine as slots [0, n) (no ownership).
ls_plan plan_slot_view(const ls_plan* P, int s0);
// New plan object with its own (empty) workspace that shares P's Green spectrum, far-field
// kernels and twiddles; P must outlive it.
ls_plan* plan_clone_shared(const ls_plan* P);
// one batched operator application y = x - G(f x) over slots [0, n) (x in V_X, y in V_R), for the autotuner
int tune_matvec(ls_plan* P, const float* f, int n, cudaStream_t st);
// a forward solve of slots [0, n) from the right-hand sides already in V_B (x0 = b), for the autotuner
int tune_forward(ls_plan* P, const float* f, int n, cudaStream_t st);
// P y (adjoint: P^H y) for one detector field; scratch holds 4 my mx double2
int apply_pupil_device(ls_plan* P, const float2* in, float2* out, int adjoint, double2* scratch, cudaStream_t st);

// ls_matvec_noalloc set-up (noalloc.cu): the device address of the static scratch array on the
// current device; loads the array's module (reserving the array) if that has not happened yet.
int noalloc_setup(void** addr);

// Launch wrapper: an NVTX range named after the kind; when profiling is on, the launch is also
// bracketed with an event pair.
cudaEvent_t prof_event(ls_plan* P);
void prof_resolve(ls_plan* P, bool wait);
inline ls_plan* prof_owner(ls_plan* P) { return P->prof_parent ? P->prof_parent : P; }
template <class F>
inline void timed(ls_plan* P0, int kind, int nslots, cudaStream_t st, F&& launch) {
  TraceRange range(trace_kind_name(kind));
  ls_plan* P = prof_owner(P0);
  if (!P->prof.on) {
    launch();
    return;
  }
  cudaEvent_t a = prof_event(P), b = prof_event(P);
  cudaEventRecord(a, st);
  launch();
  cudaEventRecord(b, st);
  P->prof.pending.push_back({kind, nslots, a, b});
}

}  // namespace lsgpu

// Launch-variant autotuner.  For one plan and batch size it times the variants that the passes and
// the solve loop can switch between at run time, on the plan's own grid and views:
//   * the z pass: TMA-staged with warp-local exchanges, or cp.async-staged with CTA-wide exchanges;
//   * the TMA-staged z pass's radix split: the default one or a second one (R1 x R2 transposed, or
//     2 R1 x R2 / 2 where R1 = R2), where the length has one;
//   * the TMA-staged z pass one CTA per tile, or persistent (one wave of CTAs, each streaming the
//     views of several tiles);
//   * FY / IY: 16 or 32 pencils per CTA;
//   * IX: L2 prefetch of its epilogue operands at kernel start, or not;
//   * FX: launch grid with the views fastest (shared potential rows from L2), or the rows fastest;
//   * the solve loop: FX in the BiCGStab iteration as the bulk-copy-staged persistent kernel (input rows
//     staged in shared memory, three row blocks ahead) or not, the views per launch of an iteration
//     (all, or chunks of n/2, n/4 or 8 views, each chunk one launch per pass), iterations between
//     host reads of the convergence mask (2, 4, 8), and replay of the iteration from a captured CUDA
//     graph or direct launches.
// Operator variants are timed on batched operator applications, the loop variants on forward solves
// of plane-wave illuminations.  Every operator variant's output is first compared with the default
// variants' (relative L2 over the batch); a variant that differs by more than 1e-5 is never chosen.
// One knob is tuned at a time, in the order above, keeping the best value of the earlier ones.  Results can be cached in a text file (LS_AUTOTUNE_CACHE) keyed by the
// device name, the grid and the number of views.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>

#include "engine.h"

namespace lsgpu {

static std::mutex g_cache_mu;

// forward solves timed per loop variant (after one untimed solve): single solves differ by about 1%,
// as much as the loop variants themselves
constexpr int kSolveReps = 3;

static std::string tune_key(const ls_plan* P, int n_views) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s:%dx%dx%d:%d", name.c_str(), P->nx, P->ny, P->nz, n_views);
  return buf;
}

static bool cache_lookup(const std::string& key, ls_tune* t) {
  const char* path = getenv("LS_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  FILE* fp = fopen(path, "r");
  if (!fp) return false;
  char k[256];
  ls_tune v;
  bool found = false;
  char line[512];
  while (fgets(line, sizeof(line), fp)) {
    if (sscanf(line, "%255s %d %d %d %d %d %lf %lf %d %d %d %d %d", k, &v.z_tma, &v.ix_prefetch,
               &v.fx_views_fastest, &v.check_every, &v.use_graphs, &v.matvec_us_per_view, &v.solve_ms, &v.z_split,
               &v.strided_wide, &v.views_per_launch, &v.z_persist, &v.fx_bulk) == 13 &&
        key == k) {
      *t = v;   // the last entry for a key wins
      found = true;
    }
  }
  fclose(fp);
  return found;
}

static void cache_store(const std::string& key, const ls_tune& t) {
  const char* path = getenv("LS_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lock(g_cache_mu);
  FILE* fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d %d %d %d %.9g %.9g %d %d %d %d %d\n", key.c_str(), t.z_tma, t.ix_prefetch,
          t.fx_views_fastest, t.check_every, t.use_graphs, t.matvec_us_per_view, t.solve_ms, t.z_split, t.strided_wide,
          t.views_per_launch, t.z_persist, t.fx_bulk);
  fclose(fp);
}

static void apply(ls_plan* P, const ls_tune& t) {
  P->tune_z_tma = t.z_tma;
  P->tune_ix_prefetch = t.ix_prefetch;
  P->tune_fx_views_fastest = t.fx_views_fastest;
  P->opt.check_every = t.check_every;
  P->opt.use_graphs = t.use_graphs;
  P->tune_z_split = t.z_split && P->zwa2_z ? 1 : 0;
  P->tune_strided_wide = t.strided_wide;
  P->tune_views_per_launch = t.views_per_launch;
  P->tune_z_persist = t.z_persist;
  P->tune_fx_bulk = t.fx_bulk;
}

// mean milliseconds of `reps` calls of fn after one untimed call; negative on error
template <typename F>
static double time_ms(cudaStream_t st, int reps, F fn) {
  if (fn() != LS_OK) return -1.0;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.0;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1.0; }
  cudaEventRecord(a, st);
  int rc = LS_OK;
  for (int r = 0; r < reps && rc == LS_OK; ++r) rc = fn();
  cudaEventRecord(b, st);
  float ms = -1.f;
  if (rc == LS_OK && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc == LS_OK && ms >= 0.f ? ms / reps : -1.0;
}

}  // namespace lsgpu

using namespace lsgpu;

extern "C" int ls_autotune(ls_plan* P, int n_views, const float* f, ls_tune* out, void* stream) {
  lsgpu::TraceRange trace_range("ls_autotune");
  if (!P || !f || n_views < 1) { set_last_error("bad arguments"); return LS_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = tune_key(P, n_views);
  // the z-pass form chosen here is used for launches of more than n_views / 2 views (smaller ones take
  // the length's default form)
  P->tune_views = n_views;
  // the workspace (and with it the z pass's TMA map) must exist before a variant is chosen
  int rc = engine_reserve(P, n_views);
  if (rc) return rc;
  ls_tune best;
  if (cache_lookup(key, &best)) {
    if (!P->eng.a2_map_ok) best.z_tma = 0;
    if (!P->zwa2_z) best.z_split = 0;
    if (best.views_per_launch >= n_views) best.views_per_launch = 0;
    apply(P, best);
    best.from_cache = 1;
    if (out) *out = best;
    return LS_OK;
  }
  Engine& e = P->eng;
  // plane-wave right-hand sides on a cone of half-angle asin(0.6) around z (numerical aperture 0.8 in
  // water), one direction per view
  std::vector<double> k(3 * (size_t)n_views);
  for (int q = 0; q < n_views; ++q) {
    const double phi = 2.0 * 3.14159265358979323846 * q / n_views, s = 0.6;
    k[3 * q] = P->kb * s * cos(phi);
    k[3 * q + 1] = P->kb * s * sin(phi);
    k[3 * q + 2] = P->kb * sqrt(1.0 - s * s);
  }
  std::vector<void*> ptrs(n_views);
  for (int q = 0; q < n_views; ++q) ptrs[q] = e.vptr(V_B, q);
  LS_CUDA_TRY(cudaMemcpyAsync(e.kvec_d, k.data(), k.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  rc = engine_upload_ptrs(P, 0, (const void* const*)ptrs.data(), n_views, st);
  if (rc) return rc;
  PlaneWaveParams pw{P->nx, P->ny, P->nz, P->h, e.kvec_d, (float2* const*)engine_ptr_table(P, 0)};
  LS_CUDA_TRY(launch_plane_waves(pw, n_views, st));
  LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_X), e.vptr(V_B), (size_t)n_views * e.N * sizeof(float2),
                              cudaMemcpyDeviceToDevice, st));
  // the per-launch profiler stays off while timing (it would also disable graph replay)
  const bool prof = P->prof.on;
  P->prof.on = false;
  ls_tune cur;
  cur.z_tma = e.a2_map_ok ? 1 : 0;
  cur.ix_prefetch = 1;
  cur.fx_views_fastest = 1;
  cur.check_every = P->opt.check_every > 0 ? P->opt.check_every : 2;
  cur.use_graphs = 1;
  cur.z_split = 0;
  cur.strided_wide = 0;
  cur.views_per_launch = 0;
  cur.z_persist = 0;
  cur.fx_bulk = 0;
  cur.from_cache = 0;
  auto matvec = [&] { return tune_matvec(P, f, n_views, st); };
  // reference output of the default variants (y = x - G f x over the batch, kept in the s vectors)
  apply(P, cur);
  if (matvec() != LS_OK) {
    P->prof.on = prof;
    return LS_ECUDA;
  }
  LS_CUDA_TRY(cudaMemcpyAsync(e.vptr(V_S), e.vptr(V_R), (size_t)n_views * e.N * sizeof(float2),
                              cudaMemcpyDeviceToDevice, st));
  // relative L2 difference of the vectors `got` from the reference vectors at ref (n_views * N
  // complex values) over the batch (negative on error)
  auto differ = [&](int got, const float2* ref) -> double {
    std::vector<void*> tab(3 * (size_t)n_views);
    for (int q = 0; q < n_views; ++q) {
      tab[q] = e.vptr(got, q);
      tab[n_views + q] = (void*)(ref + (size_t)q * e.N);
      tab[2 * n_views + q] = e.vptr(V_T, q);
    }
    if (engine_upload_ptrs(P, 1, (const void* const*)tab.data(), 3 * n_views, st) != LS_OK) return -1.0;
    void** t1 = engine_ptr_table(P, 1);
    const int nb = 64;
    ResidualParams rp{e.N, (const float2* const*)t1, (const float2* const*)(t1 + n_views),
                      (float2* const*)(t1 + 2 * n_views), e.partials};
    launch_residual(rp, nb, n_views, st);
    std::vector<double> h((size_t)n_views * nb * 4);
    if (cudaMemcpyAsync(h.data(), e.partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return -1.0;
    double dd = 0.0, rr = 0.0;
    for (size_t b = 0; b < (size_t)n_views * nb; ++b) {
      dd += h[4 * b];
      rr += h[4 * b + 1];
    }
    return rr > 0.0 ? sqrt(dd / rr) : sqrt(dd);
  };
  // the current variant's operator output against the default variants'
  auto deviation = [&]() -> double { return matvec() == LS_OK ? differ(V_R, e.vptr(V_S)) : -1.0; };
  auto tune_op = [&](int* knob, int n_values, const int* values) -> double {
    double best_ms = -1.0;
    int best_v = *knob;
    for (int i = 0; i < n_values; ++i) {
      *knob = values[i];
      apply(P, cur);
      const double dev = deviation();
      if (!(dev >= 0.0 && dev <= 1e-5)) continue;   // not the same operator: never chosen
      const double ms = time_ms(st, 3, matvec);
      if (ms > 0 && (best_ms < 0 || ms < best_ms)) { best_ms = ms; best_v = values[i]; }
    }
    *knob = best_v;
    apply(P, cur);
    return best_ms;
  };
  static const int two[2] = {1, 0};
  double mv_ms = -1.0;
  // the TMA-staged z pass's forms first (persistence, then the split), then TMA against the
  // cp.async-staged pass with the best of them: at one view the per-tile TMA form and the cp.async
  // pass are close, and only the persistent forms are fast
  static const int persist3[3] = {1, 2, 0};
  if (e.a2_map_ok) mv_ms = tune_op(&cur.z_persist, P->gxz_ok ? 3 : 2, P->gxz_ok ? persist3 : two);
  if (e.a2_map_ok && P->zwa2_z) mv_ms = tune_op(&cur.z_split, 2, two);
  if (e.a2_map_ok) mv_ms = tune_op(&cur.z_tma, 2, two);
  mv_ms = tune_op(&cur.strided_wide, 2, two);
  mv_ms = tune_op(&cur.ix_prefetch, 2, two);
  mv_ms = tune_op(&cur.fx_views_fastest, 2, two);
  // solve loop: forward solves of the plane waves
  auto solve = [&] { return tune_forward(P, f, n_views, st); };
  auto solve_views = solve;
  double sv_ms = -1.0;
  {
    // the bulk-staged first pass in the iteration: its solution must equal the plain kernel's
    // (the same arithmetic in the same order) before its time counts; the reference solution is kept
    // in the forward-field cache (every Krylov vector is overwritten by the next solve)
    {
      int rcu = engine_reserve_ucache(P, n_views);
      cur.fx_bulk = 0;
      apply(P, cur);
      double best_b_ms = time_ms(st, kSolveReps, solve_views);
      if (rcu == LS_OK)
        LS_CUDA_TRY(cudaMemcpyAsync(e.ucache, e.vptr(V_X), (size_t)n_views * e.N * sizeof(float2),
                                    cudaMemcpyDeviceToDevice, st));
      cur.fx_bulk = 1;
      apply(P, cur);
      const double ms = rcu == LS_OK ? time_ms(st, kSolveReps, solve_views) : -1.0;
      const double dev = ms > 0 ? differ(V_X, e.ucache) : -1.0;
      cur.fx_bulk = (dev >= 0.0 && dev <= 1e-6 && ms > 0 && (best_b_ms < 0 || ms < best_b_ms)) ? 1 : 0;
    }
    // views per launch of an iteration: all of them, or chunks of n/2, n/4 or 8 views
    int cands[4] = {0, n_views / 2, n_views / 4, 8};
    int best_c = 0;
    double best_c_ms = -1.0;
    for (int ci = 0; ci < 4; ++ci) {
      const int cv = cands[ci];
      if (ci > 0 && (cv < 1 || cv >= n_views)) continue;
      bool seen = false;
      for (int cj = 1; cj < ci; ++cj) seen = seen || cands[cj] == cv;
      if (seen) continue;
      cur.views_per_launch = cv;
      apply(P, cur);
      const double ms = time_ms(st, kSolveReps, solve_views);
      if (ms > 0 && (best_c_ms < 0 || ms < best_c_ms)) { best_c_ms = ms; best_c = cv; }
    }
    cur.views_per_launch = best_c;
    static const int chunks[3] = {4, 2, 8};
    int best_v = cur.check_every;
    for (int c : chunks) {
      cur.check_every = c;
      apply(P, cur);
      const double ms = time_ms(st, kSolveReps, solve);
      if (ms > 0 && (sv_ms < 0 || ms < sv_ms)) { sv_ms = ms; best_v = c; }
    }
    cur.check_every = best_v;
    int best_g = 1;
    double best_g_ms = -1.0;
    for (int g : two) {
      cur.use_graphs = g;
      apply(P, cur);
      const double ms = time_ms(st, kSolveReps, solve);
      if (ms > 0 && (best_g_ms < 0 || ms < best_g_ms)) { best_g_ms = ms; best_g = g; }
    }
    cur.use_graphs = best_g;
    if (best_g_ms > 0) sv_ms = best_g_ms;
  }
  apply(P, cur);
  P->prof.on = prof;
  LS_CUDA_TRY(cudaGetLastError());
  if (mv_ms < 0 || sv_ms < 0) { set_last_error("autotune timing failed"); return LS_ECUDA; }
  cur.matvec_us_per_view = 1e3 * mv_ms / n_views;
  cur.solve_ms = sv_ms;
  cache_store(key, cur);
  if (out) *out = cur;
  return LS_OK;
}

// Serving: continuous batching of forward and gradient requests (include/ls.h).
//
// One lane per grid size: a plan, a fixed number of solver slots (one slot
// per view) and a stream.  A request occupies a contiguous range of slots of
// its grid's lane for its whole life, so its Krylov state stays on the device.
// A worker thread loops: admit queued requests into free slot ranges (lanes are
// created while the HBM budget allows), launch one chunk of BiCGStab
// iterations over every lane (converged or idle slots are masked inside the
// batched launches), read the slot states back, and advance each request:
//   FORWARD : solve -> far field -> copy outputs -> done
//   GRADIENT: solve -> far field -> residual and loss -> G~^H r -> adjoint
//             solve (same slots, conj(Ghat)) -> gradient -> done
// Requests that arrive while others run join at the next chunk boundary and
// share the batched launches; lanes of different grids run on their own
// streams and overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <math.h>
#include <string.h>

#include "engine.h"

using namespace lsgpu;

namespace {

enum Phase { PH_QUEUED = 0, PH_FWD, PH_ADJ, PH_FINISHING, PH_DONE };

struct Lane;

struct Request {
  uint64_t ticket = 0;
  ls_request req{};
  std::vector<double> kvec;
  int phase = PH_QUEUED;
  Lane* lane = nullptr;
  int s0 = -1, n = 0;
  int status = LS_OK;
  int iters_max = 0;
  std::chrono::steady_clock::time_point t_submit, t_done;
  int nb = 0;                 // residual partial blocks per view
  std::vector<float> weights; // host copies kept until the request finishes
  std::vector<void*> ptrs;
};

struct Lane {
  ls_grid grid{};
  ls_plan* plan = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  int cap = 0;
  size_t bytes = 0;
  std::vector<Request*> owner;   // per slot
  double* part_h = nullptr;      // pinned [cap][kResidBlocks][4] residual partials
  std::vector<Request*> to_start;   // admitted, slots assigned, initialised at the next issue
  bool issued = false;
  bool shared_plan = false;         // plan borrows the spectra of the grid's first lane
  int n_iter = 0, n_resid = 0;    // host view after the last readback
};

constexpr int kResidBlocks = 32;   // residual partial blocks per view
constexpr int kChunkDefault = 2;   // BiCGStab iterations per round unless the options say otherwise

size_t plan_bytes(const ls_grid& g, int cap) {
  const size_t N = (size_t)g.nx * g.ny * g.nz;
  return ls_workspace_bytes(&g, cap) + (size_t)cap * N * sizeof(float2) /* forward fields kept for gradients */ +
         (size_t)4 * N * sizeof(float2) /* far-field kernels */;
}

}  // namespace

struct ls_server {
  ls_server_options opt{};
  int device = 0;
  size_t budget = 0, used = 0;
  int default_cap = 64;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> all;
  std::vector<Lane*> lanes;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;

  // -------------------------------------------------------------- lanes
  // a lane of grid g with a free range of n slots (s0 receives its first slot)
  Lane* lane_for(const ls_grid& g, int n, int* s0) {
    for (Lane* l : lanes)
      if (l->grid.nx == g.nx && l->grid.ny == g.ny && l->grid.nz == g.nz) {
        const int f = free_range(l, n);
        if (f >= 0) {
          *s0 = f;
          return l;
        }
      }
    return nullptr;
  }

  // slots of a new lane for grid g: room for several large requests, fewer for very large grids
  int lane_cap(const ls_grid& g, int n) const {
    if (opt.max_views_per_grid > 0) return std::max(n, opt.max_views_per_grid);
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    const int want = N <= ((size_t)1 << 21) ? 256 : 128;
    return std::max(n, want);
  }

  // frees one lane without requests (the largest), returns false if none
  bool has_clones(const Lane* b) const {
    for (Lane* x : lanes)
      if (x != b && x->shared_plan && x->grid.nx == b->grid.nx && x->grid.ny == b->grid.ny && x->grid.nz == b->grid.nz)
        return true;
    return false;
  }

  bool reclaim_idle() {
    Lane* best = nullptr;
    for (Lane* l : lanes)
      if (lane_idle(l) && !l->issued && !(!l->shared_plan && has_clones(l)) && (!best || l->bytes > best->bytes))
        best = l;
    if (!best) return false;
    used -= best->bytes;
    lanes.erase(std::find(lanes.begin(), lanes.end(), best));
    destroy_lane(best);
    return true;
  }

  int create_lane(const ls_grid& g, int cap, Lane** out) {
    ls_options o;
    ls_default_options(&o);
    o.tol = opt.tol > 0 ? opt.tol : 1e-6;
    o.max_iter = opt.max_iter > 0 ? opt.max_iter : 1000;
    Lane* l = new Lane();
    l->grid = g;
    l->cap = cap;
    l->bytes = plan_bytes(g, cap);
    int rc = LS_OK;
    Lane* base = nullptr;
    for (Lane* x : lanes)
      if (!x->shared_plan && x->grid.nx == g.nx && x->grid.ny == g.ny && x->grid.nz == g.nz) base = x;
    if (base) {
      l->plan = plan_clone_shared(base->plan);
      l->shared_plan = true;
    } else {
      rc = ls_plan_create(&g, 2, opt.k_b, opt.voxel, &o, &l->plan);
    }
    if (rc == LS_OK) rc = engine_reserve(l->plan, cap);
    if (rc == LS_OK) rc = engine_reserve_ucache(l->plan, cap);
    if (rc == LS_OK && cudaStreamCreateWithFlags(&l->stream, cudaStreamNonBlocking) != cudaSuccess) rc = LS_ECUDA;
    if (rc == LS_OK && cudaEventCreateWithFlags(&l->ev, cudaEventDisableTiming) != cudaSuccess) rc = LS_ECUDA;
    if (rc == LS_OK) {
      Engine& e = l->plan->eng;
      for (int s = 0; s < cap; ++s) {
        memset(&e.slots_h[s], 0, sizeof(SlotDev));
      }
      if (cudaMemcpy(e.slots_d, e.slots_h, (size_t)cap * sizeof(SlotDev), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = LS_ECUDA;
    }
    if (rc != LS_OK) {
      destroy_lane(l);
      return rc;
    }
    l->owner.assign(cap, nullptr);
    if (cudaMallocHost(&l->part_h, (size_t)cap * kResidBlocks * 4 * sizeof(double)) != cudaSuccess) {
      destroy_lane(l);
      return LS_ENOMEM;
    }
    lanes.push_back(l);
    used += l->bytes;
    *out = l;
    return LS_OK;
  }

  static void destroy_lane(Lane* l) {
    if (l->stream) cudaStreamSynchronize(l->stream);
    if (l->plan) ls_plan_destroy(l->plan);
    if (l->ev) cudaEventDestroy(l->ev);
    if (l->stream) cudaStreamDestroy(l->stream);
    if (l->part_h) cudaFreeHost(l->part_h);
    delete l;
  }

  int free_range(Lane* l, int n) {
    int run = 0;
    for (int s = 0; s < l->cap; ++s) {
      run = l->owner[s] ? 0 : run + 1;
      if (run == n) return s - n + 1;
    }
    return -1;
  }

  bool lane_idle(Lane* l) {
    for (Request* r : l->owner)
      if (r) return false;
    return true;
  }

  // -------------------------------------------------------------- admission (worker thread)
  void admit() {
    {
      std::lock_guard<std::mutex> lk(mu);
      for (auto it = queue.begin(); it != queue.end();) {
        Request* r = *it;
        int s0 = -1;
        Lane* l = lane_for(r->req.grid, r->n, &s0);
        if (!l) {
          const int cap = lane_cap(r->req.grid, r->n);
          int c = cap;
          while (c > r->n && used + plan_bytes(r->req.grid, c) > budget) c = std::max(r->n, c / 2);
          while (used + plan_bytes(r->req.grid, c) > budget && reclaim_idle()) {
          }
          if (used + plan_bytes(r->req.grid, c) > budget) { ++it; continue; }   // wait for memory
          if (create_lane(r->req.grid, c, &l) != LS_OK) {
            r->status = LS_ENOMEM;
            r->phase = PH_DONE;
            r->t_done = std::chrono::steady_clock::now();
            it = queue.erase(it);
            continue;
          }
          s0 = 0;
        }
        r->lane = l;
        r->s0 = s0;
        for (int q = 0; q < r->n; ++q) l->owner[s0 + q] = r;
        l->to_start.push_back(r);
        it = queue.erase(it);
      }
    }
  }

  void fail(Request* r, int code) {
    r->status = code;
    if (r->lane && r->s0 >= 0) {
      // its slots stop iterating (they may lie inside the range the lane's next rounds launch over)
      Engine& e = r->lane->plan->eng;
      for (int q = 0; q < r->n; ++q) e.slots_h[r->s0 + q].flags = 0;
      upload_slots(r->lane, r->s0, r->n);
    }
    release(r);
  }

  void release(Request* r) {
    if (r->lane)
      for (int q = 0; q < r->n; ++q) r->lane->owner[r->s0 + q] = nullptr;
    r->t_done = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(mu);
    r->phase = PH_DONE;
  }

  void upload_slots(Lane* l, int s0, int n) {
    Engine& e = l->plan->eng;
    cudaMemcpyAsync(e.slots_d + s0, e.slots_h + s0, (size_t)n * sizeof(SlotDev), cudaMemcpyHostToDevice, l->stream);
  }

  void start_forward(Request* r) {
    Lane* l = r->lane;
    ls_plan* P = l->plan;
    Engine& e = P->eng;
    cudaStream_t st = l->stream;
    // plane waves into b, then x0 = b
    r->ptrs.assign(r->n, nullptr);
    for (int q = 0; q < r->n; ++q) r->ptrs[q] = e.vptr(V_B, r->s0 + q);
    cudaMemcpyAsync(engine_ptr_table(P, 0) + r->s0, r->ptrs.data(), r->n * sizeof(void*), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(e.kvec_d + 3 * (size_t)r->s0, r->kvec.data(), 3 * r->n * sizeof(double), cudaMemcpyHostToDevice, st);
    PlaneWaveParams a{P->nx, P->ny, P->nz, P->h, e.kvec_d + 3 * (size_t)r->s0,
                      (float2* const*)(engine_ptr_table(P, 0) + r->s0)};
    if (launch_plane_waves(a, r->n, st) != cudaSuccess) {
      fail(r, LS_ECUDA);
      return;
    }
    cudaMemcpyAsync(e.vptr(V_X, r->s0), e.vptr(V_B, r->s0), (size_t)r->n * e.N * sizeof(float2),
                    cudaMemcpyDeviceToDevice, st);
    for (int q = 0; q < r->n; ++q) slot_defaults(P, e.slots_h[r->s0 + q], r->req.f, 0);
    upload_slots(l, r->s0, r->n);
    r->phase = PH_FWD;
    l->n_resid += r->n;
  }

  // far field of the request's slots into the lane's far buffer
  void far_of(Request* r) {
    ls_plan v = plan_slot_view(r->lane->plan, r->s0);
    seq_far(&v, r->n, 0, r->lane->stream);
  }

  void finish_forward(Request* r) {
    Lane* l = r->lane;
    ls_plan* P = l->plan;
    Engine& e = P->eng;
    cudaStream_t st = l->stream;
    const size_t M = (size_t)P->mx * P->my;
    far_of(r);
    if (r->req.kind == LS_REQ_FORWARD) {
      if (r->req.far)
        cudaMemcpyAsync(r->req.far, e.far + (size_t)r->s0 * M, (size_t)r->n * M * sizeof(float2),
                        cudaMemcpyDeviceToDevice, st);
      if (r->req.u_out)
        cudaMemcpyAsync(r->req.u_out, e.vptr(V_X, r->s0), (size_t)r->n * e.N * sizeof(float2),
                        cudaMemcpyDeviceToDevice, st);
      r->phase = PH_FINISHING;   // outputs are complete after this lane's next readback
      return;
    }
    // gradient: residual r_q = far_q - y_q (in place) with ||r_q||^2 and ||y_q||^2
    if (r->req.u_out)
      cudaMemcpyAsync(r->req.u_out, e.vptr(V_X, r->s0), (size_t)r->n * e.N * sizeof(float2),
                      cudaMemcpyDeviceToDevice, st);
    r->ptrs.assign(3 * r->n, nullptr);
    for (int q = 0; q < r->n; ++q) {
      r->ptrs[q] = e.far + (size_t)(r->s0 + q) * M;
      r->ptrs[r->n + q] = (void*)((const float2*)r->req.meas + (size_t)q * M);
      r->ptrs[2 * r->n + q] = e.far + (size_t)(r->s0 + q) * M;
    }
    // tables 1 (pred), 2 (meas), 3 (res) of the lane, entries [s0, s0+n)
    for (int t = 0; t < 3; ++t)
      cudaMemcpyAsync(engine_ptr_table(P, t + 1) + r->s0, r->ptrs.data() + t * r->n, r->n * sizeof(void*),
                      cudaMemcpyHostToDevice, st);
    r->nb = (int)std::min<size_t>(kResidBlocks, (M + 255) / 256);
    double* part_d = e.partials + (size_t)r->s0 * e.maxparts * 4;
    ResidualParams rp{M, (const float2* const*)(engine_ptr_table(P, 1) + r->s0),
                      (const float2* const*)(engine_ptr_table(P, 2) + r->s0),
                      (float2* const*)(engine_ptr_table(P, 3) + r->s0), part_d};
    launch_residual(rp, r->nb, r->n, st);
    cudaMemcpyAsync(l->part_h + (size_t)r->s0 * kResidBlocks * 4, part_d, (size_t)r->n * r->nb * 4 * sizeof(double),
                    cudaMemcpyDeviceToHost, st);
    // b = G~^H r (the residual table sits in table 3 of the shifted view)
    ls_plan v = plan_slot_view(P, r->s0);
    seq_far_adjoint(&v, r->n, (const float2* const*)(engine_ptr_table(P, 3) + r->s0), 0, st);
    // keep the forward fields, start the adjoint solve from x0 = b
    cudaMemcpyAsync(e.ucache + (size_t)r->s0 * e.N, e.vptr(V_X, r->s0), (size_t)r->n * e.N * sizeof(float2),
                    cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(e.vptr(V_X, r->s0), e.vptr(V_B, r->s0), (size_t)r->n * e.N * sizeof(float2),
                    cudaMemcpyDeviceToDevice, st);
    for (int q = 0; q < r->n; ++q) slot_defaults(P, e.slots_h[r->s0 + q], r->req.f, 1);
    upload_slots(l, r->s0, r->n);
    r->phase = PH_ADJ;
    l->n_resid += r->n;
  }

  void finish_adjoint(Request* r) {
    Lane* l = r->lane;
    ls_plan* P = l->plan;
    Engine& e = P->eng;
    cudaStream_t st = l->stream;
    // weights c_q = 1/||y_q||^2 and the loss sum_q ||r_q||^2 / (2 ||y_q||^2) (eq. prob)
    std::vector<float>& w = r->weights;
    w.assign(r->n, 0.f);
    double loss = 0.0;
    const double* part_h = l->part_h + (size_t)r->s0 * kResidBlocks * 4;
    for (int q = 0; q < r->n; ++q) {
      double rr = 0, yy = 0;
      for (int b = 0; b < r->nb; ++b) {
        rr += part_h[((size_t)q * r->nb + b) * 4 + 0];
        yy += part_h[((size_t)q * r->nb + b) * 4 + 1];
      }
      const double c = yy > 0 ? 1.0 / yy : 0.0;
      w[q] = (float)c;
      loss += 0.5 * c * rr;
    }
    if (r->req.loss) *r->req.loss = loss;
    cudaMemcpyAsync(e.weights_d + r->s0, w.data(), r->n * sizeof(float), cudaMemcpyHostToDevice, st);
    r->ptrs.assign(r->n, nullptr);
    for (int q = 0; q < r->n; ++q) r->ptrs[q] = e.ucache + (size_t)(r->s0 + q) * e.N;
    cudaMemcpyAsync(engine_ptr_table(P, 2) + r->s0, r->ptrs.data(), r->n * sizeof(void*), cudaMemcpyHostToDevice, st);
    GradParams g{e.N, r->n, (const float2* const*)(engine_ptr_table(P, 2) + r->s0), e.vptr(V_X, r->s0), e.N,
                 e.weights_d + r->s0, r->req.grad};
    launch_gradient(g, st);
    r->phase = PH_FINISHING;
  }

  // -------------------------------------------------------------- one round over the lanes
  void issue(Lane* l) {
    TraceRange range("serve_round");
    ls_plan* P = l->plan;
    Engine& e = P->eng;
    cudaStream_t st = l->stream;
    for (Request* r : l->to_start) start_forward(r);
    l->to_start.clear();
    // launch over the occupied slot range only (requests take slots first-fit from 0)
    int lo = l->cap, hi = 0;
    for (int s = 0; s < l->cap; ++s)
      if (l->owner[s]) {
        lo = std::min(lo, s);
        hi = s + 1;
      }
    if (hi > lo) {
      ls_plan v = plan_slot_view(P, lo);
      if (l->n_resid > 0) seq_resid(&v, hi - lo, st);
      const int chunk = opt.iters_per_round > 0 ? opt.iters_per_round : kChunkDefault;
      if (l->n_iter > 0 || l->n_resid > 0)
        for (int k = 0; k < chunk; ++k) seq_iter(&v, hi - lo, st);
      cudaMemcpyAsync(e.slots_h + lo, e.slots_d + lo, (size_t)(hi - lo) * sizeof(SlotDev), cudaMemcpyDeviceToHost, st);
      // the z pass's error word (a TMA wait that gave up), read back with the slot states
      cudaMemcpyAsync(e.counts_h + 4, e.counts_d + 4, sizeof(int), cudaMemcpyDeviceToHost, st);
    }
    cudaEventRecord(l->ev, st);
    l->issued = true;
  }

  void process(Lane* l) {
    cudaError_t err = cudaEventQuery(l->ev);
    l->issued = false;
    Engine& e = l->plan->eng;
    if (err == cudaSuccess) err = cudaGetLastError();
    bool zfail = false;
    if (e.counts_h[4]) {
      // a round's z pass gave up on a copy: the round's results are invalid for every request in it
      zfail = true;
      e.counts_h[4] = 0;
      cudaMemsetAsync(e.counts_d + 4, 0, sizeof(int), l->stream);
    }
    l->n_iter = l->n_resid = 0;
    std::vector<Request*> seen;
    for (int s = 0; s < l->cap; ++s) {
      Request* r = l->owner[s];
      if (!r) continue;
      if (std::find(seen.begin(), seen.end(), r) != seen.end()) continue;
      seen.push_back(r);
    }
    for (Request* r : seen) {
      if (err != cudaSuccess || zfail) { fail(r, LS_ECUDA); continue; }
      if (r->phase == PH_FINISHING) {
        release(r);
        continue;
      }
      bool running = false;
      int worst = LS_OK;
      for (int q = 0; q < r->n; ++q) {
        const SlotDev& sd = e.slots_h[r->s0 + q];
        if (sd.flags & SLOT_ITER) { running = true; l->n_iter++; }
        if (sd.flags & SLOT_RESID) { running = true; l->n_resid++; }
        if (sd.status != LS_OK && (worst == LS_OK || sd.status == LS_BREAKDOWN)) worst = sd.status;
        r->iters_max = std::max(r->iters_max, sd.iters);
      }
      if (running) continue;
      if (worst != LS_OK && r->status == LS_OK) r->status = worst;
      if (r->phase == PH_FWD) finish_forward(r);
      else if (r->phase == PH_ADJ) finish_adjoint(r);
    }
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      admit();
      bool progressed = false, busy = false;
      for (size_t i = 0; i < lanes.size(); ++i) {
        Lane* l = lanes[i];
        if (l->issued && cudaEventQuery(l->ev) != cudaErrorNotReady) {
          process(l);
          progressed = true;
        }
        if (!l->issued && !lane_idle(l)) {
          issue(l);
          progressed = true;
        }
        busy = busy || l->issued;
      }
      if (progressed) continue;
      std::unique_lock<std::mutex> lk(mu);
      if (!busy && queue.empty()) {
        if (stop) break;
        cv.wait_for(lk, std::chrono::milliseconds(2));
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
    }
  }
};

extern "C" {

int ls_server_create(const ls_server_options* opt, ls_server** out) {
  if (!opt || !out) { set_last_error("null argument"); return LS_EINVAL; }
  *out = nullptr;
  if (!(opt->k_b > 0) || !(opt->voxel > 0) || !(opt->k_b * opt->voxel < 3.14159265358979)) {
    set_last_error("server needs k_b > 0, voxel > 0 and k_b voxel < pi");
    return LS_EINVAL;
  }
  ls_server* S = new ls_server();
  S->opt = *opt;
  if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; set_last_error("no CUDA device"); return LS_ECUDA; }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete S; set_last_error("cudaMemGetInfo failed"); return LS_ECUDA; }
  S->budget = opt->hbm_budget_bytes ? opt->hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
  S->worker = std::thread([S] { S->run(); });
  *out = S;
  return LS_OK;
}

int ls_submit(ls_server* S, const ls_request* req, uint64_t* ticket) {
  lsgpu::TraceRange trace_range("ls_submit");
  if (!S || !req || !ticket) { set_last_error("null argument"); return LS_EINVAL; }
  if (req->n_views < 1 || !req->f || !req->kvec) { set_last_error("request needs n_views >= 1, f and kvec"); return LS_EINVAL; }
  if (req->kind != LS_REQ_FORWARD && req->kind != LS_REQ_GRADIENT) { set_last_error("unknown request kind"); return LS_EINVAL; }
  if (req->kind == LS_REQ_GRADIENT && (!req->meas || !req->grad)) { set_last_error("gradient request needs meas and grad"); return LS_EINVAL; }
  const int L[3] = {2 * req->grid.nx, 2 * req->grid.ny, 2 * req->grid.nz};
  for (int i = 0; i < 3; ++i)
    if (L[i] != 16 && L[i] != 24 && L[i] != 32 && L[i] != 48 && L[i] != 64 && L[i] != 96 && L[i] != 128 &&
        L[i] != 192 && L[i] != 256 && L[i] != 384) {
      set_last_error("grid without an FFT length");
      return LS_EUNSUPPORTED;
    }
  if (S->opt.max_views_per_grid > 0 && req->n_views > S->opt.max_views_per_grid) {
    set_last_error("request has more views than a lane holds");
    return LS_EAGAIN;
  }
  if (plan_bytes(req->grid, req->n_views) > S->budget) {
    set_last_error("request needs %zu bytes, the budget is %zu", plan_bytes(req->grid, req->n_views), S->budget);
    return LS_EAGAIN;
  }
  Request* r = new Request();
  r->req = *req;
  r->n = req->n_views;
  r->kvec.assign(req->kvec, req->kvec + 3 * req->n_views);
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->queue.push_back(r);
    S->all[r->ticket] = r;
  }
  S->cv.notify_one();
  *ticket = r->ticket;
  return LS_OK;
}

int ls_poll(ls_server* S, uint64_t ticket, ls_result* res) {
  if (!S) { set_last_error("null server"); return LS_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) { set_last_error("unknown ticket"); return LS_ENOTFOUND; }
  Request* r = it->second;
  if (r->phase != PH_DONE) return LS_PENDING;
  const int status = r->status;
  if (res) {
    res->status = status;
    res->iterations_max = r->iters_max;
    res->submit_to_done_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  }
  S->all.erase(it);
  delete r;
  return status;
}

void ls_server_destroy(ls_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Lane* l : S->lanes) ls_server::destroy_lane(l);
  for (auto& kv : S->all) delete kv.second;
  delete S;
}

}  // extern "C"

"""Benchmark of the LS forward + adjoint hot path on GB300.

One step = one pass of the whole hot path over one batch: incident plane
waves for every view, the batched BiCGStab forward solves with the far field
on the detector, the residuals against synthetic measurements, and the
adjoint solves with the gradient accumulation.  The Green spectrum and the
far-field kernels are plan data built once per grid, outside the step.

Workload: 128^3 grid (padded 256^3), 60 plane-wave views on a cone of NA 0.8,
seeded phantom of 20 random ellipsoids (radii 4-20 voxels, dn in [0, 0.05]),
128 x 128 detector, BiCGStab tol 1e-6, complex64 fields.  Measurements are
the forward model of the phantom with 1% complex Gaussian noise; the
gradient is taken at 0.9 x the phantom's potential.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import phantoms as ph  # noqa: E402

METRIC = "LS matvec GB/s (%HBM) & solves/s at 128³×60 views; p50/p99 served solve latency"
WORKLOADS = {
    "bench": dict(shape=(128, 128, 128), views=60, count=20, rmin=4.0, rmax=20.0, dn_max=0.05),
    "small": dict(shape=(32, 32, 32), views=4, count=4, rmin=2.0, rmax=6.0, dn_max=0.05),
    # same grid and phantom as "bench" with 4 and 16 views: the cases the full ncu captures run on
    "profile": dict(shape=(128, 128, 128), views=4, count=20, rmin=4.0, rmax=20.0, dn_max=0.05),
    "profile16": dict(shape=(128, 128, 128), views=16, count=20, rmin=4.0, rmax=20.0, dn_max=0.05),
    # the 144^3 grid of the Fig. 3 bead at lambda/16 (288-point transforms) with 16 views: the case the
    # column-group z pass is captured on
    "profile144": dict(shape=(144, 144, 144), views=16, count=20, rmin=4.0, rmax=20.0, dn_max=0.05),
    # the 192^3 grid of the serving mix (384-point transforms) with 4 views (about 3.5 GB on the device)
    "profile192": dict(shape=(192, 192, 192), views=4, count=20, rmin=6.0, rmax=30.0, dn_max=0.05),
}
TOL = 1e-6
NA = 0.8


def workload_name(w):
    s = w["shape"]
    return f"LS forward+adjoint, {s[2]}x{s[1]}x{s[0]} grid (pad {2*s[2]}x{2*s[1]}x{2*s[0]}), {w['views']} views NA {NA}, " \
           f"{w['count']} ellipsoids dn<={w['dn_max']}, {s[2]}x{s[1]} detector, tol {TOL:g}"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


# ----------------------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


Z_SOURCES = ["paper_1910_13844_gb300/csrc/zpass.cuh", "paper_1910_13844_gb300/csrc/pass_common.cuh",
             "paper_1910_13844_gb300/csrc/dft.cuh", "paper_1910_13844_gb300/csrc/common.cuh"]


def opcodes_per_slot(kernel: str):
    """ncu's FP32 opcode counts per slot for `kernel` (FADD2, FFMA, FMUL), if recorded for the current source."""
    vals = {k: traffic_per_slot(kernel, f"{k}_per_slot") for k in ("fadd2", "ffma", "fmul")}
    return vals if all(v is not None for v in vals.values()) else None


def traffic_per_slot(kernel: str, field: str = "dram_bytes_per_slot"):
    """An ncu figure per slot for `kernel` (DRAM bytes, or FP32 pipe lane operations), if recorded for
    the current source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
    except Exception:
        return None
    rec = d.get(kernel)
    if not rec or rec.get("source_hash") != source_hash(Z_SOURCES) or field not in rec:
        return None
    return float(rec[field])


def alu_roofline(opcodes, launch_ms, views_per_launch, fp32_peak, sm_count):
    """The z pass against the FP32 pipe, with a measured denominator.

    opcodes: ncu's warp-level counts per view of the pass's FP32 instructions (FADD2, FFMA, FMUL);
    fp32_peak: lane operations per second of each kind measured on this GPU by ls_fp32_peak.  The
    pipe's time floor for one view is sum_op lanes(op) x count(op) / rate(op) (a packed FADD2 is 64
    lane operations); achieved = lane operations / live launch time, peak = lane operations / floor."""
    if not opcodes or not launch_ms or not fp32_peak:
        return None
    lanes = {"fadd2": 64.0, "ffma": 32.0, "fmul": 32.0}
    ops = sum(lanes[k] * opcodes[k] for k in lanes)
    floor_s = sum(lanes[k] * opcodes[k] / fp32_peak[k] for k in lanes)
    achieved = ops * views_per_launch / (launch_ms / 1e3) / 1e12
    peak = ops / floor_s / 1e12
    return {"kernel": "k_zw", "bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 2),
            "unit": "T FP32 lane-ops/s", "frac": round(achieved / peak, 4), "ops_per_view": int(ops),
            "peak_source": "measured: ls_fp32_peak (FFMA, FMUL, packed FADD2 microkernels) weighted by the "
                           "pass's ncu opcode mix", "fp32_peak_lane_ops_per_s": {k: round(v / 1e12, 2) for k, v in
                                                                                fp32_peak.items()},
            "sm_count": sm_count}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- CPU oracle timing
class OracleView:
    """The FP64 oracle's operator for the workload's grid and phantom (built once, untimed)."""

    def __init__(self, w):
        from oracle import green, model

        self.model = model
        shape = w["shape"]
        self.st = model.setup_from_optics(shape, ph.LAMBDA_UM, ph.ETA_B, ph.VOXEL_UM)
        self.op = model.Operator(self.st, kernel_method="prop1")
        dn = ph.random_ellipsoids(shape, count=w["count"], rmin=w["rmin"], rmax=w["rmax"], dn_max=w["dn_max"])
        self.f = green.scattering_potential(dn, ph.ETA_B, ph.LAMBDA_UM)
        self.k = ph.cone_directions(w["views"], NA, ph.ETA_B) * self.st.kb
        self.shape = shape

    def rhs(self, q, adjoint):
        """Right-hand side of view q (untimed): the incident plane wave (forward), or G~^H r for a
        seeded detector residual r (adjoint system of Alg. 1 line 6)."""
        uin = self.model.plane_wave(self.shape, self.st.h, self.k[q % len(self.k)])
        if not adjoint:
            return uin
        r = ph.complex_normal(self.st.det, seed=ph.SEED_NOISE + q)
        return self.op.farfield_adjoint_fft(r)

    def solve(self, q, seconds_budget, iters_per_solve=None, adjoint=False, b=None):
        """Times the oracle's BiCGStab for view q at the bench tolerance, x0 = b (the forward system, or
        the adjoint one).  A solve expected to take longer than the budget is cut after the iterations
        that fit it and scaled by iters_per_solve; otherwise it runs to convergence and is timed whole."""
        model = self.model
        uin = self.rhs(q, adjoint) if b is None else b
        A = lambda x: self.op.A(x, self.f, adjoint=adjoint)  # noqa: E731
        t1 = time.perf_counter()
        A(uin)
        t1 = time.perf_counter() - t1
        guess = iters_per_solve if iters_per_solve else 8.0
        if (2.0 * guess + 2.0) * t1 <= seconds_budget:
            t0 = time.perf_counter()
            _, it, _ = model.bicgstab(A, uin, tol=TOL, maxiter=1000)
            dt = time.perf_counter() - t0
            return {"seconds": dt, "iterations": it, "full_solve": True, "solves_per_s": 1.0 / dt,
                    "threads": os.cpu_count()}
        it = max(1, int(seconds_budget / (2.0 * t1)))
        t0 = time.perf_counter()
        _, it_done, _ = model.bicgstab(A, uin, tol=1e-30, maxiter=it)
        dt = time.perf_counter() - t0
        per_iter = dt / max(it_done, 1)
        return {"seconds": dt, "iterations": it_done, "full_solve": False,
                "solves_per_s": 1.0 / (per_iter * guess), "threads": os.cpu_count()}


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_13844_gb300 as ls

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    shape, Q = w["shape"], w["views"]
    kb = 2 * np.pi * ph.ETA_B / ph.LAMBDA_UM
    t_plan = time.perf_counter()
    # the plan's built-in illumination is the workload's cone (sin theta = NA / eta_b, phi_q = 2 pi q / Q)
    plan = ls.Plan(shape, kb, ph.VOXEL_UM, tol=TOL, cone_sin_theta=NA / ph.ETA_B)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    dn = ph.random_ellipsoids(shape, count=w["count"], rmin=w["rmin"], rmax=w["rmax"], dn_max=w["dn_max"],
                              seed=ph.SEED_PHANTOM + rank)
    dn_d = torch.from_numpy(dn.astype(np.float32)).to(dev)
    f_true = torch.empty_like(dn_d)
    ls.ls_scattering_potential(dn_d, ph.ETA_B, kb, f_true)
    f0 = 0.9 * f_true
    kvec = ph.cone_directions(Q, NA, ph.ETA_B) * kb
    # synthetic measurements: forward of the phantom + 1% complex Gaussian noise
    uin = plan.plane_waves(kvec)
    _, y, code, _ = plan.forward(f_true, uin, want_fields=False)
    noise = torch.from_numpy(ph.complex_normal((Q,) + plan.det).astype(np.complex64)).to(dev)
    ynorm = torch.linalg.vector_norm(y.reshape(Q, -1), dim=1)
    y = y + 0.01 * (ynorm / np.sqrt(2 * y[0].numel())).reshape(Q, 1, 1) * noise
    weights = (1.0 / (ynorm.double() ** 2)).cpu().numpy()

    # launch variants for this grid and batch, timed once before the warm-up (outside the timed region)
    tune = None if args.no_autotune else plan.autotune(Q, f0)

    u = plan.field(Q)
    far = plan.detector(Q)
    res = plan.detector(Q)
    grad = torch.empty(shape, dtype=torch.float32, device=dev)
    stats_acc = {"fwd_iters": [], "adj_iters": [], "status": []}

    def step(f_dev, y_dev):
        # incident plane waves generated inside the forward call, straight into the solver's vectors
        c1, s1 = ls.ls_forward(plan.handle, f_dev, None, u, far, n_views=Q)
        loss = ls.ls_residual(far, y_dev, res)
        c2, s2 = ls.ls_gradient(plan.handle, f_dev, res, grad, u_fwd=u, view_weights=weights)
        stats_acc["fwd_iters"].append(np.mean([s["iterations"] for s in s1]))
        stats_acc["adj_iters"].append(np.mean([s["iterations"] for s in s2]))
        stats_acc["status"].append(max(c1, c2))
        return 0.5 * float(np.sum(loss * weights))

    for _ in range(args.warmup):
        step(f0, y)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    ls.ls_profile(plan.handle, True)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(f0, y)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    prof = ls.ls_profile(plan.handle, False)
    clocks.stop()
    ms_total = ev0.elapsed_time(ev1)

    # end-to-end through the public API with host buffers (pinned), copies inside the timed region
    f_host = f0.cpu().pin_memory()
    y_host = y.cpu().pin_memory()
    g_host = torch.empty(shape, dtype=torch.float32).pin_memory()
    f_e = torch.empty_like(f0)
    y_e = torch.empty_like(y)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        f_e.copy_(f_host, non_blocking=True)
        y_e.copy_(y_host, non_blocking=True)
        step(f_e, y_e)
        g_host.copy_(grad, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = e0.elapsed_time(e1)

    # the five passes once more with every view active (ls_matvec_batch), for per-pass GB/s free of
    # the masked launches of converged views
    ls.ls_matvec_batch(plan.handle, f0, uin, u)
    torch.cuda.synchronize()
    ls.ls_profile(plan.handle, True)
    for _ in range(5):
        ls.ls_matvec_batch(plan.handle, f0, uin, u)
    torch.cuda.synchronize()
    iso = ls.ls_profile(plan.handle, False)
    cufft_us, cufft_diff = cufft_matvec_baseline(torch, ls, plan, f0, uin, u) if rank == 0 else (None, None)
    fp32_peak = ls.ls_fp32_peak()

    solves_per_step = 2 * Q
    ms_step = ms_total / args.steps
    ms_e2e_step = ms_e2e / args.steps
    if ws > 1:
        t = torch.tensor([ms_step, ms_e2e_step], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step, ms_e2e_step = float(t[0]), float(t[1])
    value = ws * solves_per_step / (ms_step / 1e3)
    e2e_value = ws * solves_per_step / (ms_e2e_step / 1e3)

    # roofline of the dominant kernel (the z pass: FFT, Green multiply, IFFT); bytes counted for the
    # slots that actually ran (converged views are masked off inside the launches)
    N = shape[0] * shape[1] * shape[2]
    nz, ny, nx = shape
    octant = 8 * (nx + 1) * (ny + 1) * (nz + 1)            # Green spectrum octant, read once per launch
    pass_bytes = {"fx": 28 * N, "fy": 48 * N, "z": 64 * N, "iy": 48 * N, "ix": 32 * N}   # plain-matvec model
    pass_gbs = {}
    mv_bytes = mv_ms = 0.0
    for k, b in pass_bytes.items():
        ms_k, launches_k, _, active_k = prof[k]
        byt = b * active_k + (octant * launches_k if k == "z" else 0)
        if ms_k > 0:
            pass_gbs[k] = round(byt / (ms_k / 1e3) / 1e9, 1)
        mv_bytes += byt
        mv_ms += ms_k
    iso_gbs = {}
    iso_bytes = iso_ms = 0.0
    for k, b in pass_bytes.items():
        ms_k, launches_k, _, active_k = iso[k]
        byt = b * active_k + (octant * launches_k if k == "z" else 0)
        if ms_k > 0:
            iso_gbs[k] = round(byt / (ms_k / 1e3) / 1e9, 1)
        iso_bytes += byt
        iso_ms += ms_k
    # BiCGStab update x += alpha p + omega s, r = s - omega t, <rh, r>: reads p, s, t, rh, x, writes x, r
    upd_ms, _, _, upd_active = prof.get("update", (0.0, 0, 0, 0))
    update_gbs = round(56 * N * upd_active / (upd_ms / 1e3) / 1e9, 1) if upd_ms > 0 else None
    z_ms, z_launches, _, z_active = prof["z"]
    active_per_launch = z_active / max(z_launches, 1)
    bytes_per_launch = 64 * N * active_per_launch + octant
    z_ms_launch = z_ms / max(z_launches, 1)
    achieved = bytes_per_launch / (z_ms_launch / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    tr = traffic_per_slot("z_pass")
    dominant = max((k for k in prof if k != "other"), key=lambda k: prof[k][0])
    total_kernel_ms = sum(v[0] for v in prof.values())
    launches = int(sum(v[1] for v in prof.values()))

    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64",
        "data": "synthetic",
        "config": {
            "workload": workload_name(w),
            "views": Q, "grid": list(shape[::-1]), "solves_per_step": solves_per_step,
            "l2": "inputs larger than L2 (per-view Krylov state 16 MiB x 8 vectors x 60 views)",
            "plan_build_s": round(t_plan, 3), "plan_built_once": True,
            "mean_forward_iterations": float(np.mean(stats_acc["fwd_iters"])),
            "mean_adjoint_iterations": float(np.mean(stats_acc["adj_iters"])),
            "worst_status": int(max(stats_acc["status"])),
            "parallelism": f"replicas{ws}" if ws > 1 else "single",
            "autotune": ({k: tune[k] for k in ("z_tma", "z_split", "z_persist", "strided_wide", "ix_prefetch", "fx_views_fastest", "fx_bulk",
                                               "views_per_launch", "check_every", "use_graphs", "from_cache")}
                         if tune else "off (defaults)"),
        },
        "roofline": {
            "kernel": "k_z (z-pencil FFT, Green multiply, inverse FFT, crop)",
            "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": (round(tr * active_per_launch) if tr is not None else None),
            "algorithmic_bytes_per_launch": int(bytes_per_launch),
            "launch_ms": round(z_ms_launch, 4), "active_views_per_launch": round(active_per_launch, 2),
        },
        "roofline_alu": alu_roofline(opcodes_per_slot("z_pass"), z_ms_launch, active_per_launch, fp32_peak,
                                     torch.cuda.get_device_properties(dev).multi_processor_count),
        "matvec": {
            "gbs": round(mv_bytes / (mv_ms / 1e3) / 1e9, 1) if mv_ms else None,
            "frac_hbm": round(mv_bytes / (mv_ms / 1e3) / 1e9 / peak, 4) if mv_ms else None,
            "us_per_view": round(1e3 * mv_ms / max(prof["z"][3], 1), 2),
            "pass_gbs": pass_gbs,
            "bytes_model": "plain matvec per view: F-x 28N, F-y 48N, Z 64N + Ghat octant per launch, I-y 48N, "
                           "I-x 32N bytes (the fused BiCGStab prologue/epilogue traffic is not counted)",
        },
        "matvec_all_views_active": {
            "gbs": round(iso_bytes / (iso_ms / 1e3) / 1e9, 1) if iso_ms else None,
            "frac_hbm": round(iso_bytes / (iso_ms / 1e3) / 1e9 / peak, 4) if iso_ms else None,
            "us_per_view": round(1e3 * iso_ms / max(iso["z"][3], 1), 2),
            "pass_gbs": iso_gbs,
            "how": f"ls_matvec_batch over all {Q} views, 5 launches per pass, same byte model",
        },
        "cufft_matvec": {
            "us_per_view": round(cufft_us, 2) if cufft_us else None,
            "ours_us_per_view": round(1e3 * iso_ms / max(iso["z"][3], 1), 2),
            "speedup": round(cufft_us / (1e3 * iso_ms / max(iso["z"][3], 1)), 3) if cufft_us and iso_ms else None,
            "max_rel_diff": cufft_diff,
            "how": "torch.fft (cuFFT) C2C 3-D on the zero-padded f x, full Green spectrum multiply, inverse, "
                   "crop, subtract; 10 views per batched transform; timed comparison only",
        },
        "update_gbs": update_gbs,
        "fp32_peak_tlane_ops": {k: round(v / 1e12, 2) for k, v in fp32_peak.items()},
        "kernel_share": {k: round(v[0] / total_kernel_ms, 4) for k, v in prof.items()} if total_kernel_ms else {},
        "dominant_kernel": dominant,
        "gpu_launches": launches,
        "e2e": {"value": round(e2e_value, 4), "unit": "solves/s",
                "h2d_bytes_per_step": int(f0.numel() * 4 + y.numel() * 8),
                "d2h_bytes_per_step": int(grad.numel() * 4)},
    }
    out["clocks"] = clocks.summary()
    if ws == 1 and args.serve_requests_in_step_line > 0 and args.workload == "bench":
        plan.close()
        plan = None
        torch.cuda.empty_cache()
        out["serving"] = run_serving(torch, ls, args.serve_requests_in_step_line, load=0.8)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        ov = OracleView(w)
        cbs = []
        for adj in (False, True):
            ips = float(np.mean(stats_acc["adj_iters" if adj else "fwd_iters"]))
            cbs.append(ov.solve(0, seconds_budget=15.0, iters_per_solve=ips, adjoint=adj, b=ov.rhs(0, adj)))
        sps = 2.0 / sum(1.0 / c["solves_per_s"] for c in cbs)
        how = "; ".join(
            (f"{kind}: one full solve of view 0 to tol {TOL:g}, {c['iterations']} iterations in {c['seconds']:.1f} s"
             if c["full_solve"] else
             f"{kind}: {c['iterations']} iterations of view 0 in {c['seconds']:.1f} s, scaled to the GPU run's mean "
             f"iterations per solve") for kind, c in zip(("forward", "adjoint"), cbs))
        out["cpu_baseline"] = {"value": round(sps, 6), "unit": "solves/s", "cores": cbs[0]["threads"],
                               "kind": "oracle",
                               "sample": f"FP64 oracle BiCGStab on the same workload, one forward solve (x0 = u_in) "
                                         f"and one adjoint solve (x0 = G~^H r) of view 0, solves/s = 2 / total time "
                                         f"(the GPU step is 60 forward + 60 adjoint solves): {how}; oracle kernel "
                                         f"build and right-hand sides excluded"}
    if rank == 0:
        print(json.dumps(out))
    if plan is not None:
        plan.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------- serving (continuous batching)
SERVE_GRIDS = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (192, 192, 192)]


def serve_requests(n, seed=2026):
    """Seeded request mix: grid uniform over SERVE_GRIDS, 8-60 views, 70% forward / 30% gradient."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        shape = SERVE_GRIDS[int(rng.integers(len(SERVE_GRIDS)))]
        out.append({"shape": shape, "views": int(rng.integers(8, 61)), "grad": bool(rng.random() < 0.3),
                    "seed": int(rng.integers(1 << 30))})
    return out


def cufft_matvec_baseline(torch, ls, plan, f, x, y_ours, reps=3, chunk=10):
    """The same operator x - G(f x) through cuFFT (torch.fft, timed comparison only, never on the product
    path): zero-pad f x to (2nz, 2ny, 2nx), C2C 3-D FFT, multiply by the full Green spectrum, inverse
    FFT, crop, subtract -- `chunk` views per batched transform.  Returns microseconds per view and the
    largest relative L2 difference from the library's result y_ours over the views."""
    nz, ny, nx = plan.shape
    Q = x.shape[0]
    ghat = torch.empty((2 * nz, 2 * ny, 2 * nx), dtype=torch.complex64, device=x.device)
    ls.ls_green_spectrum(plan.handle, plan.options.oversample_p, ghat)
    pad = torch.zeros((chunk, 2 * nz, 2 * ny, 2 * nx), dtype=torch.complex64, device=x.device)
    out = torch.empty_like(x)

    def apply():
        for q0 in range(0, Q, chunk):
            c = min(chunk, Q - q0)
            pad[:c, :nz, :ny, :nx] = f * x[q0:q0 + c]
            spec = torch.fft.fftn(pad[:c], dim=(-3, -2, -1))
            spec *= ghat
            v = torch.fft.ifftn(spec, dim=(-3, -2, -1))
            out[q0:q0 + c] = x[q0:q0 + c] - v[:, :nz, :ny, :nx]

    apply()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        apply()
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps / Q
    d = torch.linalg.vector_norm((out - y_ours).reshape(Q, -1), dim=1) / \
        torch.linalg.vector_norm(y_ours.reshape(Q, -1), dim=1)
    del pad, ghat
    torch.cuda.empty_cache()
    return us, float(d.max())


def run_serving(torch, ls, n_requests, load=0.8, seed=2026, calib=200, iters_per_round=0, baseline_views=16):
    """Poisson arrivals at `load` x the measured batched capacity; returns latency and throughput.

    The batched capacity is measured on a burst of `calib` requests of the same mix submitted at once
    (before the stream).  The comparison point is the same requests solved one view per call (the same
    kernels without batching): their time is the per-grid cost of one forward / one forward+adjoint view
    measured on this GPU, summed over the requests' views."""
    import time as _t

    kb = 2 * np.pi * ph.ETA_B / ph.LAMBDA_UM
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev)
    pot = {}

    def potential_for(shape, s):
        key = (shape, s % 4)
        if key not in pot:
            dn = ph.random_ellipsoids(shape, count=8, rmin=shape[0] / 32, rmax=shape[0] / 6, dn_max=0.05, seed=s % 4)
            dnd = torch.from_numpy(dn.astype(np.float32)).to(dev)
            f = torch.empty_like(dnd)
            ls.ls_scattering_potential(dnd, ph.ETA_B, kb, f)
            pot[key] = f
        return pot[key]

    def make(r):
        f = potential_for(r["shape"], r["seed"])
        k = ph.cone_directions(r["views"], NA, ph.ETA_B) * kb
        Q, (nz, ny, nx) = r["views"], r["shape"]
        far = torch.empty((Q, ny, nx), dtype=torch.complex64, device=dev)
        out = {"f": f, "k": k, "far": far}
        if r["grad"]:
            gen.manual_seed(r["seed"])
            out["meas"] = 1e-3 * torch.randn((Q, ny, nx), dtype=torch.complex64, device=dev, generator=gen)
            out["g"] = torch.empty(r["shape"], dtype=torch.float32, device=dev)
        return out

    def submit(srv, r, bufs):
        if r["grad"]:
            return srv.submit_gradient(bufs["f"], bufs["k"], bufs["meas"], bufs["g"])
        return srv.submit_forward(bufs["f"], bufs["k"], far=bufs["far"])

    solves = lambda r: r["views"] * (2 if r["grad"] else 1)  # noqa: E731
    reqs = serve_requests(n_requests + calib, seed)
    for r in reqs:   # every phantom is built on the host before any timing
        potential_for(r["shape"], r["seed"])
    srv = ls.Server(kb, ph.VOXEL_UM, tol=TOL, iters_per_round=iters_per_round)
    for shape in SERVE_GRIDS:   # build the lanes (plans) before measuring
        w = {"shape": shape, "views": 8, "grad": True, "seed": 0}
        srv.wait(submit(srv, w, make(w)))
    burst = [(r, make(r)) for r in reqs[:calib]]
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    tick = [submit(srv, r, b) for r, b in burst]
    for t in tick:
        srv.wait(t)
    t_burst = _t.perf_counter() - t0
    del burst
    cap_rps = calib / t_burst
    rate = load * cap_rps
    rng = np.random.default_rng(seed + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    pending, lat, total_solves, keep = {}, [], 0, {}
    stream = reqs[calib:calib + n_requests]
    t0 = _t.perf_counter()
    i = 0
    while i < n_requests or pending:
        now = _t.perf_counter() - t0
        while i < n_requests and arrivals[i] <= now:
            b = make(stream[i])
            t = submit(srv, stream[i], b)
            pending[t] = stream[i]
            keep[t] = b
            i += 1
        for t in list(pending):
            code, info = srv.poll(t)
            if code != ls.LS_PENDING:
                lat.append(info["ms"])
                total_solves += solves(pending.pop(t))
                keep.pop(t, None)
        _t.sleep(0.0005)
    wall = _t.perf_counter() - t0
    srv.close()
    # one view per call, per grid: seconds per forward view and per forward+adjoint view (median over
    # `baseline_views` views, after one untimed forward + gradient that pays for the plan's workspace
    # allocation, the iteration graph's capture and the kernels' first launches)
    per, spread = {}, {}
    for shape in SERVE_GRIDS:
        plan = ls.Plan(shape, kb, ph.VOXEL_UM, tol=TOL)
        r = {"shape": shape, "views": baseline_views, "grad": True, "seed": 1}
        b = make(r)

        def one(q):
            torch.cuda.synchronize()
            ts = _t.perf_counter()
            uin = plan.plane_waves(b["k"][q:q + 1])
            u, far, code, _ = plan.forward(b["f"], uin)
            torch.cuda.synchronize()
            tf = _t.perf_counter() - ts
            res = torch.empty_like(far)
            ls.ls_residual(far, b["meas"][q:q + 1].contiguous(), res)
            plan.gradient(b["f"], res, u_fwd=u)
            torch.cuda.synchronize()
            return tf, _t.perf_counter() - ts

        one(0)   # warm-up, untimed
        t = np.array([one(q) for q in range(r["views"])])
        per[shape] = (float(np.median(t[:, 0])), float(np.median(t[:, 1])))
        spread[shape] = [round(1e3 * float(np.percentile(t[:, k], p)), 2) for k in (0, 1) for p in (10, 90)]
        plan.close()
    t_base = sum(r["views"] * per[r["shape"]][1 if r["grad"] else 0] for r in stream)
    burst_reqs = reqs[:calib]
    burst_solves = sum(solves(r) for r in burst_reqs)
    t_base_burst = sum(r["views"] * per[r["shape"]][1 if r["grad"] else 0] for r in burst_reqs)
    lat = np.array(lat)
    return {
        "requests": n_requests, "load": load, "iters_per_round": iters_per_round or 2,
        "rate_rps": round(rate, 3), "capacity_rps": round(cap_rps, 3),
        "p50_ms": round(float(np.percentile(lat, 50)), 2), "p99_ms": round(float(np.percentile(lat, 99)), 2),
        "mean_ms": round(float(lat.mean()), 2), "solves_per_s": round(total_solves / wall, 2),
        "one_view_at_a_time_solves_per_s": round(total_solves / t_base, 2),
        "one_view_ms_per_view": {f"{s[0]}^3": [round(1e3 * v[0], 2), round(1e3 * v[1], 2)] for s, v in per.items()},
        "one_view_ms_p10_p90": {f"{s[0]}^3": v for s, v in spread.items()},
        "burst_requests": calib,
        "batched_capacity_solves_per_s": round(burst_solves / t_burst, 2),
        "one_view_capacity_solves_per_s": round(burst_solves / t_base_burst, 2),
        "batched_over_one_view": round(t_base_burst / t_burst, 3),
        "served_over_one_view": round(t_base / wall, 3),
        "mix": "grids {64,96,128,192}^3, 8-60 views, 70% forward / 30% gradient, dn <= 0.05, seed 2026; "
               f"capacity: a burst of {calib} requests of the mix submitted at once; one-view baseline: the "
               "same requests at the per-grid one-view cost (forward, forward+adjoint), median of "
               f"{baseline_views} single-view calls per grid after one untimed warm-up call; "
               "served_over_one_view: the stream's one-view time over its wall time at the offered load",
    }


def run_serve_mode(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_13844_gb300 as ls

    out = {"mode": "serve", "metric": METRIC}
    for load in args.loads:
        out[f"load_{load}"] = run_serving(torch, ls, args.requests, load=load, iters_per_round=args.iters_per_round)
    print(json.dumps(out))


# ----------------------------------------------------------------------------- reconstruction (FISTA + TV)
def run_fista_mode(args):
    """128^3, 60 views, ellipsoids with dn up to 0.1, FISTA with TV and positivity (Alg. 1),
    batched solves vs one view per call, compared at their final relative errors."""
    import time as _t

    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_13844_gb300 as ls
    from paper_1910_13844_gb300 import recon

    shape, Q = (128, 128, 128), 60
    kb = 2 * np.pi * ph.ETA_B / ph.LAMBDA_UM
    dn = ph.random_ellipsoids(shape, count=20, rmin=4, rmax=20, dn_max=0.1)
    dev = torch.device("cuda")
    dnd = torch.from_numpy(dn.astype(np.float32)).to(dev)
    f_true = torch.empty_like(dnd)
    ls.ls_scattering_potential(dnd, ph.ETA_B, kb, f_true)
    plan = ls.Plan(shape, kb, ph.VOXEL_UM, tol=TOL)
    kvec = ph.cone_directions(Q, NA, ph.ETA_B) * kb
    uin = plan.plane_waves(kvec)
    _, y, _, _ = plan.forward(f_true, uin, want_fields=False)
    noise = torch.from_numpy(ph.complex_normal(tuple(y.shape)).astype(np.complex64)).to(dev)
    yn = torch.linalg.vector_norm(y.reshape(Q, -1), dim=1)
    y = y + 0.01 * (yn / np.sqrt(2 * y[0].numel())).reshape(Q, 1, 1) * noise
    tune = plan.autotune(Q, f_true)    # launch variants for the 60-view batch (outside the timed runs)
    prob = recon.Problem(plan, kvec, y)
    f0 = torch.zeros_like(f_true)
    _, d0 = recon.data_grad(prob, f0)
    gamma0 = 0.5 * float(f_true.abs().max()) / float(d0.abs().max())
    out = {"mode": "fista", "workload": "128^3, 60 views NA 0.8, 20 ellipsoids dn <= 0.1, 1% noise, TV + positivity",
           "iterations": args.fista_iters, "gamma0": gamma0, "tau": args.tau,
           "autotune": {k: tune[k] for k in ("z_tma", "z_split", "z_persist", "strided_wide", "ix_prefetch", "fx_views_fastest", "fx_bulk",
                                             "views_per_launch", "check_every", "use_graphs")}}
    for name, batched, warm in (("batched", True, False), ("batched_warm_start", True, True),
                                ("one_view_at_a_time", False, False)):
        torch.cuda.synchronize()
        solver = []
        t0 = _t.perf_counter()
        st = recon.fista(prob, f0, args.fista_iters, gamma0=gamma0, tau=args.tau, tv_iters=10, batched=batched,
                         f_true=f_true, warm_start=warm, solver_stats=solver)
        torch.cuda.synchronize()
        out[name] = {"seconds": round(_t.perf_counter() - t0, 2), "final_rel_error": st.history[-1][2],
                     "final_loss": st.history[-1][1],
                     "mean_forward_iterations": round(float(np.mean([s["iterations"] for s in solver])), 3)}
    out["speedup_batched"] = round(out["one_view_at_a_time"]["seconds"] / out["batched"]["seconds"], 3)
    out["speedup_batched_warm_start"] = round(out["one_view_at_a_time"]["seconds"]
                                              / out["batched_warm_start"]["seconds"], 3)
    plan.close()
    print(json.dumps(out))


# ----------------------------------------------------------------------------- Fig. 3 bead
def run_bead_mode(args):
    """Forward solves of the Fig. 3 bead (homogeneous sphere of diameter 3 lambda, dn = 0.1 in a
    background of index 1.3388, 9 lambda box) at h = lambda/8 (72^3, 144-point transforms) and
    lambda/16 (144^3, 288-point transforms): one plane wave along z, and 16 views on the NA 0.8 cone,
    each batch timed with CUDA events after warm-up (plane waves + batched BiCGStab + far field)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1910_13844_gb300 as ls

    lam, eta_b, dn_bead = 0.532, 1.3388, 0.1
    box, radius = 9 * lam, 1.5 * lam
    kb = 2 * np.pi * eta_b / lam
    out = {"mode": "bead", "workload": "Fig. 3 bead: sphere diameter 3 lambda, dn 0.1, eta_b 1.3388, 9 lambda box, "
                                       "tol 1e-06"}
    for n in (72, 144):
        h = box / n
        shape = (n, n, n)
        plan = ls.Plan(shape, kb, h, tol=TOL)
        dnd = torch.from_numpy(ph.sphere(shape, radius / h, dn_bead).astype(np.float32)).cuda()
        f = torch.empty_like(dnd)
        ls.ls_scattering_potential(dnd, eta_b, kb, f)
        N = n ** 3
        octant = 8 * (n + 1) ** 3
        for Q in (1, 16):
            kvec = np.array([[0.0, 0.0, kb]]) if Q == 1 else ph.cone_directions(Q, NA, eta_b) * kb
            tune = plan.autotune(Q, f)
            uin = plan.field(Q)
            u = plan.field(Q)
            far = plan.detector(Q)
            stats = []

            def solve():
                ls.ls_plane_waves(plan.handle, kvec, uin)
                code, st = ls.ls_forward(plan.handle, f, uin, u, far)
                stats.append((code, st))

            for _ in range(2):
                solve()
            torch.cuda.synchronize()
            reps = 5
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                solve()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ls.ls_profile(plan.handle, True)
            solve()
            torch.cuda.synchronize()
            prof = ls.ls_profile(plan.handle, False)
            z_ms, z_launches, _, z_active = prof["z"]
            z_gbs = (64 * N * z_active + octant * z_launches) / (z_ms / 1e3) / 1e9 if z_ms else None
            its = [s["iterations"] for _, st in stats[-reps:] for s in st]
            out[f"{n}^3_{Q}_views"] = {
                "solves_per_s": round(Q / (ms / 1e3), 2), "ms_per_batch": round(ms, 3),
                "mean_iterations": float(np.mean(its)),
                "worst_status": int(max(c for c, _ in stats)),
                "z_pass_gbs": round(z_gbs, 1) if z_gbs else None,
                "z_kernel": ("k_zg (TMA-staged column groups)" if tune["z_tma"] else "k_z (cp.async staging)")
                if 2 * n in (144, 288) else ("k_zw" if tune["z_tma"] else "k_z (cp.async staging)"),
                "autotune": {k: tune[k] for k in ("z_tma", "z_split", "z_persist", "strided_wide", "ix_prefetch", "fx_views_fastest", "fx_bulk",
                                                  "views_per_launch", "check_every", "use_graphs")},
            }
        plan.close()
        torch.cuda.empty_cache()
    print(json.dumps(out))


# ----------------------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    budget = 20.0
    ov = OracleView(w)                 # the oracle's kernel build, outside the timed steps

    def step(q):
        # one forward and one adjoint solve of view q (right-hand sides built outside the timing)
        bf, ba = ov.rhs(q, False), ov.rhs(q, True)
        f_ = ov.solve(q, seconds_budget=budget, b=bf)
        a_ = ov.solve(q, seconds_budget=budget, adjoint=True, b=ba)
        return {"seconds": f_["seconds"] + a_["seconds"], "iterations": f_["iterations"] + a_["iterations"],
                "full_solve": f_["full_solve"] and a_["full_solve"],
                "solves_per_s": 2.0 / (1.0 / f_["solves_per_s"] + 1.0 / a_["solves_per_s"]), "threads": f_["threads"]}

    for q in range(args.warmup):
        step(q)
    samples = [step(args.warmup + q) for q in range(args.steps)]
    sps = float(np.median([s["solves_per_s"] for s in samples]))
    s0 = samples[0]
    full = all(s["full_solve"] for s in samples)
    how = ("each step: one forward solve (x0 = u_in) and one adjoint solve (x0 = G~^H r) of one view, each to "
           f"convergence by the FP64 oracle's BiCGStab (tol {TOL:g}; {np.mean([s['iterations'] for s in samples]):.1f} "
           "iterations per step on average), solves/s = 2 / step time; median over steps"
           if full else
           "each step: a bounded number of FP64 oracle BiCGStab iterations of one forward and one adjoint solve, "
           "scaled to 8 iterations per solve; median over steps")
    out = {
        "metric": METRIC, "value": round(sps, 6), "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.median([s["seconds"] for s in samples])), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "impl": "reference",
        "config": {"workload": workload_name(w), "views": w["views"], "oracle_processes": 1},
        "cpu_baseline": {"value": round(sps, 6), "unit": "solves/s", "cores": s0["threads"], "kind": "oracle",
                         "sample": how + (f"; launched on {ws} ranks, rank 0 alone runs the oracle" if ws > 1 else "")},
        "e2e": {"value": round(sps, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="bench", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch variants")
    ap.add_argument("--serve", action="store_true", help="serving benchmark (Poisson request stream) instead")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--loads", type=float, nargs="+", default=[0.5, 0.8, 1.0])
    ap.add_argument("--serve-requests-in-step-line", type=int, default=2000,
                    help="requests of the serving stream (0.8 load) added to the step line (0: none)")
    ap.add_argument("--iters-per-round", type=int, default=0, help="serving: iterations per lane round (0 = 2)")
    ap.add_argument("--fista", action="store_true", help="FISTA/TV reconstruction benchmark instead")
    ap.add_argument("--fista-iters", type=int, default=200)
    ap.add_argument("--tau", type=float, default=1e-6)
    ap.add_argument("--bead", action="store_true", help="Fig. 3 bead forward solves (72^3 and 144^3) instead")
    args = ap.parse_args()
    if args.bead:
        run_bead_mode(args)
        return
    if args.fista:
        run_fista_mode(args)
        return
    if args.serve:
        run_serve_mode(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

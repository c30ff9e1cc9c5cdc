"""Benchmark of the hybrid FEM/FDM inverse-problem hot path on GB300.

One step = one iteration of Algorithm 3 (hyb_cg_step): forward sweep (keeping
checkpoints or the FEM-region history), data misfit, exact adjoint sweep
(recomputing each checkpoint segment) with the fused FP64 gradient
accumulation, gradient + Tikhonov term, projected Fletcher-Reeves direction,
one trial forward for the step length and the projected update.

Workload (default, the large batched configuration): 257^3 lattice on
[-1,1]^3 (h = 1/128), FEM block nodes 64..192 (129^3), smooth Gaussian-bump
sigma with the voxels above 0.1 max sigma refined once, eight plane-wave
sources sin(40 t) advanced by the same launches (six faces, two body
diagonals), 3000 time steps, checkpoints every 50 steps, FP32 fields with
FP64 gradient and CG reductions, data = FP64 forward at the true coefficient
plus 3 % noise, gamma = 0.01, a in [1, 2.5]; the timed steps are the first
10 iterations of a CG loop started at a = 1.  A second record on the 129^3
single-source workload (whose fields fit in L2) follows.

Metric: lattice-node updates per second, n_src x (lattice + centre nodes) x
N_t x 2 (forward and adjoint) per CG iteration over the iteration's wall time
(which also holds the recompute and the trial forward); the count over every
sweep actually run is reported beside it.  Also: the roofline of the
dominant step kernel, the FP64 oracle on the host cores (one core and all
cores), an end-to-end figure with host buffers, serving latency, the SM
clocks during the timed region and the number of library kernels launched.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "forward+adjoint Glattice-updates/s and %HBM roofline; gradients/s + p50/p99 served"
UNIT = "Glattice-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10, help="timed CG iterations (the first K of a fresh loop)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="large_257", choices=["large_257", "inverse_129", "anisotropic_box"],
                   help="anisotropic_box: with --sweeps-only (its bench record is the anisotropic block)")
    p.add_argument("--nsteps", type=int, default=0, help="time steps (0: the workload's own)")
    p.add_argument("--e2e-steps", type=int, default=2, help="CG iterations of the end-to-end measurement")
    p.add_argument("--no-secondary", action="store_true", help="skip the 129^3 record")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-steps", type=int, default=30)
    p.add_argument("--serve-requests", type=int, default=512, help="requests of the serving stream (0: skip)")
    p.add_argument("--serve-workers", type=int, default=4)
    p.add_argument("--serve-batch", type=int, default=8, help="requests of one class per batched solve")
    p.add_argument("--serve-batch-work", type=float, default=6.5e9,
                   help="cap on a batch's lattice node-steps (default: about two 129^3 x 1500-step requests)")
    p.add_argument("--sources", type=int, default=0, help="with --sweeps-only: use the first K sources")
    p.add_argument("--no-refine", action="store_true", help="with --sweeps-only: the large workload unrefined")
    p.add_argument("--sweeps-only", type=int, default=0,
                   help="profiling aid: run this many forward+adjoint sweep pairs of the workload "
                        "(FP32, --nsteps steps, history kept) and exit without timing")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the step kernels' code (comments and blank lines left out, so
    that a comment edit keeps a recorded ncu figure valid)."""
    code = []
    for name in ("step_kernels.cu", "async_copy.cuh", "hyb_internal.h"):
        p = os.path.join(ROOT, "paper_1509_01399_gb300", "csrc", name)
        for ln in open(p, encoding="utf-8"):
            ln = ln.split("//", 1)[0].rstrip()
            if ln:
                code.append(ln)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_source_hash()
    for ln in open(path):
        f = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("workload") == workload and f.get("source") == h:
            try:
                return float(f["bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def make_workload(name, nsteps=0, refine=True):
    import synth
    if name == "large_257":
        return synth.large_257(refine=refine, **({"nsteps": nsteps} if nsteps else {}))
    if name == "anisotropic_box":
        return synth.anisotropic_box(**({"nsteps": nsteps} if nsteps else {}))
    return synth.inverse_129(**({"nsteps": nsteps} if nsteps else {}))


def algorithmic_bytes(w, info, n_src, es=4):
    """Algorithmic bytes of one forward and one adjoint launch: an FDM-owned
    node reads u^k, u^{k-1} and writes u^{k+1} (3 es); a FEM-owned node adds
    its coefficient (4 es; the adjoint also reads the stored u^k: 5 es); a
    centre node of a refined voxel likewise (4 es / 5 es).  Times the
    sources of the launch."""
    n_lat = w.n_nodes
    n_fo = int(info.n_fem_owned)
    nc = int(info.n_centres)
    fdm = n_lat - n_fo
    fwd = fdm * 3 * es + n_fo * 4 * es + nc * 4 * es
    adj = fdm * 3 * es + n_fo * 5 * es + nc * 5 * es
    return n_src * fwd, n_src * adj


def rel_l2(x, ref):
    import torch
    x = x.double()
    ref = ref.double()
    d = float(torch.linalg.vector_norm(ref))
    return float(torch.linalg.vector_norm(x - ref)) / (d if d > 0 else 1.0)


# ------------------------------------------------------------------ CG runs
def make_data(H, w, dev, m32):
    """Observations: per source, the FP64 forward at the true coefficient
    plus 3 % noise (one FP64 mesh per source, so that its checkpoints stay
    small).  Also returns, per source, the relative L2 difference between the
    FP32 trace at the true coefficient and the FP64 one."""
    import torch
    import synth
    srcs, nsteps, dt = w.sources, w.nsteps, w.dt
    tr32 = m32.forward(w.a_true(), srcs, nsteps, dt)
    obs = torch.zeros_like(tr32)
    errs = []
    m64 = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=w.ckpt_every, device=dev)
    for s, src in enumerate(srcs):
        tr64 = m64.forward(w.a_true(), [src], nsteps, dt)
        errs.append(rel_l2(tr32[s], tr64[0]))
        obs[s] = synth.add_noise_device(tr64[0], w.extra["noise"], w.extra["noise_seed"] + s).to(obs.dtype)
        del tr64
    m64.sync()
    m64.close()
    del tr32
    torch.cuda.empty_cache()
    return obs, errs


def run_telegraph(H, dev, nsteps=800, reps=3, sweep_levels=300):
    """The telegraph reading (damping sigma on the unknown voxels, a = 1) on
    the large workload's lattice, FEM block and eight sources (no
    refinement): sigma = the workload's Gaussian bumps generates the data
    (800 steps: the waves reach the damped region and come back to the
    faces), then `reps` gradient evaluations at half of it (forward with
    checkpoints every 50 steps, misfit, adjoint with recompute, gradient),
    timed with CUDA events; and the step launch times of sweeps with the
    history kept."""
    import numpy as np
    import torch
    import synth
    w = synth.large_257(nsteps=nsteps, refine=False)
    srcs, dt = w.sources, w.dt
    S = len(srcs)
    m = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=50, device=dev, model=H.HYB_MODEL_TELEGRAPH)
    sig_true = torch.tensor(w.sigma, dtype=torch.float64, device=dev)
    sig = 0.5 * sig_true
    obs = m.forward(sig_true, srcs, nsteps, dt).clone()

    def grad():
        tr = m.forward(sig, srcs, nsteps, dt)
        J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_QUADRATURE, want_cot=True)
        m.adjoint(cot)
        return m.gradient(sig, 0.0, 0.0), J

    grad()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(m.stream)
    for _ in range(reps):
        g, J = grad()
    ev1.record(m.stream)
    torch.cuda.synchronize(dev)
    el = ev0.elapsed_time(ev1) / reps
    gn = float(torch.linalg.vector_norm(g))
    m.close()
    nl = sweep_levels
    mr = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=0, device=dev, model=H.HYB_MODEL_TELEGRAPH)
    tr = mr.new_trace(S, nl)
    cot = torch.randn_like(tr) * 1e-3
    for _ in range(2):
        mr.forward(sig, srcs, nl, dt, tr)
        mr.adjoint(cot)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(mr.stream)
    mr.forward(sig, srcs, nl, dt, tr)
    e[1].record(mr.stream)
    mr.adjoint(cot)
    e[2].record(mr.stream)
    torch.cuda.synchronize(dev)
    mr.close()
    per = S * w.n_nodes * nsteps * 2
    return {"workload": "257^3 lattice, FEM block nodes 64..192, 8 sources, damping sigma on the unknown voxels "
                        "(the large workload's bumps), %d steps, checkpoints every 50, FP32" % nsteps,
            "gradient_ms": el, "value": per / (el * 1e-3) / 1e9, "unit": UNIT,
            "counted": "n_src x lattice nodes x N_t x 2 (forward + adjoint) per gradient evaluation",
            "forward_launch_ms": e[0].elapsed_time(e[1]) / nl, "adjoint_launch_ms": e[1].elapsed_time(e[2]) / nl,
            "J": J, "gnorm": gn}


def run_anisotropic(H, dev, peak, peak_kind, nsteps=600, reps=2, sweep_levels=100):
    """Per-axis lattice steps (the 257 x 193 x 321 box with steps 2/256,
    2/192, 2/320, eight sources, no refinement): data from the FP32 forward
    at the true coefficient, then `reps` gradient evaluations at
    a = 1 + sigma / 2 (forward with checkpoints every 50 steps, misfit,
    adjoint with recompute, gradient) timed with CUDA events; and the launch
    times of forward and transposed sweeps with the history kept, against
    the algorithmic bytes of a launch."""
    import torch
    import synth
    w = synth.anisotropic_box(nsteps)
    srcs, dt = w.sources, w.dt
    S = len(srcs)
    m = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=50, device=dev)
    info = m.query()
    a_true = torch.tensor(w.a_true(), dtype=torch.float64, device=dev)
    a = 1.0 + 0.5 * (a_true - 1.0)
    obs = m.forward(a_true, srcs, nsteps, dt).clone()

    def grad():
        tr = m.forward(a, srcs, nsteps, dt)
        J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_QUADRATURE, want_cot=True)
        m.adjoint(cot)
        return m.gradient(a, 0.0, 1.0), J

    grad()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(m.stream)
    for _ in range(reps):
        g, J = grad()
    ev1.record(m.stream)
    torch.cuda.synchronize(dev)
    el = ev0.elapsed_time(ev1) / reps
    gn = float(torch.linalg.vector_norm(g))
    m.close()
    nl = sweep_levels
    mr = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=0, device=dev)
    tr = mr.new_trace(S, nl)
    cot = torch.randn_like(tr) * 1e-3
    for _ in range(2):
        mr.forward(a, srcs, nl, dt, tr)
        mr.adjoint(cot)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(mr.stream)
    mr.forward(a, srcs, nl, dt, tr)
    e[1].record(mr.stream)
    mr.adjoint(cot)
    e[2].record(mr.stream)
    torch.cuda.synchronize(dev)
    mr.sync()
    mr.close()
    fwd_ms, adj_ms = e[0].elapsed_time(e[1]) / nl, e[1].elapsed_time(e[2]) / nl
    fb, ab = algorithmic_bytes(w, info, S)
    per = S * w.n_nodes * nsteps * 2
    roof = {}
    for k, b, ms in (("forward", fb, fwd_ms), ("adjoint", ab, adj_ms)):
        gbs = b / (ms * 1e-3) / 1e9
        roof[k] = {"kernel": ("ani_fwd_bulk_kernel<float> + ani_fwd_shell_kernel<float>" if k == "forward" else
                              "ani_adj_bulk_kernel<float> + ani_adj_shell_kernel<float>") + " (one level)",
                   "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                   "peak_kind": peak_kind, "algorithmic_bytes_per_launch": b, "launch_ms": ms}
    return {"workload": "257 x 193 x 321 lattice on [-1,1]^3, steps 2/256, 2/192, 2/320, FEM block = central half, "
                        "8 sources, no refinement, %d steps, checkpoints every 50, FP32 (bulk and face-shell kernels)" % nsteps,
            "gradient_ms": el, "value": per / (el * 1e-3) / 1e9, "unit": UNIT,
            "counted": "n_src x lattice nodes x N_t x 2 (forward + adjoint) per gradient evaluation",
            "roofline": roof, "J": J, "gnorm": gn}


def run_cg(H, w, dev, steps, warmup, e2e_steps, clocks=None):
    """W warm-up CG iterations, then the first K iterations of a fresh CG
    loop timed with CUDA events on the mesh's stream; per-iteration F and
    ||g||; the step kernels' launch times; the end-to-end figure."""
    import numpy as np
    import torch
    srcs, nsteps, dt = w.sources, w.nsteps, w.dt
    S = len(srcs)
    m = H.HybMesh.from_workload(w, precision="fp32", device=dev)
    info = m.query()
    t0 = time.perf_counter()
    obs, trace_errs = make_data(H, w, dev, m)
    data_s = time.perf_counter() - t0
    gamma, a0 = w.extra["gamma"], w.extra["a0"]
    stream = m.stream
    a = torch.ones(w.n_unknown, dtype=torch.float64, device=dev)
    state = m.new_cg_state()

    def step():
        return m.cg_step(a, obs, srcs, nsteps, dt, state, gamma=gamma, a0=a0, a_min=1.0, a_max=w.a_max)

    for _ in range(warmup):
        step()
    a.fill_(1.0)  # the timed iterations are the first K of a fresh loop
    state = m.new_cg_state()
    torch.cuda.synchronize(dev)
    if clocks:
        clocks.start()
    l0 = m.launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = [step() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop() if clocks else None
    el_ms = ev0.elapsed_time(ev1)
    launches = m.launches() - l0
    a_final = a.clone()
    # step-kernel launch times: sweeps of a shorter run with the history kept
    # (no checkpoint copies, no recompute), same launches per level
    nl = min(nsteps, 300)
    mr = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=0, device=dev)
    tr = mr.new_trace(S, nl)
    cot = torch.randn_like(tr) * 1e-3
    for _ in range(2):  # the second call captures the sweep graphs
        mr.forward(a_final, srcs, nl, dt, tr)
        mr.adjoint(cot)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(mr.stream)
    mr.forward(a_final, srcs, nl, dt, tr)
    e[1].record(mr.stream)
    e[2].record(mr.stream)
    mr.adjoint(cot)
    e[3].record(mr.stream)
    torch.cuda.synchronize(dev)
    fwd_ms = e[0].elapsed_time(e[1]) / nl
    adj_ms = e[2].elapsed_time(e[3]) / nl
    mr.sync()
    mr.close()
    del tr, cot
    # end to end through the C ABI with host buffers: observations and the
    # coefficient copied in from pinned host memory, the coefficient back
    obs_host = obs.cpu().pin_memory()
    a_host = torch.ones(w.n_unknown, dtype=torch.float64).pin_memory()
    a_back = torch.empty_like(a_host).pin_memory()
    st2 = m.new_cg_state()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        obs.copy_(obs_host, non_blocking=True)
        a.copy_(a_host, non_blocking=True)
        m.cg_step(a, obs, srcs, nsteps, dt, st2, gamma=gamma, a0=a0, a_min=1.0, a_max=w.a_max)
        a_back.copy_(a, non_blocking=True)
        torch.cuda.synchronize(dev)
        a_host.copy_(a_back)
    e2e_s = time.perf_counter() - t0
    h2d = obs_host.numel() * obs_host.element_size() + a_host.numel() * 8
    d2h = a_back.numel() * 8 + 64
    m.sync()
    m.close()
    del obs, obs_host
    torch.cuda.empty_cache()
    n_nodes = w.n_nodes + int(info.n_centres)
    sweeps_run = 4 if w.ckpt_every else 3  # forward, (recompute,) adjoint, trial forward
    return dict(w=w, info=info, el_ms=el_ms, reps=reps, launches=launches, clocks=clk, fwd_ms=fwd_ms,
                adj_ms=adj_ms, e2e_s=e2e_s, h2d=h2d, d2h=d2h, n_nodes=n_nodes, S=S, sweeps_run=sweeps_run,
                trace_errs=trace_errs, data_s=data_s, a_final=a_final)


def fp32_vs_fp64_gradient(H, w, dev):
    """FP32 and FP64 forward + misfit + adjoint + gradient at a = 1 on the
    same observations (the FP64 forward at the true coefficient): relative
    L2 difference of the gradients and of J."""
    import torch
    out = {}
    m64 = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=w.ckpt_every, device=dev)
    obs64 = m64.forward(w.a_true(), w.sources, w.nsteps, w.dt).clone()
    res = {}
    for prec, dtype in (("fp64", torch.float64), ("fp32", torch.float32)):
        m = m64 if prec == "fp64" else H.HybMesh.from_workload(w, precision="fp32", device=dev)
        a = torch.ones(w.n_unknown, dtype=torch.float64, device=dev)
        tr = m.forward(a, w.sources, w.nsteps, w.dt)
        J, cot = m.misfit(tr, obs64.to(dtype), H.HYB_WEIGHTS_QUADRATURE, want_cot=True)
        m.adjoint(cot)
        res[prec] = (J, m.gradient(a, w.extra["gamma"], w.extra["a0"]).clone())
        m.sync()
        if prec == "fp32":
            m.close()
    m64.close()
    out["gradient_rel_l2"] = rel_l2(res["fp32"][1], res["fp64"][1])
    out["J_rel"] = abs(res["fp32"][0] - res["fp64"][0]) / abs(res["fp64"][0])
    return out


def cg_record(r, steps):
    """Line fields of one CG run."""
    w, S = r["w"], r["S"]
    el_s = r["el_ms"] * 1e-3
    per_step = S * r["n_nodes"] * w.nsteps
    return dict(
        value=steps * 2 * per_step / el_s / 1e9,
        all_sweeps=steps * r["sweeps_run"] * per_step / el_s / 1e9,
        ms_per_step=r["el_ms"] / steps,
        gradients_per_s=steps / el_s,
        cg={"iterations": steps, "F": [rp.J for rp in r["reps"]], "gnorm": [rp.gnorm for rp in r["reps"]],
            "alpha": [rp.alpha for rp in r["reps"]], "beta": [rp.beta for rp in r["reps"]],
            "F_first": r["reps"][0].J, "F_last": r["reps"][-1].J})


def roofline(r, peak, peak_kind, workload):
    w, S = r["w"], r["S"]
    fwd_b, adj_b = algorithmic_bytes(w, r["info"], S)
    # launches per CG iteration: forward, recompute (checkpointing), trial
    # forward; one adjoint sweep
    n_fwd = r["sweeps_run"] - 1
    t_fwd, t_adj = n_fwd * r["fwd_ms"], r["adj_ms"]
    fwd_dom = t_fwd >= t_adj
    name = "step_kernel<float,forward>" if fwd_dom else "step_kernel<float,adjoint>"
    b, ms = (fwd_b, r["fwd_ms"]) if fwd_dom else (adj_b, r["adj_ms"])
    ach = b / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": peak_kind, "traffic": recorded_traffic(name, workload),
            "algorithmic_bytes_per_launch": b, "launch_ms": ms, "time_share": max(t_fwd, t_adj) / (t_fwd + t_adj),
            "fwd": {"launch_ms": r["fwd_ms"], "bytes": fwd_b, "frac": fwd_b / (r["fwd_ms"] * 1e-3) / 1e9 / peak},
            "adj": {"launch_ms": r["adj_ms"], "bytes": adj_b, "frac": adj_b / (r["adj_ms"] * 1e-3) / 1e9 / peak}}


# ------------------------------------------------------------ CPU baseline
def _oracle_sample_worker(args):
    """One process: the oracle (as it stands) on the sample lattice, k
    forward + k adjoint steps of one source.  Returns (node updates, s)."""
    steps, src_index = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    import numpy as np
    import oracle
    import synth
    w = synth.large_batched(129, nsteps=steps)
    P = oracle.problem_from_workload(w)
    src = w.sources[src_index % len(w.sources)]
    a = w.a_true()
    t0 = time.perf_counter()
    res = P.forward(a, src, steps, w.dt, keep_hist=True)
    cot = np.random.default_rng(0).standard_normal(res["trace"].shape)
    P.adjoint(a, src, steps, w.dt, cot, res["hist"])
    el = time.perf_counter() - t0
    return 2.0 * (w.n_nodes + P.NC) * steps, el


CPU_SAMPLE = ("the large workload's recipe (FEM central half, Gaussian bumps, voxels above 0.1 max sigma refined, "
              "face and diagonal sources) on a 129^3 lattice (h = 1/64): %d forward + %d adjoint steps of one "
              "source per process; building the oracle on the 257^3 lattice alone takes ~30 s and 15 GB per process")


def cpu_baseline(sample_steps, all_cores=True):
    """The FP64 oracle timed on the host cores: one process on one core, and
    one process per core (spawned) on the same sample, each its own source."""
    import multiprocessing as mp
    import platform
    ctx = mp.get_context("spawn")
    out = {"kind": "oracle", "sample": CPU_SAMPLE % (sample_steps, sample_steps), "unit": UNIT}
    with ctx.Pool(1) as pool:
        n, el = pool.map(_oracle_sample_worker, [(sample_steps, 6)])[0]
    out.update(value=n / el / 1e9, cores=1, seconds=el)
    cpu_model = platform.processor() or platform.machine()
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                cpu_model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    nproc = os.cpu_count() or 1
    out["nproc"] = nproc
    out["cpu_model"] = cpu_model + " (" + platform.machine() + ")"
    if all_cores and nproc > 1:
        t0 = time.perf_counter()
        with ctx.Pool(nproc) as pool:
            res = pool.map(_oracle_sample_worker, [(sample_steps, i) for i in range(nproc)])
        wall = time.perf_counter() - t0
        out["all_cores"] = {"value": sum(r[0] for r in res) / max(r[1] for r in res) / 1e9, "cores": nproc,
                            "seconds": max(r[1] for r in res), "wall_with_setup_s": wall}
    return out


# ------------------------------------------------------------------ serving
def run_serving(args, dev):
    """Serving stream: FP32 forward + adjoint + gradient solves on lattices
    drawn from {33, 65, 97, 129}^3 (FEM block = central half, 2-4 inclusions,
    400-1500 steps by size).  Capacity is measured with requests arriving
    back to back; the stream then arrives as a Poisson process at 80% of it,
    served in batches and, for comparison, one request per solve.
    Beside it, the FP64 path with one request at a time on a sample of the
    same requests, and each sampled FP32 gradient's relative L2 difference
    from its FP64 counterpart."""
    import numpy as np
    import synth
    from paper_1509_01399_gb300.serve import Request, ServingEngine, latency_stats, poisson_arrivals
    R = args.serve_requests
    eng = ServingEngine(workers=args.serve_workers, device=str(dev), max_batch=args.serve_batch,
                        batch_work=args.serve_batch_work)
    sizes = (33, 65, 97, 129)
    warm = []
    for N in sizes:  # pools and sweep graphs of every class, outside timing
        i = next(i for i in range(1000) if synth.serving_request(i).n[0] == N)
        warm += [Request(-1 - len(warm), synth.serving_request(i), 0.0) for _ in range(3)]
    eng.run(warm)
    cap_n = min(R, 128)
    cap = eng.run([Request(i, synth.serving_request(i), 0.0) for i in range(cap_n)])
    mu = latency_stats(cap)["solves_per_s"]
    lam = 0.8 * mu
    arr = poisson_arrivals(R, lam, seed=3)
    res = eng.run([Request(i, synth.serving_request(i), float(arr[i])) for i in range(R)])
    st = latency_stats(res)
    batches = {"batches": eng.batches, "max_batch": eng.max_batch_seen}
    eng.close()
    # the same arrivals served one request per solve (no batching), for comparison
    e1 = ServingEngine(workers=args.serve_workers, device=str(dev), max_batch=1)
    e1.run(warm)
    st1 = latency_stats(e1.run([Request(i, synth.serving_request(i), float(arr[i])) for i in range(R)]))
    e1.close()
    n64 = min(R, 16)
    e64 = ServingEngine(workers=1, precision="fp64", device=str(dev), max_batch=1)
    e64.run([Request(-1, synth.serving_request(i), 0.0) for i in range(2)])
    r64 = e64.run([Request(i, synth.serving_request(i), 0.0) for i in range(n64)])
    e64.close()
    lat64 = np.array([r.finish - r.start for r in r64])
    errs = []
    for r in r64:
        g32 = res[r.rid].gradient
        errs.append(float(np.linalg.norm(g32 - r.gradient) / np.linalg.norm(r.gradient)))
    return {"requests": R, "workers": args.serve_workers, "max_batch": args.serve_batch,
            "batch_work": args.serve_batch_work, **batches,
            "capacity_solves_per_s": mu, "rate_per_s": lam,
            "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "dtype": "f32",
            "unbatched_same_arrivals": {"solves_per_s": st1["solves_per_s"], "p50_ms": st1["p50_ms"],
                                        "p99_ms": st1["p99_ms"]},
            "grad_rel_err_vs_fp64": {"max": max(errs), "median": float(np.median(errs)), "requests": len(errs)},
            "fp64_one_at_a_time": {"sample": n64, "solves_per_s": float(n64 / lat64.sum()),
                                   "p50_ms": float(np.percentile(lat64, 50) * 1e3),
                                   "p99_ms": float(np.percentile(lat64, 99) * 1e3)}}


# ---------------------------------------------------------------- reference
def run_reference(args):
    """The oracle, as it stands, on the host cores: each step one bounded
    sample (one process, one core) of the workload's scheme."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    s = max(2, args.cpu_sample_steps // 3)
    times, vals = [], []
    with ctx.Pool(1) as pool:
        for i in range(args.warmup + args.steps):
            n, el = pool.map(_oracle_sample_worker, [(s, 6)])[0]
            if i >= args.warmup:
                vals.append(n / el / 1e9)
                times.append(el)
    value = statistics.median(vals)
    w = make_workload(args.workload, args.nsteps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name + " (oracle sample, see cpu_baseline)", "parallelism": "one host core"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": CPU_SAMPLE % (s, s)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- sweeps only
def run_sweeps_only(args):
    """Forward + adjoint sweeps of the workload with its sources, for ncu
    captures: no data generation, no CG, no timing."""
    import torch
    from paper_1509_01399_gb300 import hyb as H
    w = make_workload(args.workload, args.nsteps, refine=not args.no_refine)
    srcs = w.sources[: args.sources] if args.sources > 0 else w.sources
    m = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=0)
    a = torch.tensor(w.a_true(), dtype=torch.float64, device="cuda")
    tr = m.new_trace(len(srcs), w.nsteps)
    cot = torch.randn_like(tr) * 1e-3
    for _ in range(args.sweeps_only):
        m.forward(a, srcs, w.nsteps, w.dt, tr)
        m.adjoint(cot)
    m.sync()
    m.close()
    print(json.dumps({"sweeps": args.sweeps_only, "workload": w.name, "nsteps": w.nsteps, "sources": len(srcs)}))
    return 0


# --------------------------------------------------------------------- ours
def describe(w):
    srcs = ", ".join(("face %d" % s.face) if s.direction is None else
                     ("dir (%g,%g,%g)" % tuple(s.direction)) for s in w.sources)
    ref = int(w.refine.sum()) if w.refine is not None else 0
    return ("%s: %d^3 lattice h=1/%d, FEM block nodes %d..%d, %d refined voxels, %d sources [%s], %d steps "
            "dt=%.6g, checkpoints every %d, FP32 fields, FP64 gradient and CG reductions"
            % (w.name, w.n[0], round(1 / w.h), w.fem_lo[0], w.fem_hi[0], ref, len(w.sources), srcs, w.nsteps,
               w.dt, w.ckpt_every))


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (one all-reduce; the identity
    without a process group): the timed region of N replicas ends when the
    slowest one does."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    from paper_1509_01399_gb300 import hyb as H

    rank, world, local = dist_env()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_steps)  # spawned before the first GPU call
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_workload(args.workload, args.nsteps)
    peak, peak_kind = measured_peak()
    if dist:
        dist.barrier()
    r = run_cg(H, w, dev, args.steps, args.warmup, args.e2e_steps, clocks=ClockSampler(local))
    el_ms = r["el_ms"]
    if dist:
        r["el_ms"] = el_ms = max_over_ranks(el_ms, dist, dev)
        dist.barrier()
    rec = cg_record(r, args.steps)
    per_step = r["S"] * r["n_nodes"] * w.nsteps
    e2e_value = world * args.e2e_steps * 2 * per_step / r["e2e_s"] / 1e9
    line = {"metric": METRIC, "value": world * rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(w), "n_nodes": w.n_nodes, "n_centres": int(r["info"].n_centres),
                       "sources": r["S"], "nsteps": w.nsteps,
                       "counted": "n_src x (lattice + centre nodes) x N_t x 2 (forward + adjoint) per CG iteration",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: 8 x 68.7 MB per field level, 6.3 GB observation trace"},
            "lattice_updates_all_sweeps": {"value": world * rec["all_sweeps"], "unit": UNIT,
                                           "sweeps_per_step": r["sweeps_run"]},
            "gradients_per_s": world * rec["gradients_per_s"],
            "roofline": roofline(r, peak, peak_kind, w.name),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": r["h2d"],
                    "d2h_bytes_per_step": r["d2h"], "steps": args.e2e_steps},
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
            "cg": rec["cg"],
            "fp32_trace_rel_err_vs_fp64": {"max": max(r["trace_errs"]), "per_source": r["trace_errs"],
                                           "at": "true coefficient, all steps"}}
    del r
    torch.cuda.empty_cache()
    if dist:  # the secondary record, serving and the baselines: rank 0 alone
        dist.barrier()
        dist.destroy_process_group()
        dist = None
        if rank != 0:
            return 0
    if not args.no_secondary and args.workload != "inverse_129":
        w2 = make_workload("inverse_129")
        r2 = run_cg(H, w2, dev, 20, 3, 2)
        rec2 = cg_record(r2, 20)
        err = fp32_vs_fp64_gradient(H, w2, dev)
        line["secondary"] = {
            "workload": describe(w2) + " (the three field levels fit in the 126 MB L2: its roofline fraction is "
                                       "bytes over time, not DRAM bandwidth)",
            "value": rec2["value"], "lattice_updates_all_sweeps": rec2["all_sweeps"],
            "ms_per_step": rec2["ms_per_step"], "gradients_per_s": rec2["gradients_per_s"],
            "roofline_l2_resident": roofline(r2, peak, peak_kind, w2.name), "cg": rec2["cg"],
            "fp32_vs_fp64": {"trace_rel_l2": max(r2["trace_errs"]), **err}}
        del r2
        torch.cuda.empty_cache()
    if not args.no_secondary and args.workload != "inverse_129":
        from paper_1509_01399_gb300 import hyb as H
        line["telegraph"] = run_telegraph(H, dev)
        torch.cuda.empty_cache()
        line["anisotropic"] = run_anisotropic(H, dev, peak, peak_kind)
        torch.cuda.empty_cache()
    if args.serve_requests > 0:
        line["serving"] = run_serving(args, dev)
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.sweeps_only:
        return run_sweeps_only(args)
    if args.workload == "anisotropic_box":
        sys.exit("--workload anisotropic_box needs --sweeps-only")
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

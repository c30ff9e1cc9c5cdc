"""Benchmark of the hybrid FEM/FDM inverse-problem hot path on GB300.

One step = one iteration of Algorithm 3 (hyb_cg_step): forward sweep with the
FEM-region history kept, data misfit, exact adjoint sweep with the fused FP64
gradient accumulation, gradient + Tikhonov term, Fletcher-Reeves direction,
one trial forward for the step length and the projected update.

Workload (default): 129^3 lattice on [-1,1]^3 (h = 1/64), FEM block nodes
32..96 (65^3), three random cubic inclusions sigma ~ U[0.5, 2], 1500 time
steps at the CFL step for a_max = 5, plane wave sin(40 t) from the top face,
data = FP64 forward at the true coefficient + 3% Gaussian noise, FP32 fields
with FP64 gradient and CG reductions, gamma = 0.01, a0 = 1, a in [1, 5].

Metric: lattice-node updates per second over the three sweeps of a step
(forward, adjoint, trial forward).  Also reported: the roofline of the
dominant step kernel, the FP64 oracle on the host cores as a CPU baseline,
an end-to-end figure with host buffers, the SM clocks during the timed
region and the number of library kernels launched.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
L2_NOTE = "inputs larger than L2: per-step u history 1.5 GB and observation trace 100 MB"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=6)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--nsteps", type=int, default=1500, help="time steps of the workload")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-steps", type=int, default=30)
    p.add_argument("--serve-requests", type=int, default=512, help="requests of the serving stream (0: skip)")
    p.add_argument("--serve-workers", type=int, default=8)
    p.add_argument("--workload", default="inverse_129", choices=["inverse_129", "large_257"])
    p.add_argument("--sources", type=int, default=0, help="with --sweeps-only: use the first K sources")
    p.add_argument("--sweeps-only", type=int, default=0,
                   help="profiling aid: run this many forward+adjoint sweep pairs of the workload "
                        "(FP32, --nsteps steps) and exit without timing")
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
    p = os.path.join(ROOT, "paper_1509_01399_gb300", "csrc", "step_kernels.cu")
    code = []
    for ln in open(p, encoding="utf-8"):
        ln = ln.split("//", 1)[0].rstrip()
        if ln:
            code.append(ln)
    return hashlib.sha256("\n".join(code).encode()).hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    h = kernel_source_hash()
    for ln in open(path):
        f = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("source") == h:
            try:
                return float(f["bytes_per_launch"])
            except (KeyError, ValueError):
                return None
    return None


def make_workload(nsteps, name="inverse_129"):
    import synth
    if name == "large_257":
        return synth.large_257(nsteps=nsteps)
    return synth.inverse_129(nsteps=nsteps)


def run_sweeps_only(args):
    """Forward + adjoint sweeps of the workload with all its sources, for
    ncu captures: no data generation, no CG, no timing."""
    import torch
    from paper_1509_01399_gb300 import hyb as H
    w = make_workload(args.nsteps, args.workload)
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
    print(json.dumps({"sweeps": args.sweeps_only, "workload": w.name, "nsteps": w.nsteps,
                      "sources": len(srcs)}))
    return 0


def algorithmic_bytes(w, es=4):
    """Algorithmic bytes per launch: FDM-owned node reads u^k,
    u^{k-1} and writes u^{k+1} (3 es); a FEM-owned node adds its coefficient
    (forward) and, in the adjoint, the stored u^k (4 es / 5 es)."""
    n_nodes = w.n_nodes
    fo = 1
    for d in range(3):
        fo *= (w.fem_hi[d] - w.fem_lo[d] - 1)
    fdm = n_nodes - fo
    return fdm * 3 * es + fo * 4 * es, fdm * 3 * es + fo * 5 * es, fdm, fo


# ------------------------------------------------------------ CPU baseline
def oracle_sample(w, sample_steps):
    """Time the FP64 oracle (as it stands) on a bounded sample of the
    workload: `sample_steps` forward steps and the same number of adjoint
    steps on the full 129^3 lattice.  Returns lattice updates per second."""
    import numpy as np
    import oracle
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a = np.ones(P.n_unknown)
    t0 = time.perf_counter()
    res = P.forward(a, src, sample_steps, w.dt, keep_hist=True)
    cot = np.random.default_rng(0).standard_normal(res["trace"].shape)
    P.adjoint(a, src, sample_steps, w.dt, cot, res["hist"])
    el = time.perf_counter() - t0
    return 2.0 * w.n_nodes * sample_steps / el / 1e9, el


# ------------------------------------------------------------------ serving
def run_serving(args, dev):
    """Serving stream: FP32 forward + adjoint + gradient solves on lattices
    drawn from {33, 65, 97, 129}^3 (FEM block = central half, 2-4 inclusions,
    400-1500 steps by size).  Capacity is measured with requests arriving
    back to back; the stream then arrives as a Poisson process at 80% of it.
    Beside it, the FP64 path with one request at a time."""
    import numpy as np
    import synth
    from paper_1509_01399_gb300.serve import Request, ServingEngine, latency_stats, poisson_arrivals
    R = args.serve_requests
    eng = ServingEngine(workers=args.serve_workers, device=str(dev))
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
    eng.close()
    # FP64 path, one request at a time, on a sample of the same stream
    n64 = min(R, 16)
    e64 = ServingEngine(workers=1, precision="fp64", device=str(dev))
    e64.run([Request(-1, synth.serving_request(i), 0.0) for i in range(2)])
    r64 = e64.run([Request(i, synth.serving_request(i), 0.0) for i in range(n64)])
    e64.close()
    lat64 = np.array([r.finish - r.start for r in r64])
    return {"requests": R, "workers": args.serve_workers, "capacity_solves_per_s": mu, "rate_per_s": lam,
            "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "dtype": "f32",
            "fp64_one_at_a_time": {"sample": n64, "solves_per_s": float(n64 / lat64.sum()),
                                   "p50_ms": float(np.percentile(lat64, 50) * 1e3),
                                   "p99_ms": float(np.percentile(lat64, 99) * 1e3)}}


# ---------------------------------------------------------------- reference
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args.nsteps)
    times, vals = [], []
    s = max(2, args.cpu_sample_steps // 3)
    for i in range(args.warmup + args.steps):
        v, el = oracle_sample(w, s)
        if i >= args.warmup:
            vals.append(v)
            times.append(el)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "inverse_129 (oracle sample: %d forward + %d adjoint steps on 129^3)" % (s, s),
                       "parallelism": "host cores, one process"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d forward + %d adjoint steps of the 129^3 workload per step" % (s, s)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- ours
def run_ours(args):
    import numpy as np
    import torch
    import synth
    from paper_1509_01399_gb300 import hyb as H

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = make_workload(args.nsteps)
    srcs = w.sources
    nsteps, dt = w.nsteps, w.dt

    # data: FP64 forward at the true coefficient + 3% noise (outside timing)
    m64 = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0, device=dev)
    obs64 = m64.forward(w.a_true(), srcs, nsteps, dt)
    m64.sync()
    obs_np = synth.add_noise(obs64.cpu().numpy(), w.extra["noise"], w.extra["noise_seed"])
    m64.close()
    del obs64
    m = H.HybMesh.from_workload(w, precision="fp32", ckpt_every=0, device=dev)
    obs = torch.from_numpy(obs_np.astype(np.float32)).to(dev)
    a = torch.ones(w.n_unknown, dtype=torch.float64, device=dev)
    state = m.new_cg_state()
    stream = m.stream
    gamma, a0 = w.extra["gamma"], w.extra["a0"]

    def step():
        return m.cg_step(a, obs, srcs, nsteps, dt, state, gamma=gamma, a0=a0, a_min=1.0, a_max=w.a_max)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = m.launches()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    reps = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = clk.stop()
    el_ms = ev0.elapsed_time(ev1)
    launches = m.launches() - l0
    if dist:
        t = torch.tensor([el_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el_ms = float(t.item())
        dist.barrier()
    sweeps = 3
    updates = sweeps * w.n_nodes * nsteps * len(srcs)
    value = world * args.steps * updates / (el_ms * 1e-3) / 1e9
    grads_per_s = world * args.steps / (el_ms * 1e-3)

    # roofline of the step kernels: forward and adjoint sweeps timed alone
    peak, peak_kind = measured_peak()
    fwd_b, adj_b, n_fdm, n_fo = algorithmic_bytes(w)
    trace = m.new_trace(len(srcs), nsteps)
    for _ in range(2):
        m.forward(a, srcs, nsteps, dt, trace)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m.forward(a, srcs, nsteps, dt, trace)
    e1.record(stream)
    J, cot = m.misfit(trace, obs, H.HYB_WEIGHTS_QUADRATURE, want_cot=True)
    for _ in range(2):  # the second call captures the adjoint sweep graph
        m.adjoint(cot)
    e1b = torch.cuda.Event(enable_timing=True)
    e1b.record(stream)
    m.adjoint(cot)
    e2.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1) / nsteps
    adj_ms = e1b.elapsed_time(e2) / nsteps
    dom = "step_kernel<float,adjoint>" if adj_ms >= fwd_ms else "step_kernel<float,forward>"
    dom_ms, dom_b = (adj_ms, adj_b) if adj_ms >= fwd_ms else (fwd_ms, fwd_b)
    achieved = dom_b / (dom_ms * 1e-3) / 1e9
    traffic = recorded_traffic(dom)

    # end to end through the public API with host buffers
    obs_host = torch.from_numpy(obs_np.astype(np.float32)).pin_memory()
    a_host = torch.ones(w.n_unknown, dtype=torch.float64).pin_memory()
    a_back = torch.empty_like(a_host).pin_memory()
    obs_dev = torch.empty_like(obs)
    st2 = m.new_cg_state()
    a_dev = torch.empty_like(a)
    for _ in range(1):
        obs_dev.copy_(obs_host, non_blocking=True)
        a_dev.copy_(a_host, non_blocking=True)
        m.cg_step(a_dev, obs_dev, srcs, nsteps, dt, st2, gamma=gamma, a0=a0, a_min=1.0, a_max=w.a_max)
        a_back.copy_(a_dev, non_blocking=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        obs_dev.copy_(obs_host, non_blocking=True)
        a_dev.copy_(a_host, non_blocking=True)
        m.cg_step(a_dev, obs_dev, srcs, nsteps, dt, st2, gamma=gamma, a0=a0, a_min=1.0, a_max=w.a_max)
        a_back.copy_(a_dev, non_blocking=True)
        torch.cuda.synchronize(dev)
        a_host.copy_(a_back)
    e2e_s = time.perf_counter() - t0
    e2e_value = world * args.steps * updates / e2e_s / 1e9
    h2d = obs_host.numel() * 4 + a_host.numel() * 8
    d2h = a_back.numel() * 8 + 64

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "inverse_129: 129^3 lattice h=1/64, FEM block 65^3 (nodes 32..96), "
                                   "3 cubic inclusions sigma~U[0.5,2], %d steps, FP32 fields, FP64 gradient "
                                   "accumulation and CG reductions, one CG iteration per step" % nsteps,
                       "n_nodes": w.n_nodes, "nsteps": nsteps, "sweeps_per_step": sweeps,
                       "parallelism": "replicas" if world > 1 else "single GPU", "l2": L2_NOTE},
            "gradients_per_s": grads_per_s,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_launch": dom_b, "launch_ms": dom_ms,
                         "fwd_launch_ms": fwd_ms, "adj_launch_ms": adj_ms},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "cg": {"J_first": reps[0].J, "J_last": reps[-1].J, "gnorm_last": reps[-1].gnorm}}
    m.close()
    del obs, obs_dev, a_dev, trace, cot
    torch.cuda.empty_cache()
    if args.serve_requests > 0:
        line["serving"] = run_serving(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, el = oracle_sample(w, args.cpu_sample_steps)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "%d forward + %d adjoint steps of the 129^3 workload (%.1f s)"
                                          % (args.cpu_sample_steps, args.cpu_sample_steps, el)}
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
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

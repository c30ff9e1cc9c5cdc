"""Serving form: continuous batching of forward + adjoint + gradient solves.

A request is one FP32 solve on its own lattice (Model Problem 2 with its own
coefficient a = 1 + sigma): the forward sweep records the trace on the
source face, the misfit against the observations gives the cotangent, the
exact adjoint sweep accumulates dJ/da (Eq. (gradient1)) and the gradient is
copied to the host.

The engine keeps a pool of meshes per lattice class (size, FEM block, step
count, source) resident on the device, with their fields and checkpoints.
A request is admitted as soon as a worker is free and a mesh of its class is
free, or a new one fits in the HBM budget; otherwise it waits.  Each worker
owns a CUDA stream, so the solves of all admitted requests run concurrently
on the GPU, and requests that arrive while others are in flight join as
soon as a slot and memory free up.  A request's arithmetic depends only on
its own mesh and inputs, so its result is the same alone and in a mix.
"""
from __future__ import annotations

import math
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
import torch

from . import hyb as H


@dataclass
class Request:
    rid: int
    workload: object          # a synth.Workload (lattice, FEM block, sources, steps, sigma)
    arrival: float = 0.0      # seconds after the start of the stream


@dataclass
class Result:
    rid: int
    gradient: np.ndarray
    J: float
    arrival: float
    start: float
    finish: float
    mesh_class: tuple

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def class_key(w, precision) -> tuple:
    srcs = tuple((s.face, s.omega, getattr(s, "amp", 1.0)) for s in w.sources)
    return (tuple(w.n), tuple(w.fem_lo), tuple(w.fem_hi), tuple(w.bc), w.nsteps, w.dt, w.h, w.a_max, srcs,
            precision)


def estimate_bytes(w, precision) -> int:
    """Device bytes one pooled mesh of this class holds after a solve."""
    es = 8 if precision == "fp64" else 4
    N = ((w.n[0] + 3) // 4 * 4) * w.n[1] * w.n[2]  # rows padded to a multiple of 4
    fn = [w.fem_hi[d] - w.fem_lo[d] - 1 for d in range(3)]
    nown = (fn[0] + 6) * fn[1] * fn[2]  # history box rows padded and aligned
    un = [max(0, v - 1) for v in fn]
    nu = un[0] * un[1] * un[2]
    wsz = (fn[0] + 2) * (fn[1] + 2) * (fn[2] + 2)
    stride = max(w.n[0] * w.n[1], w.n[0] * w.n[2], w.n[1] * w.n[2])
    ns = len(w.sources)
    trace = ns * (w.nsteps + 1) * stride * es
    return int(6 * ns * N * es + w.nsteps * ns * nown * es + 3 * wsz * es + 8 * nu * (ns + 2) + 3 * trace
               + (1 << 20))


class _Pooled:
    def __init__(self, mesh: H.HybMesh, key, nbytes: int):
        self.mesh = mesh
        self.key = key
        self.nbytes = nbytes
        self.trace = None
        self.grad = None


class ServingEngine:
    """Continuous-batching solve engine on one GPU.

    hbm_budget: bytes of device memory the pooled meshes may hold (default:
    half of the free memory at start).  workers: concurrent solves (one CUDA
    stream each)."""

    def __init__(self, hbm_budget: Optional[int] = None, workers: int = 8, precision: str = "fp32",
                 device: str = "cuda:0"):
        self.device = torch.device(device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.5 * free)
        self.budget = int(hbm_budget)
        self.workers = int(workers)
        self.precision = precision
        self._cv = threading.Condition()
        self._free: Dict[tuple, List[_Pooled]] = {}
        self._used = 0
        self._meshes: List[_Pooled] = []
        self._obs: Dict[tuple, torch.Tensor] = {}
        self._obs_lock = threading.Lock()
        self._streams = [torch.cuda.Stream(self.device) for _ in range(self.workers)]
        self._stream_free = list(range(self.workers))
        self.in_flight = 0
        self.max_in_flight = 0
        self.max_meshes = 0

    # ---------------------------------------------------------- admission
    def _acquire(self, w) -> _Pooled:
        key = class_key(w, self.precision)
        need = estimate_bytes(w, self.precision)
        if need > self.budget:
            raise H.HybError(H.HYB_ERR_OOM, f"request needs ~{need} bytes, above the HBM budget {self.budget}")
        with self._cv:
            while True:
                lst = self._free.get(key)
                if lst:
                    return lst.pop()
                if self._used + need <= self.budget:
                    self._used += need
                    break
                # evict an idle mesh of another class if that makes room
                victim = None
                for k, l in self._free.items():
                    if l:
                        victim = l.pop()
                        break
                if victim is not None:
                    self._used -= victim.nbytes
                    self._meshes.remove(victim)
                    victim.mesh.close()
                    continue
                self._cv.wait()
        mesh = H.HybMesh.from_workload(w, precision=self.precision, ckpt_every=0, device=self.device)
        p = _Pooled(mesh, key, need)
        with self._cv:
            self._meshes.append(p)
            self.max_meshes = max(self.max_meshes, len(self._meshes))
        return p

    def _release(self, p: _Pooled):
        with self._cv:
            self._free.setdefault(p.key, []).append(p)
            self._cv.notify_all()

    def _stream(self) -> int:
        with self._cv:
            while not self._stream_free:
                self._cv.wait()
            s = self._stream_free.pop()
            self.in_flight += 1
            self.max_in_flight = max(self.max_in_flight, self.in_flight)
            return s

    def _stream_done(self, s: int):
        with self._cv:
            self._stream_free.append(s)
            self.in_flight -= 1
            self._cv.notify_all()

    # --------------------------------------------------------------- solve
    def observations(self, w) -> torch.Tensor:
        """Observed trace of a request class: the recorded trace of the
        background medium a = 1 (so the misfit is the scattered field)."""
        key = class_key(w, self.precision)
        with self._obs_lock:
            if key not in self._obs:
                m = H.HybMesh.from_workload(w, precision=self.precision, ckpt_every=0, device=self.device)
                self._obs[key] = m.forward(np.ones(m.n_unknown), w.sources, w.nsteps, w.dt).clone()
                m.sync()
                m.close()
            return self._obs[key]

    def solve(self, req: Request, t0: float = 0.0) -> Result:
        w = req.workload
        obs = self.observations(w)
        s = self._stream()
        stream = self._streams[s]
        start = time.perf_counter() - t0
        try:
            with torch.cuda.stream(stream):
                p = self._acquire(w)
                try:
                    m = p.mesh
                    m.set_stream(stream)
                    if p.trace is None:
                        p.trace = m.new_trace(len(w.sources), w.nsteps)
                        p.cot = torch.empty_like(p.trace)
                        p.a = torch.empty(m.n_unknown, dtype=torch.float64, device=self.device)
                        p.grad = torch.empty(m.n_unknown, dtype=torch.float64, device=self.device)
                        p.host = torch.empty(m.n_unknown, dtype=torch.float64).pin_memory()
                    p.a.copy_(torch.from_numpy(1.0 + np.asarray(w.sigma, dtype=np.float64)), non_blocking=False)
                    H.hyb_forward(m.handle, p.a.data_ptr(), w.sources, w.nsteps, w.dt, p.trace.data_ptr())
                    J = H.hyb_misfit(m.handle, p.trace.data_ptr(), obs.data_ptr(), H.HYB_WEIGHTS_PLAIN, True,
                                     p.cot.data_ptr())
                    H.hyb_adjoint(m.handle, p.cot.data_ptr(), 0)
                    H.hyb_gradient(m.handle, p.a.data_ptr(), 0.0, 1.0, p.grad.data_ptr())
                    p.host.copy_(p.grad, non_blocking=True)
                    H.hyb_sync(m.handle)
                    g = p.host.numpy().copy()
                finally:
                    self._release(p)
        finally:
            self._stream_done(s)
        finish = time.perf_counter() - t0
        return Result(req.rid, g, J, req.arrival, start, finish, class_key(w, self.precision))

    # -------------------------------------------------------------- stream
    def run(self, requests: List[Request]) -> List[Result]:
        """Serve requests arriving at their `arrival` times (seconds from now):
        a dispatcher hands each one, at its arrival, to a pool of `workers`
        threads; it starts as soon as a worker and memory allow.  Returns the
        results in request order."""
        for r in requests:  # observation traces are inputs, prepared up front
            self.observations(r.workload)
        torch.cuda.synchronize(self.device)
        order = sorted(requests, key=lambda r: r.arrival)
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=self.workers) as ex:
            futs = []
            for r in order:
                delay = r.arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                futs.append(ex.submit(self.solve, r, t0))
            done = {f.result().rid: f.result() for f in futs}
        return [done[r.rid] for r in requests]

    def close(self):
        with self._cv:
            for p in self._meshes:
                p.mesh.close()
            self._meshes.clear()
            self._free.clear()
            self._used = 0


def poisson_arrivals(n: int, rate: float, seed: int = 3) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n)) - 0.0


def latency_stats(results: List[Result]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "solves_per_s": len(results) / span, "requests": len(results)}

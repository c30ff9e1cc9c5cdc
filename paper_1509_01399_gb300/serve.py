"""Serving form: continuous, iteration-level batching of forward + adjoint +
gradient solves.

A request is one FP32 solve on its own lattice (Model Problem 2 with its own
coefficient a = 1 + sigma): the forward sweep records the trace on the
source face, the misfit against the observations gives the cotangent, the
exact adjoint sweep accumulates dJ/da (Eq. (gradient1)) and the gradient is
copied to the host.

The engine keeps a pool of meshes per lattice class (size, FEM block, step
count, source) resident on the device, with their fields and checkpoints.
Arriving requests queue by class; a worker takes up to max_batch waiting
requests of one class and advances them together: one launch per time level
carries every request of the batch as its own slot with its own coefficient
(hyb_forward_batch), and the per-request misfits, adjoints and gradients
follow in the same way.  A batch is admitted as soon as a worker is free and
a mesh of its class is free, or a new one fits in the HBM budget; otherwise
it waits.  Each worker owns a CUDA stream, so batches of different classes
run concurrently on the GPU, and requests that arrive while others are in
flight join the next batch of their class.  A slot's arithmetic depends only
on its own coefficient and source, so a request's result is the same alone
and in a batch.
"""
from __future__ import annotations

import math
import threading
import time
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
        self.bufs = None


class ServingEngine:
    """Continuous-batching solve engine on one GPU.

    hbm_budget: bytes of device memory the pooled meshes may hold (default:
    half of the free memory at start).  workers: concurrent batches (one CUDA
    stream each).  max_batch: requests of one lattice class advanced by the
    same launches (iteration-level batching, hyb_forward_batch).  batch_work:
    cap on a batch's lattice node-steps (nodes x time levels, summed over its
    requests; at least one request): small lattices batch up to max_batch,
    large ones in small batches, so that a batch's time, which every request
    in it waits for, stays bounded (None: no cap)."""

    def __init__(self, hbm_budget: Optional[int] = None, workers: int = 8, precision: str = "fp32",
                 device: str = "cuda:0", max_batch: int = 8, batch_work: Optional[float] = None):
        self.device = torch.device(device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.5 * free)
        self.budget = int(hbm_budget)
        self.workers = int(workers)
        self.max_batch = max(1, min(int(max_batch), H.MAX_SOURCES))
        self.batch_work = batch_work
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
        self.max_batch_seen = 0
        self.batches = 0

    # ---------------------------------------------------------- admission
    def _acquire(self, w) -> _Pooled:
        key = class_key(w, self.precision)
        need = estimate_bytes(w, self.precision) * self.max_batch
        if need > self.budget:
            raise H.HybError(H.HYB_ERR_OOM, f"a batch needs ~{need} bytes, above the HBM budget {self.budget}")
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

    def _buffers(self, p: _Pooled, w, obs):
        """Per-mesh device arrays for a batch of up to max_batch requests:
        coefficients, observations (the class's, once per slot), trace,
        cotangent, gradients, and the pinned host copy of the gradients."""
        if p.bufs is None:
            B, m = self.max_batch, p.mesh
            tr = torch.zeros((B, w.nsteps + 1, m.obs_stride), dtype=m.dtype, device=self.device)
            p.bufs = dict(a=torch.empty((B, m.n_unknown), dtype=torch.float64, device=self.device),
                          obs=obs.expand(B, -1, -1).contiguous(), trace=tr, cot=torch.empty_like(tr),
                          g=torch.empty((B, m.n_unknown), dtype=torch.float64, device=self.device),
                          host=torch.empty((B, m.n_unknown), dtype=torch.float64).pin_memory())
        return p.bufs

    def solve_batch(self, reqs: List[Request], t0: float = 0.0) -> List[Result]:
        """One batched solve of requests of one class: forward, per-request
        misfit, adjoint and per-request gradient, all requests advanced by the
        same launches on the worker's stream."""
        w = reqs[0].workload
        obs = self.observations(w)
        s = self._stream()
        stream = self._streams[s]
        start = time.perf_counter() - t0
        b = len(reqs)
        try:
            with torch.cuda.stream(stream):
                p = self._acquire(w)
                try:
                    m = p.mesh
                    m.set_stream(stream)
                    bf = self._buffers(p, w, obs)
                    host_a = np.stack([1.0 + np.asarray(r.workload.sigma, dtype=np.float64) for r in reqs])
                    bf["a"][:b].copy_(torch.from_numpy(host_a), non_blocking=False)
                    srcs = [r.workload.sources[0] for r in reqs]
                    H.hyb_forward_batch(m.handle, bf["a"].data_ptr(), srcs, w.nsteps, w.dt, bf["trace"].data_ptr())
                    J = H.hyb_misfit_batch(m.handle, bf["trace"].data_ptr(), bf["obs"].data_ptr(),
                                           H.HYB_WEIGHTS_PLAIN, b, bf["cot"].data_ptr())
                    H.hyb_adjoint(m.handle, bf["cot"].data_ptr(), 0)
                    H.hyb_gradient_batch(m.handle, bf["a"].data_ptr(), 0.0, 1.0, bf["g"].data_ptr())
                    bf["host"][:b].copy_(bf["g"][:b], non_blocking=True)
                    H.hyb_sync(m.handle)
                    g = bf["host"][:b].numpy().copy()
                finally:
                    self._release(p)
        finally:
            self._stream_done(s)
        finish = time.perf_counter() - t0
        with self._cv:
            self.batches += 1
            self.max_batch_seen = max(self.max_batch_seen, b)
        key = class_key(w, self.precision)
        return [Result(r.rid, g[i], J[i], r.arrival, start, finish, key) for i, r in enumerate(reqs)]

    def batch_size(self, w) -> int:
        """Requests of w's class that one batch takes: max_batch, lowered so
        that the batch's node-steps stay within batch_work."""
        if self.batch_work is None:
            return self.max_batch
        work = float(np.prod(w.n)) * w.nsteps
        return max(1, min(self.max_batch, int(self.batch_work // work)))

    def solve(self, req: Request, t0: float = 0.0) -> Result:
        return self.solve_batch([req], t0)[0]

    # -------------------------------------------------------------- stream
    def run(self, requests: List[Request]) -> List[Result]:
        """Serve requests arriving at their `arrival` times (seconds from now).
        Arrivals join a queue per lattice class; each of `workers` threads
        takes the class whose oldest request has waited longest and solves up
        to max_batch of its waiting requests in one batch, so requests that
        arrive while others are on the GPU join the next batch of their class
        as soon as a worker and memory free up.  Returns the results in
        request order."""
        for r in requests:  # observation traces are inputs, prepared up front
            self.observations(r.workload)
        torch.cuda.synchronize(self.device)
        order = sorted(requests, key=lambda r: r.arrival)
        queues: Dict[tuple, List[Request]] = {}
        qcv = threading.Condition()
        done: Dict[int, Result] = {}
        state = {"pending": len(order), "error": None}
        t0 = time.perf_counter()

        def worker():
            while True:
                with qcv:
                    while True:
                        if state["pending"] == 0 or state["error"] is not None:
                            return
                        ready = [(q[0].arrival, k) for k, q in queues.items() if q]
                        if ready:
                            _, k = min(ready)
                            batch = queues[k][: self.batch_size(queues[k][0].workload)]
                            del queues[k][: len(batch)]
                            break
                        qcv.wait()
                try:
                    res = self.solve_batch(batch, t0)
                except Exception as e:  # surfaces in the dispatcher
                    with qcv:
                        state["error"] = e
                        qcv.notify_all()
                    return
                with qcv:
                    for r in res:
                        done[r.rid] = r
                    state["pending"] -= len(res)
                    qcv.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for th in threads:
            th.start()
        for r in order:
            delay = r.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            with qcv:
                queues.setdefault(class_key(r.workload, self.precision), []).append(r)
                qcv.notify_all()
        for th in threads:
            th.join()
        if state["error"] is not None:
            raise state["error"]
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

"""Python binding of the C ABI in include/hyb.h (ctypes; argument marshalling only).

Every function of the C ABI is exposed under the same name and raises
HybError on a non-zero status.  ``HybMesh`` is a small convenience wrapper
that allocates the caller-owned device arrays with torch and passes torch's
current CUDA stream.  There is no CPU fallback: importing this module fails
loudly when libhyb.so has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_void_p, c_char_p
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhyb.so")

HYB_OK, HYB_ERR_ARG, HYB_ERR_CFL, HYB_ERR_OOM, HYB_ERR_CUDA, HYB_ERR_TIMEOUT, HYB_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
HYB_BC_NEUMANN0, HYB_BC_ABC = 0, 1
HYB_FP64, HYB_FP32 = 0, 1
HYB_WEIGHTS_PLAIN, HYB_WEIGHTS_QUADRATURE = 0, 1
HYB_FIELD_U_LAST, HYB_FIELD_U_PREV, HYB_FIELD_LAMBDA_FIRST = 0, 1, 2
HYB_WAIT_NONE = -1
HYB_ADJ_EXACT, HYB_ADJ_PAPER = 0, 1
HYB_FEM_STENCIL, HYB_FEM_TET_ALL = 0, 1
HYB_MODEL_WAVE, HYB_MODEL_TELEGRAPH = 0, 1
MAX_SOURCES = 16


class HybError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hyb status {status}: {msg}")
        self.status = status


class hyb_mesh_desc(ctypes.Structure):
    _fields_ = [("n", c_int32 * 3), ("h", c_double), ("origin", c_double * 3),
                ("fem_lo", c_int32 * 3), ("fem_hi", c_int32 * 3), ("bc", c_int32 * 6),
                ("precision", c_int32), ("ckpt_every", c_int32), ("a_max", c_double),
                ("refine_mask", c_void_p), ("wait_cycles", c_int64), ("adjoint_mode", c_int32),
                ("fem_path", c_int32), ("model", c_int32), ("spacing", c_double * 3)]


class hyb_mesh_info(ctypes.Structure):
    _fields_ = [("n_nodes", c_int64), ("n_unknown", c_int64), ("n_fem_owned", c_int64),
                ("unknown_dims", c_int32 * 3), ("obs_stride", c_int32), ("dt_max", c_double),
                ("voxel_volume", c_double), ("device_bytes", c_int64), ("launches", c_int64),
                ("n_centres", c_int64), ("n_sparse_rows", c_int64), ("n_sparse_nnz", c_int64)]


class hyb_source(ctypes.Structure):
    _fields_ = [("face", c_int32), ("omega", c_double), ("amp", c_double), ("dir", c_double * 3)]


class hyb_cg_params(ctypes.Structure):
    _fields_ = [("gamma", c_double), ("a0", c_double), ("a_min", c_double), ("a_max", c_double),
                ("weights", c_int32)]


class hyb_cg_state(ctypes.Structure):
    _fields_ = [("d", c_void_p), ("gnorm2", c_double), ("alpha", c_double), ("J", c_double), ("iter", c_int32)]


class hyb_cg_report(ctypes.Structure):
    _fields_ = [("J", c_double), ("J_data", c_double), ("gnorm", c_double), ("gpnorm", c_double),
                ("alpha", c_double), ("beta", c_double), ("dJ0", c_double), ("alpha_trial", c_double),
                ("J_trial", c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1509_01399_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "hyb_mesh_create": [POINTER(hyb_mesh_desc), P, POINTER(c_void_p)],
        "hyb_mesh_query": [P, POINTER(hyb_mesh_info)],
        "hyb_mesh_destroy": [P],
        "hyb_set_stream": [P, P],
        "hyb_forward": [P, P, POINTER(hyb_source), c_int32, c_int32, c_double, P],
        "hyb_adjoint": [P, P, c_int32],
        "hyb_set_initial": [P, P, P, P, P],
        "hyb_forward_batch": [P, P, POINTER(hyb_source), c_int32, c_int32, c_double, P],
        "hyb_gradient_batch": [P, P, c_double, c_double, P],
        "hyb_misfit_batch": [P, P, P, c_int32, POINTER(c_double), P],
        "hyb_gradient": [P, P, c_double, c_double, P],
        "hyb_misfit": [P, P, P, c_int32, POINTER(c_double), P],
        "hyb_cg_step": [P, P, P, POINTER(hyb_source), c_int32, c_int32, c_double,
                        POINTER(hyb_cg_params), POINTER(hyb_cg_state), POINTER(hyb_cg_report)],
        "hyb_get_field": [P, c_int32, c_int32, P],
        "hyb_sync": [P],
        "hyb_misfit_noalloc": [P, P, c_int32, c_int32, c_int32, c_int32, POINTER(c_int32), c_double, c_double,
                               c_int32, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hyb_last_error.argtypes = []
    lib.hyb_last_error.restype = c_char_p
    return lib


_lib = _load()
EXPORTED = ("hyb_mesh_create", "hyb_mesh_query", "hyb_mesh_destroy", "hyb_set_stream", "hyb_forward",
            "hyb_adjoint", "hyb_gradient", "hyb_misfit", "hyb_cg_step", "hyb_get_field", "hyb_sync",
            "hyb_last_error", "hyb_misfit_noalloc", "hyb_set_initial", "hyb_forward_batch",
            "hyb_gradient_batch", "hyb_misfit_batch")


def hyb_last_error() -> str:
    return _lib.hyb_last_error().decode()


def _check(st):
    if st != HYB_OK:
        raise HybError(st, hyb_last_error())


def _sources(srcs) -> tuple:
    arr = (hyb_source * len(srcs))()
    for i, s in enumerate(srcs):
        arr[i].face = int(s.face)
        arr[i].omega = float(s.omega)
        arr[i].amp = float(getattr(s, "amp", 1.0))
        d = getattr(s, "direction", None)
        for a in range(3):
            arr[i].dir[a] = 0.0 if d is None else float(d[a])
    return arr, len(srcs)


# ---- the C ABI under the same names (raw pointers as ints) ----
def hyb_mesh_create(desc: hyb_mesh_desc, stream: int = 0) -> int:
    h = c_void_p()
    _check(_lib.hyb_mesh_create(ctypes.byref(desc), c_void_p(stream), ctypes.byref(h)))
    return h.value


def hyb_mesh_query(mesh: int) -> hyb_mesh_info:
    info = hyb_mesh_info()
    _check(_lib.hyb_mesh_query(c_void_p(mesh), ctypes.byref(info)))
    return info


def hyb_mesh_destroy(mesh: int) -> None:
    _check(_lib.hyb_mesh_destroy(c_void_p(mesh)))


def hyb_set_stream(mesh: int, stream: int) -> None:
    _check(_lib.hyb_set_stream(c_void_p(mesh), c_void_p(stream)))


def hyb_forward(mesh: int, a_ptr: int, sources, nsteps: int, dt: float, trace_ptr: int) -> None:
    arr, n = _sources(sources)
    _check(_lib.hyb_forward(c_void_p(mesh), c_void_p(a_ptr), arr, n, int(nsteps), float(dt), c_void_p(trace_ptr)))


def hyb_set_initial(mesh: int, u0_ptr: int, u_prev_ptr: int, c0_ptr: int = 0, c_prev_ptr: int = 0) -> None:
    _check(_lib.hyb_set_initial(c_void_p(mesh), c_void_p(u0_ptr or None), c_void_p(u_prev_ptr or None),
                                c_void_p(c0_ptr or None), c_void_p(c_prev_ptr or None)))


def hyb_forward_batch(mesh: int, a_ptr: int, sources, nsteps: int, dt: float, trace_ptr: int) -> None:
    arr, n = _sources(sources)
    _check(_lib.hyb_forward_batch(c_void_p(mesh), c_void_p(a_ptr), arr, n, int(nsteps), float(dt),
                                  c_void_p(trace_ptr)))


def hyb_misfit_batch(mesh: int, trace_ptr: int, obs_ptr: int, weights: int, n_src: int, cot_ptr: int = 0):
    J = (c_double * n_src)()
    _check(_lib.hyb_misfit_batch(c_void_p(mesh), c_void_p(trace_ptr), c_void_p(obs_ptr), int(weights), J,
                                 c_void_p(cot_ptr) if cot_ptr else None))
    return [float(v) for v in J]


def hyb_gradient_batch(mesh: int, a_ptr: int, gamma: float, a0: float, g_ptr: int) -> None:
    _check(_lib.hyb_gradient_batch(c_void_p(mesh), c_void_p(a_ptr), float(gamma), float(a0), c_void_p(g_ptr)))


def hyb_adjoint(mesh: int, cot_ptr: int, accumulate: int = 0) -> None:
    _check(_lib.hyb_adjoint(c_void_p(mesh), c_void_p(cot_ptr), int(accumulate)))


def hyb_gradient(mesh: int, a_ptr: int, gamma: float, a0: float, g_ptr: int) -> None:
    _check(_lib.hyb_gradient(c_void_p(mesh), c_void_p(a_ptr), float(gamma), float(a0), c_void_p(g_ptr)))


def hyb_misfit(mesh: int, trace_ptr: int, obs_ptr: int, weights: int, want_value: bool = True,
               cot_ptr: int = 0) -> Optional[float]:
    J = c_double(0.0)
    _check(_lib.hyb_misfit(c_void_p(mesh), c_void_p(trace_ptr), c_void_p(obs_ptr), int(weights),
                           ctypes.byref(J) if want_value else None, c_void_p(cot_ptr) if cot_ptr else None))
    return J.value if want_value else None


def hyb_cg_step(mesh: int, a_ptr: int, obs_ptr: int, sources, nsteps: int, dt: float,
                params: hyb_cg_params, state: hyb_cg_state) -> hyb_cg_report:
    arr, n = _sources(sources)
    rep = hyb_cg_report()
    _check(_lib.hyb_cg_step(c_void_p(mesh), c_void_p(a_ptr), c_void_p(obs_ptr), arr, n, int(nsteps), float(dt),
                            ctypes.byref(params), ctypes.byref(state), ctypes.byref(rep)))
    return rep


def hyb_get_field(mesh: int, which: int, isrc: int, out_ptr: int) -> None:
    _check(_lib.hyb_get_field(c_void_p(mesh), int(which), int(isrc), c_void_p(out_ptr)))


def hyb_sync(mesh: int) -> None:
    _check(_lib.hyb_sync(c_void_p(mesh)))


def hyb_misfit_noalloc(trace_ptr: int, obs_ptr: int, precision: int, n_src: int, nsteps: int, obs_stride: int,
                       face_dims, dt: float, h: float, weights: int, J_dev_ptr: int, cot_ptr: int = 0,
                       stream: int = 0) -> None:
    """Misfit without any device allocation (see include/hyb.h); writes the
    value to the device double at J_dev_ptr."""
    dims = (c_int32 * (2 * n_src))(*[int(v) for pair in face_dims for v in pair])
    _check(_lib.hyb_misfit_noalloc(c_void_p(trace_ptr), c_void_p(obs_ptr), int(precision), int(n_src), int(nsteps),
                                   int(obs_stride), dims, float(dt), float(h), int(weights), c_void_p(J_dev_ptr),
                                   c_void_p(cot_ptr) if cot_ptr else None, c_void_p(stream)))


# ---- convenience wrapper with torch-owned device arrays ----
class HybMesh:
    """One mesh (lattice + FEM block) with torch tensors for the caller-owned
    arrays.  precision: "fp64" or "fp32" (FP32 fields, FP64 gradient/CG)."""

    def __init__(self, n, h, fem_lo=None, fem_hi=None, bc=(1,) * 6, precision="fp64", ckpt_every=0,
                 a_max=4.0, origin=(0.0, 0.0, 0.0), device="cuda", stream=None, refine=None, wait_cycles=0,
                 adjoint_mode=HYB_ADJ_EXACT, fem_path=HYB_FEM_STENCIL, model=HYB_MODEL_WAVE, spacing=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        d = hyb_mesh_desc()
        for i in range(3):
            d.n[i] = int(n[i])
            d.origin[i] = float(origin[i])
            d.fem_lo[i] = -1 if fem_lo is None else int(fem_lo[i])
            d.fem_hi[i] = -1 if fem_hi is None else int(fem_hi[i])
        d.h = float(h)
        if spacing is not None:
            for i in range(3):
                d.spacing[i] = float(spacing[i])
        for f in range(6):
            d.bc[f] = int(bc[f])
        d.precision = HYB_FP64 if precision == "fp64" else HYB_FP32
        d.ckpt_every = int(ckpt_every)
        d.a_max = float(a_max)
        d.wait_cycles = int(wait_cycles)
        d.adjoint_mode = int(adjoint_mode)
        d.fem_path = int(fem_path)
        d.model = int(model)
        self._refine = None
        if refine is not None:
            import numpy as _np
            self._refine = _np.ascontiguousarray(_np.asarray(refine).astype(_np.uint8).ravel())
            d.refine_mask = self._refine.ctypes.data
        self.desc = d
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        with torch.cuda.device(self.device):
            st = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.stream = st
            self.handle = hyb_mesh_create(d, st.cuda_stream)
        self.info = hyb_mesh_query(self.handle)
        self.n = tuple(int(v) for v in n)
        self.n_unknown = int(self.info.n_unknown)
        self.obs_stride = int(self.info.obs_stride)
        self.nsteps = None
        self.n_src = None
        self._generation = 0

    @classmethod
    def from_workload(cls, w, precision=None, ckpt_every=None, **kw):
        kw.setdefault("refine", getattr(w, "refine", None))
        kw.setdefault("spacing", getattr(w, "spacing", None))
        return cls(w.n, w.h, w.fem_lo, w.fem_hi, w.bc, precision or w.precision,
                   w.ckpt_every if ckpt_every is None else ckpt_every, w.a_max, w.origin, **kw)

    def close(self):
        if getattr(self, "handle", None):
            hyb_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self) -> hyb_mesh_info:
        return hyb_mesh_query(self.handle)

    def set_stream(self, stream):
        self.stream = stream
        hyb_set_stream(self.handle, stream.cuda_stream)

    def new_trace(self, n_src, nsteps):
        return self.torch.zeros((n_src, nsteps + 1, self.obs_stride), dtype=self.dtype, device=self.device)

    def coef(self, a):
        t = self.torch.as_tensor(a, dtype=self.torch.float64, device=self.device)
        return t.contiguous()

    def forward(self, a, sources, nsteps, dt, trace=None):
        a = self.coef(a)
        if trace is None:
            trace = self.new_trace(len(sources), nsteps)
        hyb_forward(self.handle, a.data_ptr(), sources, nsteps, dt, trace.data_ptr())
        self._generation += 1
        self._a_keep = a
        self.nsteps, self.n_src = nsteps, len(sources)
        return trace

    def set_initial(self, u0=None, u_prev=None, c0=None, c_prev=None):
        """Initial state of Model Problem 1 for the forwards that follow (None:
        the zero state of Model Problem 2).  Arrays over the lattice nodes
        (x fastest) and the centre nodes of refined voxels."""
        if u0 is None:
            hyb_set_initial(self.handle, 0, 0)
            self._init_keep = None
            return
        t = [None if v is None else self.torch.as_tensor(v, dtype=self.dtype, device=self.device).contiguous()
             for v in (u0, u_prev, c0, c_prev)]
        self._init_keep = t
        hyb_set_initial(self.handle, *[0 if v is None else v.data_ptr() for v in t])

    def adjoint(self, cot, accumulate=False):
        cot = cot.to(dtype=self.dtype, device=self.device).contiguous()
        hyb_adjoint(self.handle, cot.data_ptr(), 1 if accumulate else 0)
        self._cot_keep = cot

    def gradient(self, a, gamma=0.0, a0=1.0, out=None):
        a = self.coef(a)
        if out is None:
            out = self.torch.empty(self.n_unknown, dtype=self.torch.float64, device=self.device)
        hyb_gradient(self.handle, a.data_ptr(), gamma, a0, out.data_ptr())
        self._a_keep2 = a
        return out

    def misfit(self, trace, obs, weights=HYB_WEIGHTS_PLAIN, want_cot=False):
        obs = obs.to(dtype=self.dtype, device=self.device).contiguous()
        cot = self.torch.empty_like(trace) if want_cot else None
        J = hyb_misfit(self.handle, trace.data_ptr(), obs.data_ptr(), weights, True,
                       cot.data_ptr() if cot is not None else 0)
        return (J, cot) if want_cot else J

    def cg_step(self, a, obs, sources, nsteps, dt, state, gamma=0.01, a0=1.0, a_min=1.0, a_max=None,
                weights=HYB_WEIGHTS_QUADRATURE):
        p = hyb_cg_params(gamma, a0, a_min, self.desc.a_max if a_max is None else a_max, weights)
        return hyb_cg_step(self.handle, a.data_ptr(), obs.data_ptr(), sources, nsteps, dt, p, state)

    def new_cg_state(self):
        d = self.torch.zeros(self.n_unknown, dtype=self.torch.float64, device=self.device)
        st = hyb_cg_state(d.data_ptr(), 0.0, 0.0, 0.0, 0)
        st._d = d
        return st

    def field(self, which=HYB_FIELD_U_LAST, isrc=0):
        out = self.torch.empty(self.n[2], self.n[1], self.n[0], dtype=self.dtype, device=self.device)
        hyb_get_field(self.handle, which, isrc, out.data_ptr())
        return out

    def sync(self):
        hyb_sync(self.handle)

    def launches(self) -> int:
        return int(hyb_mesh_query(self.handle).launches)

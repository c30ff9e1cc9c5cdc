"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds workload recipes only: grid sizes, the placement of the
cubic inclusions, source parameters, seeds and the additive data noise.  It
contains none of the method's arithmetic (no stencil, no element matrix, no
time step), so both the FP64 oracle and the CUDA path can take their inputs
from here without sharing any computation.

Shapes follow the paper's numerical study (Sec. 9): a box domain, a central
finite-element block, a plane wave launched from one face with
p(t) = sin(omega t) on (0, 2 pi / omega) (Eq. (f)), small cubic scatterers in
which the coefficient a exceeds its background value 1 (Eq. (2.3)), and
additive noise on the recorded backscatter.  The paper's own scatterer
geometry lives only in a figure that is not available, so the inclusion sets
below are synthetic stand-ins.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# Face numbering used everywhere: f = 2 * axis + side, axis 0/1/2 = x/y/z,
# side 0 = the face at coordinate 0, side 1 = the face at coordinate n - 1.
FACE_XM, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP = range(6)
BC_NEUMANN0 = 0
BC_ABC = 1


@dataclass
class Source:
    """Plane-wave source.  Without a direction: a Neumann flux on one face,
    d_n u = amp * sin(omega t) for 0 < t <= 2 pi / omega, after which the face
    takes the mesh's own boundary condition (Model Problem 2 with Eq. (f)).
    With a direction d: the plane wave travelling along d, entering through
    every face whose outward normal n has d . n < 0 with the flux
    -(d . n) amp p(t - d . (x - x0)) (x0 the entry corner); `face` is then
    the observation face whose trace is recorded."""

    face: int = FACE_ZP
    omega: float = 40.0
    amp: float = 1.0
    direction: Optional[Tuple[float, float, float]] = None

    @property
    def t1(self) -> float:
        return 2.0 * math.pi / self.omega


@dataclass
class Workload:
    """One problem instance: lattice, FEM block, boundary conditions, time grid
    and the true coefficient a = 1 + sigma on the unknown voxels."""

    name: str
    n: Tuple[int, int, int]
    h: float
    origin: Tuple[float, float, float]
    fem_lo: Optional[Tuple[int, int, int]]
    fem_hi: Optional[Tuple[int, int, int]]
    bc: Tuple[int, ...]
    sources: List[Source]
    nsteps: int
    dt: float
    a_max: float
    sigma: np.ndarray  # float64, one value per unknown voxel, x fastest
    precision: str = "fp64"  # "fp64" or "fp32"
    ckpt_every: int = 0
    extra: dict = field(default_factory=dict)
    refine: Optional[np.ndarray] = None  # bool per unknown voxel: refined once
    spacing: Optional[Tuple[float, float, float]] = None  # per-axis steps dx_1, dx_2, dx_3 (None: h on every axis)

    @property
    def hv(self) -> Tuple[float, float, float]:
        """The lattice step along each axis."""
        return tuple(self.spacing) if self.spacing is not None else (self.h, self.h, self.h)

    @property
    def unknown_dims(self) -> Tuple[int, int, int]:
        return unknown_dims(self.fem_lo, self.fem_hi)

    @property
    def n_unknown(self) -> int:
        d = self.unknown_dims
        return d[0] * d[1] * d[2]

    @property
    def n_nodes(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def a_true(self) -> np.ndarray:
        return 1.0 + self.sigma


def unknown_dims(fem_lo, fem_hi) -> Tuple[int, int, int]:
    """Unknown voxels are the cells whose eight corners are all FEM-owned:
    cell indices lo+1 .. hi-2 per axis."""
    if fem_lo is None:
        return (0, 0, 0)
    return tuple(max(0, fem_hi[d] - fem_lo[d] - 2) for d in range(3))


def cube_grid(n: int):
    """Lattice of n^3 nodes on [-1, 1]^3."""
    h = 2.0 / (n - 1)
    return (n, n, n), h, (-1.0, -1.0, -1.0)


def central_half(n: int):
    lo = (n - 1) // 4
    hi = 3 * (n - 1) // 4
    return (lo, lo, lo), (hi, hi, hi)


def voxel_centres(n_cells: int, first_cell: int, h: float, origin: float) -> np.ndarray:
    return origin + h * (np.arange(first_cell, first_cell + n_cells) + 0.5)


def box_inclusion_mask(fem_lo, fem_hi, h, origin, centre, side_cells) -> np.ndarray:
    """Boolean mask over unknown voxels (shape (nz, ny, nx)) of a cube of
    side_cells voxels per axis centred at `centre` (world coordinates): a voxel
    is inside when its centre lies in [p - s h / 2, p + s h / 2) on every axis."""
    ud = unknown_dims(fem_lo, fem_hi)
    inside = []
    for d in range(3):
        c = voxel_centres(ud[d], fem_lo[d] + 1, h, origin[d])
        half = 0.5 * side_cells * h
        eps = 1e-9 * h
        inside.append((c >= centre[d] - half - eps) & (c < centre[d] + half - eps))
    return inside[2][:, None, None] & inside[1][None, :, None] & inside[0][None, None, :]


def random_box_inclusions(fem_lo, fem_hi, count, side_range, sigma_range, rng, margin=2):
    """Non-overlapping cubic inclusions on the unknown-voxel lattice: integer
    side drawn from side_range (inclusive), corner uniform with `margin` voxels
    kept free at the unknown-block boundary, sigma uniform in sigma_range."""
    ud = unknown_dims(fem_lo, fem_hi)
    sigma = np.zeros((ud[2], ud[1], ud[0]))
    taken = np.zeros_like(sigma, dtype=bool)
    placed = 0
    tries = 0
    while placed < count:
        tries += 1
        if tries > 10000:
            raise RuntimeError("could not place inclusions")
        s = int(rng.integers(side_range[0], side_range[1] + 1))
        corner = []
        ok = True
        for d in range(3):
            hi_c = ud[d] - margin - s
            if hi_c < margin:
                ok = False
                break
            corner.append(int(rng.integers(margin, hi_c + 1)))
        if not ok:
            continue
        x0, y0, z0 = corner
        # one voxel of clearance between inclusions
        sl = (slice(max(z0 - 1, 0), z0 + s + 1), slice(max(y0 - 1, 0), y0 + s + 1),
              slice(max(x0 - 1, 0), x0 + s + 1))
        if taken[sl].any():
            continue
        val = float(rng.uniform(*sigma_range))
        sigma[z0:z0 + s, y0:y0 + s, x0:x0 + s] = val
        taken[z0:z0 + s, y0:y0 + s, x0:x0 + s] = True
        placed += 1
    return sigma.ravel()


def gaussian_bumps(fem_lo, fem_hi, h, origin, count, amp_range, width_range, rng):
    """Smooth sigma made of Gaussian bumps centred in the unknown block (h:
    the lattice step, or one per axis)."""
    ud = unknown_dims(fem_lo, fem_hi)
    hs = tuple(h) if isinstance(h, (tuple, list)) else (h, h, h)
    cs = [voxel_centres(ud[d], fem_lo[d] + 1, hs[d], origin[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(cs[2], cs[1], cs[0], indexing="ij")
    sigma = np.zeros_like(X)
    for _ in range(count):
        c = [rng.uniform(cs[d][0], cs[d][-1]) for d in range(3)]
        w = rng.uniform(*width_range)
        A = rng.uniform(*amp_range)
        sigma += A * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * w * w))
    return sigma.ravel()


def add_noise_device(trace, level: float, seed: int = 1):
    """The same noise model on a torch tensor (for traces too large for the
    host): trace + level * max|trace| * xi, xi ~ N(0, 1) drawn by torch's
    generator on the trace's device, seeded with `seed`; FP64 arithmetic."""
    import torch
    gen = torch.Generator(device=trace.device)
    gen.manual_seed(int(seed))
    t = trace.to(torch.float64)
    xi = torch.randn(t.shape, generator=gen, device=t.device, dtype=torch.float64)
    return t + level * t.abs().max() * xi


def add_noise(trace: np.ndarray, level: float, seed: int = 1) -> np.ndarray:
    """u_obs = u + level * max|u| * xi with xi ~ N(0, 1) i.i.d. per entry
    (additive noise on the backscattered data, Sec. 9)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.asarray(trace, dtype=np.float64)
    return t + level * np.abs(t).max() * rng.standard_normal(t.shape)


def dilate(mask3: np.ndarray, r: int = 1) -> np.ndarray:
    """Cubic (Chebyshev) dilation of a boolean (z, y, x) voxel mask by r voxels."""
    out = mask3.copy()
    nz, ny, nx = mask3.shape
    for dz in range(-r, r + 1):
        for dy in range(-r, r + 1):
            for dx in range(-r, r + 1):
                src = mask3[max(0, -dz):nz - max(0, dz), max(0, -dy):ny - max(0, dy), max(0, -dx):nx - max(0, dx)]
                out[max(0, dz):nz - max(0, -dz), max(0, dy):ny - max(0, -dy), max(0, dx):nx - max(0, -dx)] |= src
    return out


def refine_around(sigma: np.ndarray, ud, r: int = 1) -> np.ndarray:
    """Refinement mask: the voxels with sigma > 0 dilated by r voxels."""
    m = (np.asarray(sigma).reshape(ud[2], ud[1], ud[0]) > 0)
    return dilate(m, r).ravel()


def refined_dt(h: float, a_max: float, safety: float = 0.9) -> float:
    """Time step for meshes with voxels refined once: 2 / sqrt(32 a_max / h^2)
    scaled by a safety factor (32 / h^2 bounds the rows of the once-bisected
    Kuhn voxels, 12 / h^2 those of the lattice)."""
    return safety * 2.0 * h / math.sqrt(32.0 * a_max)


def anisotropic_dt(spacing, a_max: float, safety: float = 0.9) -> float:
    """Time step for per-axis steps dx_d: tau <= 1 / sqrt(a sum_d 1 / dx_d^2)
    (the bound h / sqrt(3 a) of Eq. (CFL) when the steps are equal), scaled
    by a safety factor."""
    return safety / math.sqrt(a_max * sum(1.0 / (d * d) for d in spacing))


def structured_dt(h: float, a_max: float, safety: float = 0.9) -> float:
    """Time step from the CFL bound tau <= h / sqrt(3 a) (Eq. (CFL)) scaled by
    a safety factor."""
    return safety * h / math.sqrt(3.0 * a_max)


ALL_ABC = (BC_ABC,) * 6


def pr1_ref_33() -> Workload:
    """33^3 lattice on [-1,1]^3 (h = 1/16), FEM nodes 8..24, first-order
    absorbing faces, plane wave sin(40 t) from the top face, two 3x3x3-voxel
    inclusions sigma = 1 at x = +-0.3, dt = 0.5 h / sqrt(3), 400 steps, FP64."""
    n, h, origin = cube_grid(33)
    lo, hi = central_half(33)
    m = box_inclusion_mask(lo, hi, h, origin, (0.3, 0.0, 0.0), 3) | \
        box_inclusion_mask(lo, hi, h, origin, (-0.3, 0.0, 0.0), 3)
    sigma = np.where(m, 1.0, 0.0).ravel()
    return Workload("pr1_ref_33", n, h, origin, lo, hi, ALL_ABC, [Source(FACE_ZP, 40.0)],
                    400, 0.5 * h / math.sqrt(3.0), 4.0, sigma, "fp64")


def inverse_129(nsteps: int = 1500) -> Workload:
    """129^3 lattice (h = 1/64), FEM nodes 32..96, three random cubic
    inclusions (side 3..6 voxels, sigma ~ U[0.5, 2]), 1500 steps at the CFL
    step for a_max = 5, FP32 fields with FP64 gradient and CG reductions."""
    n, h, origin = cube_grid(129)
    lo, hi = central_half(129)
    rng = np.random.Generator(np.random.PCG64(2))
    sigma = random_box_inclusions(lo, hi, 3, (3, 6), (0.5, 2.0), rng)
    ud = unknown_dims(lo, hi)
    return Workload("inverse_129", n, h, origin, lo, hi, ALL_ABC, [Source(FACE_ZP, 40.0)],
                    nsteps, refined_dt(h, 5.0), 5.0, sigma, "fp32",
                    extra=dict(cg_iters=20, gamma=0.01, a0=1.0, noise=0.03, noise_seed=1),
                    refine=refine_around(sigma, ud, 1))


def autograd_97(nsteps: int = 1200) -> Workload:
    """97^3 lattice (h = 1/48), FEM nodes 24..72, two 9-voxel inclusions
    sigma = 1 at x = +-0.3, 1200 steps, checkpoints every 50 steps."""
    n, h, origin = cube_grid(97)
    lo, hi = central_half(97)
    m = box_inclusion_mask(lo, hi, h, origin, (0.3, 0.0, 0.0), 9) | \
        box_inclusion_mask(lo, hi, h, origin, (-0.3, 0.0, 0.0), 9)
    sigma = np.where(m, 1.0, 0.0).ravel()
    return Workload("autograd_97", n, h, origin, lo, hi, ALL_ABC, [Source(FACE_ZP, 40.0)],
                    nsteps, structured_dt(h, 4.0), 4.0, sigma, "fp64", ckpt_every=50)


def serving_request(i: int, sizes=(33, 65, 97, 129), nsteps: Optional[int] = None) -> Workload:
    """Request i of the serving stream: grid drawn from `sizes`, FEM block =
    central half, 2-4 random cubic inclusions with sigma ~ U[0.2, 2], step
    count linear in the grid size (400 at 33^3 .. 1500 at 129^3), FP32."""
    rng = np.random.Generator(np.random.PCG64(1000 + i))
    N = int(sizes[int(rng.integers(0, len(sizes)))])
    n, h, origin = cube_grid(N)
    lo, hi = central_half(N)
    count = int(rng.integers(2, 5))
    ud = unknown_dims(lo, hi)
    side_hi = max(2, int(round(0.12 * (N - 1))))
    side_lo = max(2, int(round(0.06 * (N - 1))))
    side_hi = min(side_hi, max(2, (ud[0] - 4) // 3))
    side_lo = min(side_lo, side_hi)
    sigma = random_box_inclusions(lo, hi, count, (side_lo, side_hi), (0.2, 2.0), rng)
    if nsteps is None:
        nsteps = int(round(400 + (N - 33) * (1500 - 400) / (129 - 33)))
    return Workload(f"serve_{i}", n, h, origin, lo, hi, ALL_ABC, [Source(FACE_ZP, 40.0)],
                    nsteps, structured_dt(h, 3.0), 3.0, sigma, "fp32")


def large_257(nsteps: int = 3000, n_src: int = 8, refine: bool = True) -> Workload:
    """The large batched workload on its 257^3 lattice (see `large_batched`)."""
    return large_batched(257, nsteps, n_src, refine)


def large_batched(N: int = 257, nsteps: int = 3000, n_src: int = 8, refine: bool = True) -> Workload:
    """N^3 lattice on [-1,1]^3 (257: h = 1/128), FEM nodes = central half (64..192), smooth sigma
    made of 4-8 Gaussian bumps (amplitude U[0, 1.5], width U[0.05, 0.15],
    centres in the unknown block; seed 5), voxels with sigma > 0.1 max sigma
    refined once, a_max = 2.5, 3000 steps at 0.9 of the refined mesh's
    stability bound, checkpoints every 50 steps, FP32 fields with FP64
    gradient accumulation.  Eight plane waves sin(40 t) batched as independent
    sources: from the six faces (observed on their own face) and along the two
    body diagonals +-(1, 1, 1) / sqrt(3) (entering through three faces,
    observed on the z face they enter through).  Data: the FP64 forward at
    the true coefficient plus 3 % noise; 10 CG iterations."""
    n, h, origin = cube_grid(N)
    lo, hi = central_half(N)
    rng = np.random.Generator(np.random.PCG64(5))
    sigma = gaussian_bumps(lo, hi, h, origin, int(rng.integers(4, 9)), (0.0, 1.5), (0.05, 0.15), rng)
    srcs = [Source(f, 40.0) for f in (FACE_XM, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP)]
    srcs += [Source(FACE_ZM, 40.0, 1.0, (1.0, 1.0, 1.0)), Source(FACE_ZP, 40.0, 1.0, (-1.0, -1.0, -1.0))]
    ref = (sigma > 0.1 * sigma.max()) if refine else None
    dt = refined_dt(h, 2.5) if refine else structured_dt(h, 2.5)
    return Workload("large_%d" % N, n, h, origin, lo, hi, ALL_ABC, srcs[:n_src], nsteps, dt, 2.5, sigma, "fp32",
                    ckpt_every=50, refine=ref,
                    extra=dict(cg_iters=10, gamma=0.01, a0=1.0, noise=0.03, noise_seed=1))


def anisotropic_box(nsteps: int = 600, n_src: int = 8) -> Workload:
    """257 x 193 x 321 lattice on [-1,1]^3 (steps 2/256, 2/192, 2/320: the
    7-point Laplacian with unequal steps), FEM block = the central half of
    every axis, the large workload's smooth sigma recipe (Gaussian bumps,
    seed 5) on the brick voxels, no refinement, a_max = 2.5, 0.9 of the
    stability bound 1 / sqrt(a_max sum 1 / dx^2), its eight plane-wave
    sources, checkpoints every 50 steps, FP32 fields with FP64 gradient
    accumulation."""
    n = (257, 193, 321)
    spacing = tuple(2.0 / (v - 1) for v in n)
    origin = (-1.0, -1.0, -1.0)
    lo = tuple((v - 1) // 4 for v in n)
    hi = tuple(3 * (v - 1) // 4 for v in n)
    rng = np.random.Generator(np.random.PCG64(5))
    sigma = gaussian_bumps(lo, hi, spacing, origin, int(rng.integers(4, 9)), (0.0, 1.5), (0.05, 0.15), rng)
    srcs = [Source(f, 40.0) for f in (FACE_XM, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP)]
    srcs += [Source(FACE_ZM, 40.0, 1.0, (1.0, 1.0, 1.0)), Source(FACE_ZP, 40.0, 1.0, (-1.0, -1.0, -1.0))]
    return Workload("anisotropic_box", n, spacing[0], origin, lo, hi, ALL_ABC, srcs[:n_src], nsteps,
                    anisotropic_dt(spacing, 2.5), 2.5, sigma, "fp32", ckpt_every=50, spacing=spacing,
                    extra=dict(gamma=0.01, a0=1.0, noise=0.03, noise_seed=1))


def small_problem(n=9, fem=(2, 6), nsteps=60, bc=ALL_ABC, src_face=FACE_ZP, omega=12.0,
                  sigma_seed=0, sigma_scale=1.0, a_max=4.0, courant=0.5, cubic=True,
                  name="small", refine_frac=0.0, refine_seed=5, spacing=None) -> Workload:
    """Tiny problem for unit and parity tests: n^3 (or n = (nx, ny, nz))
    lattice with spacing 1 / (n - 1) on [-1/2, 1/2]^3-ish (or the per-axis
    steps `spacing`, with the time step of `anisotropic_dt` at the given
    courant factor), FEM block nodes fem[0]..fem[1] on every axis, random
    sigma in [0, sigma_scale) on the unknown voxels."""
    if isinstance(n, int):
        n = (n, n, n)
    h = 1.0 / (max(n) - 1)
    origin = (0.0, 0.0, 0.0)
    if fem is None:
        lo = hi = None
        sigma = np.zeros(0)
    else:
        lo = tuple(fem[0] for _ in range(3)) if isinstance(fem[0], int) else tuple(fem[0])
        hi = tuple(fem[1] for _ in range(3)) if isinstance(fem[1], int) else tuple(fem[1])
        ud = unknown_dims(lo, hi)
        rng = np.random.Generator(np.random.PCG64(sigma_seed))
        sigma = sigma_scale * rng.random(ud[0] * ud[1] * ud[2])
    refine = None
    if refine_frac > 0 and sigma.size:
        rng = np.random.Generator(np.random.PCG64(refine_seed))
        refine = rng.random(sigma.size) < refine_frac
        dt = courant * 2.0 * h / math.sqrt(32.0 * a_max)
    else:
        dt = courant * h / math.sqrt(3.0 * a_max)
    if spacing is not None:
        spacing = tuple(float(v) for v in spacing)
        h = spacing[0]
        dt = anisotropic_dt(spacing, a_max, courant)
    srcs = [] if src_face is None else [Source(src_face, omega)]
    return Workload(name, n, h, origin, lo, hi, tuple(bc), srcs, nsteps, dt, a_max, sigma, "fp64",
                    refine=refine, spacing=spacing)


def model1_initial(w: Workload):
    """Initial state of Model Problem 1 (Eq. (model1)) from Eq. (initcond):
    u(x, 0) = exp(-(x1^2 + x2^2 + x3^2)) on the whole domain (the printed
    exponent x3^3 read as x3^2), u_t(x, 0) = 0, started with
    u^{-1} = u^0 - tau u_t(x, 0) = u^0.  Returns (u0, u_prev) on the lattice
    nodes (x fastest) and (c0, c_prev) on the centre nodes of refined voxels
    (in unknown-voxel order), each a float64 array."""
    nx, ny, nz = w.n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    hv = w.hv
    X = [w.origin[0] + hv[0] * x, w.origin[1] + hv[1] * y, w.origin[2] + hv[2] * z]
    u0 = np.exp(-(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)).ravel()
    c0 = np.zeros(0)
    if w.refine is not None and np.any(w.refine):
        ud = w.unknown_dims
        ids = np.flatnonzero(w.refine)
        cv = [ids % ud[0], (ids // ud[0]) % ud[1], ids // (ud[0] * ud[1])]
        C = [w.origin[d] + hv[d] * (cv[d] + w.fem_lo[d] + 1 + 0.5) for d in range(3)]
        c0 = np.exp(-(C[0] ** 2 + C[1] ** 2 + C[2] ** 2))
    return (u0, u0.copy()), (c0, c0.copy())


def random_cotangent(n_src, nsteps, n_obs, seed=7) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal((n_src, nsteps + 1, n_obs))
    c[:, 0, :] = 0.0
    return c


def waveguide(omega: float = 40.0, model: int = 2, refine: bool = False, nsteps: int = 500) -> Workload:
    """The waveguide of the paper's numerical study (Sec. 9): Omega =
    (-3.4, 3.4) x (-0.8, 0.8)^2, h = 0.1 (69 x 17 x 17 nodes), Omega_FEM =
    (-3.2, 3.2) x (-0.6, 0.6)^2 (FEM nodes 2..66 x 2..14 x 2..14), the plane
    wave p(t) = sin(omega t) of Eq. (f) launched from the front side
    x1 = -3.4 (observed there: the backscattered data), absorbing back side
    x1 = 3.4, reflecting long sides (S_3 of Eq. (model1)), tau = 0.006 and
    T = 3 (500 steps), a in [1, 5] (Eq. (admpar)).  The scatterers of the
    paper's figure are not available: six small symmetric cubes of 2 x 2 x 2
    voxels with a = 4 on the waveguide's axis at x1 = +-0.8, +-1.6, +-2.4
    stand in for them.  refine: the 1-voxel dilation of the scatterers refined
    once (the finer mesh the paper generates its data on).  model 1 adds the
    initial state of Eq. (initcond) (synth.model1_initial)."""
    n = (69, 17, 17)
    h = 0.1
    origin = (-3.4, -0.8, -0.8)
    lo, hi = (2, 2, 2), (66, 14, 14)
    sigma = np.zeros(unknown_dims(lo, hi)[::-1]).ravel()
    for x1 in (-2.4, -1.6, -0.8, 0.8, 1.6, 2.4):
        sigma = np.where(box_inclusion_mask(lo, hi, h, origin, (x1, 0.0, 0.0), 2).ravel(), 3.0, sigma)
    bc = (BC_ABC, BC_ABC, BC_NEUMANN0, BC_NEUMANN0, BC_NEUMANN0, BC_NEUMANN0)
    ud = unknown_dims(lo, hi)
    return Workload("waveguide_m%d_w%g" % (model, omega), n, h, origin, lo, hi, bc, [Source(FACE_XM, omega)],
                    nsteps, 0.006, 5.0, sigma, "fp64",
                    extra=dict(model=model, gamma=0.01, a0=1.0, a_exact=4.0, theta=1e-6),
                    refine=refine_around(sigma, ud, 1) if refine else None)


CONFIG_BUILDERS = {
    "pr1_ref_33": pr1_ref_33,
    "inverse_129": inverse_129,
    "autograd_97": autograd_97,
    "large_257": large_257,
}

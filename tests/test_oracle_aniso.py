"""Pins of the oracle on lattices with per-axis steps dx_1, dx_2, dx_3 (the
7-point Laplacian of Sec. 7.3 written for unequal steps; the FEM block made of
bricks, each cut into the six Kuhn tetrahedra).  Each pin rests on a fact fixed
by the mathematics, not on the oracle's own formulas:

* the second difference is exact on quadratics, and so is the lumped-mass
  Kuhn row on a brick lattice (it equals the per-axis 7-point stencil): the
  space operator of u = x^2 + 2 y^2 + 3 z^2 is -12 on every interior row; any
  P1 stiffness with a constant coefficient annihilates linear functions,
  refined voxels included (their centres placed at the brick centres computed
  here), and with any coefficient the constants;
* a plane wave along one axis, between reflecting side faces, is a 1-D
  problem: the 3-D traces equal a 1-D leapfrog written out in this file (the
  step, source ghost and absorbing coefficient of that axis alone);
* with reflecting faces the scheme conserves its discrete energy exactly;
* the exact adjoint's gradient equals central finite differences;
* the lumped face quadrature integrates bilinear functions exactly over the
  face's rectangle (dx_p (n_p - 1) by dx_q (n_q - 1));
* rotating the axes of the whole problem (lattice, steps, FEM block,
  coefficient, refinement, source direction) rotates its traces.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.hybrid import Problem

HV = (0.05, 0.0625, 0.08)


def _coords(n, hv, origin=(0.0, 0.0, 0.0)):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [origin[0] + hv[0] * x.ravel(), origin[1] + hv[1] * y.ravel(), origin[2] + hv[2] * z.ravel()]


@pytest.mark.parametrize("hv", [HV, (0.08, 0.05, 0.0625), (0.07, 0.07, 0.045)])
def test_space_operator_exact_on_quadratics(hv):
    n = (11, 10, 9)
    P = Problem(n, hv, (2, 2, 2), (8, 7, 6), (1,) * 6)
    L = P.space_operator(np.ones(P.n_unknown))
    x, y, z = _coords(n, hv)
    u = x * x + 2.0 * y * y + 3.0 * z * z
    Lu = L @ u
    I = P.I
    interior = np.all((I > 0) & (I < np.array(n) - 1), axis=1)
    assert interior[P.owned[: P.N]].all() and (interior & P.fdm_owned[: P.N]).sum() > 100
    np.testing.assert_allclose(Lu[interior], -12.0, rtol=1e-11)


def test_stiffness_annihilates_linear_functions_with_refinement():
    n = (12, 11, 10)
    fem_lo, fem_hi = (2, 2, 2), (9, 8, 7)
    ud = synth.unknown_dims(fem_lo, fem_hi)
    rng = np.random.default_rng(4)
    refine = rng.random(ud[0] * ud[1] * ud[2]) < 0.4
    P = Problem(n, HV, fem_lo, fem_hi, (1,) * 6, refine=refine)
    x, y, z = _coords(n, HV)
    ids = np.flatnonzero(refine)
    cv = [ids % ud[0], (ids // ud[0]) % ud[1], ids // (ud[0] * ud[1])]
    cx, cy, cz = [HV[d] * (cv[d] + fem_lo[d] + 1 + 0.5) for d in range(3)]
    lin = lambda a, b, c: 0.2 + 0.3 * a - 0.7 * b + 1.1 * c
    u = np.concatenate([lin(x, y, z), lin(cx, cy, cz)])
    K, ML = P.assemble(np.ones(P.n_unknown))
    assert P.NC == refine.sum() > 0
    assert np.abs((K @ u)[P.owned]).max() < 1e-13 * abs(K).max() * np.abs(u).max()
    # with a variable coefficient only the constants stay in the kernel
    Ka, _ = P.assemble(rng.uniform(1.0, 3.0, P.n_unknown))
    assert np.abs((Ka @ np.ones(P.NT))[P.owned]).max() < 1e-13 * abs(Ka).max()
    assert np.abs((Ka @ u)[P.owned]).max() > 1e-6 * abs(Ka).max()
    # the lumped masses add up to the block's volume
    vol = np.prod([(fem_hi[d] - fem_lo[d]) * HV[d] for d in range(3)])
    assert abs(ML.sum() - vol) < 1e-13 * vol


def _leapfrog_1d(m, h, dt, nsteps, omega, amp, far_abc):
    """The 1-D problem u_tt = u_xx on nodes 0..m-1 (step h): node 0 carries
    the flux d_n u = amp sin(omega t) while t_k <= 2 pi / omega (mirror ghost
    u_{-1} = u_1 + 2 h g) and absorbs afterwards; node m-1 absorbs (far_abc)
    or reflects.  Absorbing node b with inward neighbour b1:
    u_b^{k+1} = u_b1^k + r u_b^k - r u_b1^{k+1}, r = (h - dt) / (h + dt)."""
    c = (dt / h) ** 2
    r = (h - dt) / (h + dt)
    u_prev = np.zeros(m)
    u = np.zeros(m)
    out = [u[0]]
    t1 = 2.0 * math.pi / omega
    for k in range(nsteps):
        t = k * dt
        flux = t <= t1
        new = np.zeros(m)
        new[1:-1] = 2 * u[1:-1] - u_prev[1:-1] + c * (u[2:] - 2 * u[1:-1] + u[:-2])
        if not far_abc:
            new[-1] = 2 * u[-1] - u_prev[-1] + c * (2 * u[-2] - 2 * u[-1])
        else:
            new[-1] = u[-2] + r * u[-1] - r * new[-2]
        if flux:
            g = amp * math.sin(omega * t) if t >= 0 else 0.0
            new[0] = 2 * u[0] - u_prev[0] + c * (2 * u[1] - 2 * u[0]) + dt * dt * 2.0 / h * g
        else:
            new[0] = u[1] + r * u[0] - r * new[1]
        u_prev, u = u, new
        out.append(u[0])
    return np.array(out)


@pytest.mark.parametrize("ax", [0, 1, 2])
@pytest.mark.parametrize("far_abc", [True, False])
def test_plane_wave_along_an_axis_is_one_dimensional(ax, far_abc):
    """Source on the high face of axis `ax`, reflecting faces on the other two
    axes, a FEM block with a = 1: every node of a cross-section moves alike,
    and the trace is the 1-D leapfrog along that axis with its own step."""
    n = [7, 8, 9]
    n[ax] = 23
    bc = [0] * 6
    bc[2 * ax] = 1 if far_abc else 0
    bc[2 * ax + 1] = 1
    lo, hi = [2, 2, 2], [4, 5, 6]
    lo[ax], hi[ax] = 6, 15
    P = Problem(tuple(n), HV, tuple(lo), tuple(hi), tuple(bc))
    dt = synth.anisotropic_dt(HV, 1.0, 0.8)
    nsteps, omega = 110, 25.0
    src = synth.Source(2 * ax + 1, omega, 1.3)
    tr = P.forward(np.ones(P.n_unknown), src, nsteps, dt)["trace"]
    ref = _leapfrog_1d(n[ax], HV[ax], dt, nsteps, omega, 1.3, far_abc)
    assert np.abs(ref).max() > 1e-3
    np.testing.assert_allclose(tr, np.repeat(ref[:, None], tr.shape[1], axis=1), rtol=0, atol=1e-12 * np.abs(ref).max())


def test_energy_is_conserved_with_reflecting_faces():
    """E^{k+1/2} = |u^{k+1} - u^k|_M^2 + tau^2 (u^{k+1})^T M L u^k is constant
    (M L symmetric) for reflecting faces, no source and a random coefficient."""
    n = (12, 10, 11)
    P = Problem(n, HV, (2, 2, 2), (9, 7, 8), (0,) * 6)
    rng = np.random.default_rng(8)
    a = rng.uniform(1.0, 3.0, P.n_unknown)
    x, y, z = _coords(n, HV)
    u0 = np.exp(-((x - 0.25) ** 2 + (y - 0.3) ** 2 + (z - 0.4) ** 2) / 0.02)
    dt = synth.anisotropic_dt(HV, 3.0, 0.9)
    nsteps = 150
    res = P.forward(a, None, nsteps, dt, init=(u0, u0.copy()), keep_fields=True)
    F = res["fields"]
    L = P.space_operator(a)
    M = P.lumped_mass(a)
    ML = M[:, None] * L.toarray()
    assert np.abs(ML - ML.T).max() < 1e-12 * np.abs(ML).max()
    E = []
    for k in range(nsteps):
        d = F[k + 1] - F[k]
        E.append(float(np.dot(M * d, d) + dt * dt * F[k + 1] @ (ML @ F[k])))
    E = np.array(E)
    assert E[0] > 0 and np.abs(E - E[0]).max() < 1e-11 * E[0]
    assert np.abs(F[-1] - F[0]).max() > 0.1 * np.abs(F[0]).max()


@pytest.mark.parametrize("mode", ["plain", "quadrature"])
def test_gradient_matches_finite_differences(mode):
    w = synth.small_problem(n=(9, 10, 11), fem=(2, 6), nsteps=70, omega=14.0, courant=0.8,
                            spacing=(0.11, 0.09, 0.1))
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(9)
    a_obs = 1.0 + 2.0 * rng.random(P.n_unknown)
    a = 1.0 + 2.0 * rng.random(P.n_unknown)
    src = w.sources[0]
    obs = [P.forward(a_obs, src, w.nsteps, w.dt)["trace"]]
    J, g, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, obs, mode=mode)
    assert J > 0 and np.abs(g).max() > 0
    eps = 1e-5
    for v in range(P.n_unknown):
        e = np.zeros(P.n_unknown)
        e[v] = eps
        Jp, _, _ = oracle.value_and_grad(P, a + e, [src], w.nsteps, w.dt, obs, mode=mode, need_grad=False)
        Jm, _, _ = oracle.value_and_grad(P, a - e, [src], w.nsteps, w.dt, obs, mode=mode, need_grad=False)
        assert abs((Jp - Jm) / (2 * eps) - g[v]) <= 1e-6 * np.abs(g).max(), v


def test_face_quadrature_is_exact_on_bilinear_functions():
    n = (6, 7, 8)
    P = Problem(n, HV, None, None, (1,) * 6)
    X = _coords(n, HV)
    for f in range(6):
        ax = f // 2
        p, q = [d for d in range(3) if d != ax]
        nodes = P.face_nodes(f)
        w = P.face_weights(f)
        Lp, Lq = (n[p] - 1) * HV[p], (n[q] - 1) * HV[q]
        assert abs(w.sum() - Lp * Lq) < 1e-14 * Lp * Lq
        xp, xq = X[p][nodes], X[q][nodes]
        fv = (0.3 + 1.7 * xp) * (-0.4 + 2.2 * xq)
        exact = (0.3 * Lp + 0.85 * Lp * Lp) * (-0.4 * Lq + 1.1 * Lq * Lq)
        assert abs(np.dot(w, fv) - exact) < 1e-13 * abs(exact)


def _rotate(v):  # (x, y, z) -> (z, x, y): new axis 0 is the old axis 2
    return (v[2], v[0], v[1])


def test_rotating_the_axes_rotates_the_traces():
    """Old node (i, j, k) becomes new node (k, i, j).  An oblique wave with
    direction d enters through the three low faces and is observed on the
    low z face; after the rotation the same face is the low x face, whose
    in-face order (new y fastest = old x, new z = old y) matches the old one."""
    n = (10, 9, 11)
    lo, hi = (2, 2, 2), (7, 6, 8)
    ud = synth.unknown_dims(lo, hi)
    rng = np.random.default_rng(12)
    a = 1.0 + 1.5 * rng.random(ud[0] * ud[1] * ud[2])
    refine = rng.random(a.size) < 0.3
    d = (1.0, 2.0, 3.0)
    P = Problem(n, HV, lo, hi, (1,) * 6, refine=refine)
    Q = Problem(_rotate(n), _rotate(HV), _rotate(lo), _rotate(hi), (1,) * 6,
                refine=refine.reshape(ud[2], ud[1], ud[0]).transpose(1, 2, 0).ravel())
    a_q = a.reshape(ud[2], ud[1], ud[0]).transpose(1, 2, 0).ravel()  # [z, y, x] -> [y, x, z]
    dt = synth.anisotropic_dt(HV, 2.5, 0.5)
    nsteps = 90
    tp = P.forward(a, synth.Source(synth.FACE_ZM, 20.0, 1.0, d), nsteps, dt)["trace"]
    tq = Q.forward(a_q, synth.Source(synth.FACE_XM, 20.0, 1.0, _rotate(d)), nsteps, dt)["trace"]
    assert np.abs(tp).max() > 1e-3
    np.testing.assert_allclose(tq, tp, rtol=0, atol=1e-12 * np.abs(tp).max())


def test_equal_steps_are_the_isotropic_problem_bitwise():
    w = synth.small_problem(n=(9, 10, 11), fem=(2, 6), nsteps=50, omega=14.0)
    P = oracle.problem_from_workload(w)
    Q = Problem(w.n, (w.h, w.h, w.h), w.fem_lo, w.fem_hi, w.bc, w.origin)
    assert Q.iso and Q.h == P.h
    a = w.a_true()
    np.testing.assert_array_equal(P.forward(a, w.sources[0], w.nsteps, w.dt)["trace"],
                                  Q.forward(a, w.sources[0], w.nsteps, w.dt)["trace"])

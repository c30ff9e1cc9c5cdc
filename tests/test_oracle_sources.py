"""Pins of the oracle's plane-wave sources against closed forms.

A source without a direction is the face source of Model Problem 2
(d_n u = p(t) on one face, Eq. (model2), Eq. (f)).  A source with a
direction d launches the plane wave u = F(t - d . (x - x0)) with F' = p: on a
face with outward normal n its normal derivative is -(d . n) p, so the entry
faces (d . n < 0) carry that Neumann flux, the side faces (d . n = 0) are
reflecting, and until the wave reaches an exit face the discrete solution
must converge to the closed form at second order.
"""
import math

import numpy as np
import pytest

import synth
from oracle.hybrid import Problem


def _F(s, omega):
    """F(s) = int_0^s p = (1 - cos(omega s)) / omega on [0, 2 pi / omega], 0 elsewhere."""
    s = np.asarray(s, dtype=float)
    return np.where((s >= 0) & (s <= 2 * np.pi / omega), (1 - np.cos(omega * s)) / omega, 0.0)


def _oblique_error(n_in, n_flat, d, obs_face, omega=5.0, L=3.0, T=1.9):
    """Errors against F(t - d.(x - x0)): max over the recorded trace, RMS over
    the final field (and the RMS of the exact field), on a box of n_in nodes
    along the axes where d has a component and n_flat nodes along the others
    (reflecting there)."""
    d = np.asarray(d, dtype=float)
    d = d / np.linalg.norm(d)
    n = tuple(n_in if abs(d[ax]) > 0 else n_flat for ax in range(3))
    h = L / (n_in - 1)
    dt = 0.5 * h / math.sqrt(3.0)
    nsteps = int(round(T / dt))
    # reflecting side faces, absorbing exit faces, the entry faces carry the flux
    bc = []
    for f in range(6):
        ax, side = divmod(f, 2)
        bc.append(0 if d[ax] == 0 else 1)
    P = Problem(n, h, None, None, tuple(bc), (0.0, 0.0, 0.0))
    src = synth.Source(obs_face, omega, 1.0, tuple(d))
    res = P.forward(np.zeros(0), src, nsteps, dt)
    x0 = np.array([0 if d[ax] >= 0 else n[ax] - 1 for ax in range(3)], dtype=float)
    delay = h * ((P.I - x0) @ d)
    t = dt * np.arange(nsteps + 1)
    obs = P.face_nodes(obs_face)
    exact_trace = _F(t[:, None] - delay[obs][None, :], omega)
    e_trace = np.abs(res["trace"] - exact_trace).max()
    exact = _F(t[-1] - delay, omega)
    e_field = np.sqrt(np.mean((res["u"][: P.N] - exact) ** 2))
    return e_trace, e_field, np.sqrt(np.mean(exact ** 2))


def test_oblique_plane_wave_2d_second_order():
    """d = (1, 0, 1) / sqrt(2) on a slab one cell thick in y: entry through the
    x-low and z-low faces with the factor 1 / sqrt(2).  Halving h and tau
    together divides the trace error (max norm) and the field error (RMS) by
    about 4.  (F has a jump in F'' at the front and tail of the pulse, which
    costs the field's max norm its second order; the RMS keeps it.)"""
    d = (1.0, 0.0, 1.0)
    r = [_oblique_error(n, 3, d, synth.FACE_ZM) for n in (31, 61, 121)]
    (t1, f1, amp), (t2, f2, _), (t3, f3, _) = r
    assert f3 < 0.005 * amp
    assert 3.5 < t1 / t2 < 4.5 and 3.5 < t2 / t3 < 4.5, r
    assert 3.0 < f1 / f2 < 5.0 and 3.0 < f2 / f3 < 5.0, r


def test_oblique_plane_wave_3d_diagonal():
    """d = -(1, 1, 1) / sqrt(3): entry through the three high faces (corner
    x0 = (n-1, n-1, n-1)), observed on z-high; the errors fall by about 4
    from 21^3 to 41^3."""
    d = (-1.0, -1.0, -1.0)
    t1, f1, amp = _oblique_error(21, 21, d, synth.FACE_ZP, T=1.6)
    t2, f2, _ = _oblique_error(41, 41, d, synth.FACE_ZP, T=1.6)
    assert f2 < 0.01 * amp
    assert 3.0 < t1 / t2 < 5.0, (t1, t2)
    assert 3.0 < f1 / f2 < 5.0, (f1, f2)


def test_oblique_flux_sign_and_factor_would_fail():
    """The same run with the flux factor -(d . n) replaced by 1 (the face
    source's factor) is an O(1) miss: the closed-form check above is
    sensitive to it."""
    d = np.array([1.0, 0.0, 1.0]) / math.sqrt(2.0)
    n_in, L, omega = 61, 3.0, 5.0
    h = L / (n_in - 1)
    dt = 0.5 * h / math.sqrt(3.0)
    nsteps = int(round(1.9 / dt))
    P = Problem((n_in, 3, n_in), h, None, None, (1, 1, 0, 0, 1, 1), (0.0, 0.0, 0.0))
    good = P.forward(np.zeros(0), synth.Source(synth.FACE_ZM, omega, 1.0, tuple(d)), nsteps, dt)["u"]
    # a unit factor on the two entry faces is the same run with amp = sqrt(2)
    bad = P.forward(np.zeros(0), synth.Source(synth.FACE_ZM, omega, math.sqrt(2.0), tuple(d)), nsteps, dt)["u"]
    delay = h * (P.I @ d)
    exact = _F(nsteps * dt - delay, omega)
    assert np.abs(good[: P.N] - exact).max() < 0.05 * exact.max()
    assert np.abs(bad[: P.N] - exact).max() > 0.2 * exact.max()


def test_face_source_is_the_normal_incidence_case():
    """A face source equals the plane wave along d = -n of its face: same
    trace and field, and the face switches to its own condition at t1."""
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=70, omega=12.0, courant=0.8)
    P = Problem(w.n, w.h, w.fem_lo, w.fem_hi, w.bc, w.origin)
    a = w.a_true()
    r1 = P.forward(a, synth.Source(synth.FACE_ZP, 12.0), w.nsteps, w.dt)
    r2 = P.forward(a, synth.Source(synth.FACE_ZP, 12.0, 1.0, (0.0, 0.0, -1.0)), w.nsteps, w.dt)
    np.testing.assert_array_equal(r1["trace"], r2["trace"])
    np.testing.assert_array_equal(r1["u"], r2["u"])
    t1 = 2 * math.pi / 12.0
    assert P.switch_time(synth.Source(synth.FACE_ZP, 12.0), synth.FACE_ZP) == t1
    k_on = int(math.floor(t1 / w.dt))
    assert P.phase(synth.Source(synth.FACE_ZP, 12.0), k_on, w.dt).src_faces == (synth.FACE_ZP,)
    assert P.phase(synth.Source(synth.FACE_ZP, 12.0), k_on + 1, w.dt).src_faces == ()


def test_diagonal_switch_times_follow_the_wave():
    """Each entry face keeps its flux until the pulse has crossed its farthest
    node: t1 + h sum over the in-face axes of |d_b| (n_b - 1)."""
    P = Problem((9, 11, 13), 0.1, None, None, (1,) * 6)
    src = synth.Source(synth.FACE_ZM, 10.0, 1.0, (1.0, 1.0, 1.0))
    d, i0, entry = P.plane_wave(src)
    assert i0 == [0, 0, 0] and sorted(entry) == [0, 2, 4]
    for f in entry:
        assert entry[f] == pytest.approx(1 / math.sqrt(3))
    t1 = 2 * math.pi / 10.0
    s = 1 / math.sqrt(3)
    assert P.switch_time(src, 0) == pytest.approx(t1 + 0.1 * s * (10 + 12))
    assert P.switch_time(src, 2) == pytest.approx(t1 + 0.1 * s * (8 + 12))
    assert P.switch_time(src, 4) == pytest.approx(t1 + 0.1 * s * (8 + 10))

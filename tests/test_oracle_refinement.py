"""Pins of the oracle on locally refined meshes (voxels refined once by
bisection of their Kuhn tetrahedra along the voxel diagonal)."""
import math

import numpy as np
import pytest
import scipy.sparse as sps

import oracle
import synth
from oracle.hybrid import Problem, kuhn_tets, p1_element, element_stiffness, refine_voxels


def _refined_voxel(h):
    """The 12 children of one refined voxel: corner ids 0..7 (a + 2b + 4c),
    centre id 8."""
    tets = kuhn_tets(np.zeros((1, 3), dtype=np.int64))[0]
    corner = tets[..., 0] + 2 * tets[..., 1] + 4 * tets[..., 2]
    nodes, unk, _ = refine_voxels(corner, np.zeros(6, dtype=np.int64), np.array([True]), 8)
    X = np.zeros((9, 3))
    for c in range(8):
        X[c] = h * np.array([c & 1, (c >> 1) & 1, c >> 2])
    X[8] = h * 0.5
    vol, grads = p1_element(X[nodes])
    return nodes, vol, grads, X


@pytest.mark.parametrize("h", [1.0, 0.3])
def test_refined_voxel_masses_by_hand(h):
    """Bisecting the diagonal halves each Kuhn tetrahedron (volume h^3/6)
    into two children of volume h^3/12.  Lumped mass |K|/4 per vertex: the
    centre is in all 12 children (h^3/4), the two diagonal corners in 6
    (h^3/8), the other corners in 4 (h^3/12)."""
    nodes, vol, grads, X = _refined_voxel(h)
    np.testing.assert_allclose(vol, h ** 3 / 12.0, rtol=1e-12)
    M = np.bincount(nodes.ravel(), weights=np.repeat(vol / 4.0, 4), minlength=9)
    expect = np.array([1 / 8, 1 / 12, 1 / 12, 1 / 12, 1 / 12, 1 / 12, 1 / 12, 1 / 8, 1 / 4]) * h ** 3
    np.testing.assert_allclose(M, expect, rtol=1e-12)
    assert abs(M.sum() - h ** 3) < 1e-12 * h ** 3


def test_refined_voxel_stiffness_invariants():
    """The assembled 9 x 9 stiffness of a refined voxel is symmetric, kills
    constants, has a one-dimensional kernel and integrates the energy of a
    linear function exactly: u^T K u = |voxel| |g|^2."""
    h = 0.7
    nodes, vol, grads, X = _refined_voxel(h)
    Kl = element_stiffness(vol, grads, np.ones(12))
    K = np.zeros((9, 9))
    for t in range(12):
        for i in range(4):
            for j in range(4):
                K[nodes[t, i], nodes[t, j]] += Kl[t, i, j]
    np.testing.assert_allclose(K, K.T, atol=1e-14)
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-13)
    ev = np.linalg.eigvalsh(K)
    assert abs(ev[0]) < 1e-12 and ev[1] > 1e-3
    g = np.array([0.3, -1.1, 0.7])
    u = X @ g
    assert abs(u @ K @ u - h ** 3 * g @ g) < 1e-12


def _mass(P, a):
    """Lumped mass of every row: the assembled M^L on FEM-owned rows, the
    lattice node volume (h^3 halved per boundary axis) elsewhere."""
    _, ML = P.assemble(a)
    m = np.zeros(P.NT)
    nat = np.full(P.N, P.h ** 3)
    for d in range(3):
        b = (P.I[:, d] == 0) | (P.I[:, d] == P.n[d] - 1)
        nat[b] *= 0.5
    m[: P.N] = nat
    m[P.owned] = ML[P.owned]
    return m


def test_refined_energy_conservation():
    w = synth.small_problem(n=11, fem=(2, 8), nsteps=250, bc=(0,) * 6, omega=15.0, sigma_scale=2.0,
                            sigma_seed=9, refine_frac=0.5, courant=0.9)
    P = oracle.problem_from_workload(w)
    assert P.NC > 10
    a = w.a_true()
    L = P.space_operator(a)
    M = _mass(P, a)
    Km = (sps.diags(M) @ L).tocsr()
    assert abs(Km - Km.T).max() < 1e-12 * abs(Km).max()
    res = P.forward(a, w.sources[0], w.nsteps, w.dt, keep_fields=True)
    F = res["fields"]
    k0 = int(math.ceil(w.sources[0].t1 / w.dt)) + 2
    E = []
    for k in range(k0, w.nsteps):
        v = (F[k + 1] - F[k]) / w.dt
        E.append(0.5 * np.dot(M * v, v) + 0.5 * F[k + 1] @ (Km @ F[k]))
    E = np.array(E)
    assert E[0] > 0 and np.abs(E - E[0]).max() < 1e-11 * E[0]


def test_refined_adjoint_dot_product():
    w = synth.small_problem(n=(8, 9, 10), fem=(2, 6), nsteps=40, omega=20.0, refine_frac=0.6, courant=0.8)
    P = oracle.problem_from_workload(w)
    assert P.NC > 0
    a = w.a_true()
    src = w.sources[0]
    rng = np.random.default_rng(12)
    f = rng.standard_normal((w.nsteps, P.NT))
    t0, _ = P.forward_matrix(a, src, w.nsteps, w.dt)
    tf, _ = P.forward_matrix(a, src, w.nsteps, w.dt, forcing=f)
    c = rng.standard_normal(tf.shape)
    c[0] = 0
    _, lams = P.adjoint(a, src, w.nsteps, w.dt, c, np.zeros((w.nsteps, P.owned_nodes.size)), keep_lambdas=True)
    lhs = np.sum((tf - t0) * c)
    rhs = sum(np.dot(f[k], lams[k + 1]) for k in range(w.nsteps))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_refined_gradient_matches_central_differences():
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=80, omega=12.0, sigma_seed=1, refine_frac=0.5,
                            courant=0.8)
    P = oracle.problem_from_workload(w)
    assert P.NC > 0
    src = w.sources[0]
    a = w.a_true()
    a_obs = 1.0 + 1.5 * np.random.default_rng(2).random(P.n_unknown)
    obs = P.forward(a_obs, src, w.nsteps, w.dt)["trace"]
    J, g, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs])
    eps = 1e-6
    fd = np.zeros(P.n_unknown)
    for c in range(P.n_unknown):
        e = np.zeros(P.n_unknown)
        e[c] = eps
        Jp, _, _ = oracle.value_and_grad(P, a + e, [src], w.nsteps, w.dt, [obs], need_grad=False)
        Jm, _, _ = oracle.value_and_grad(P, a - e, [src], w.nsteps, w.dt, [obs], need_grad=False)
        fd[c] = (Jp - Jm) / (2 * eps)
    assert np.linalg.norm(g - fd) < 1e-6 * np.linalg.norm(fd)


def test_refined_hybrid_equals_all_fem():
    n = 13
    w = synth.small_problem(n=n, fem=(3, 9), nsteps=100, omega=10.0, sigma_seed=4, refine_frac=0.5)
    P = oracle.problem_from_workload(w)
    ref_small = w.refine.reshape(P.unknown_dims[::-1])
    big = np.zeros((n - 3, n - 3, n - 3), dtype=bool)
    big[3:7, 3:7, 3:7] = ref_small
    Q = Problem(w.n, w.h, (0, 0, 0), (n - 1, n - 1, n - 1), w.bc, w.origin, refine=big.ravel())
    aQ = np.ones(Q.n_unknown).reshape(Q.unknown_dims[::-1])
    aQ[3:7, 3:7, 3:7] = w.a_true().reshape(P.unknown_dims[::-1])
    r1 = P.forward(w.a_true(), w.sources[0], w.nsteps, w.dt)
    r2 = Q.forward(aQ.ravel(), w.sources[0], w.nsteps, w.dt)
    assert np.linalg.norm(r1["trace"] - r2["trace"]) < 1e-12 * np.linalg.norm(r2["trace"])

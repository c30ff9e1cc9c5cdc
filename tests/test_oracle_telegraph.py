"""Pins of the oracle's telegraph reading u_tt + sigma u_t - div grad u = 0
(damping on the unknown voxels, a = 1): it reduces to the wave scheme at
sigma = 0, its damping term removes exactly the discrete energy the scheme
says it does, and its adjoint gradient matches central finite differences."""
import numpy as np

import oracle
import synth
from oracle import hybrid as O


def _problem(n=11, fem=(3, 7), bc=(1,) * 6, nsteps=80, omega=14.0, courant=0.8):
    return synth.small_problem(n=n, fem=fem, nsteps=nsteps, bc=bc, omega=omega, courant=courant)


def test_zero_damping_is_the_wave_scheme_bitwise():
    w = _problem()
    P = oracle.problem_from_workload(w)
    ones = np.ones(P.n_unknown)
    t0 = P.forward(ones, w.sources[0], w.nsteps, w.dt)["trace"]
    t1 = O.telegraph_forward(P, np.zeros(P.n_unknown), w.sources[0], w.nsteps, w.dt)["trace"]
    np.testing.assert_array_equal(t0, t1)


def test_damping_weights_are_the_lumped_voxel_masses():
    """A voxel gives each corner h^3 / 4 on its diagonal and h^3 / 12
    elsewhere (the Kuhn lumping), so a uniform sigma gives every node
    surrounded by eight unknown voxels D = sigma h^3."""
    w = _problem(n=11, fem=(2, 8))
    P = oracle.problem_from_workload(w)
    W = O.damping_weights(P).toarray()
    h3 = P.h ** 3
    row = W[0][W[0] > 0]
    assert sorted(np.round(row / h3 * 12).astype(int).tolist()) == [1, 1, 1, 1, 1, 1, 3, 3]
    D = W.T @ np.full(P.n_unknown, 2.0)
    inner = [i for i in range(P.N) if (W[:, i] > 0).sum() == 8]
    assert inner and np.allclose(D[inner], 2.0 * h3, rtol=1e-14)


def test_discrete_energy_balance():
    """Reflecting faces, the Gaussian initial state of Model Problem 1, no
    source: with E^{k+1/2} = |u^{k+1} - u^k|_M^2 + tau^2 (u^{k+1})^T M L u^k,
    E^{k+1/2} - E^{k-1/2} = -sum_i M_i s_i (u^{k+1}_i - u^{k-1}_i)^2 exactly
    (multiply the damped row by M (u^{k+1} - u^{k-1})); the energy decays."""
    w = _problem(n=11, fem=(2, 8), bc=(0,) * 6, nsteps=200)
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(3)
    sigma = 3.0 * rng.random(P.n_unknown)
    (u0, up), _ = synth.model1_initial(w)
    s = O.damping_ratio(P, sigma, w.dt)
    res = P.forward(np.ones(P.n_unknown), None, w.nsteps, w.dt, init=(u0, up), keep_fields=True, damp=s)
    F = res["fields"]
    L = P.space_operator(np.ones(P.n_unknown))
    M = P.lumped_mass(np.ones(P.n_unknown))
    ML = (M[:, None] * L.toarray())
    assert np.abs(ML - ML.T).max() < 1e-12 * np.abs(ML).max()
    tau2 = w.dt * w.dt

    def energy(k):  # E^{k+1/2}
        d = F[k + 1] - F[k]
        return float(np.dot(M * d, d) + tau2 * F[k + 1] @ (ML @ F[k]))

    E = np.array([energy(k) for k in range(w.nsteps)])
    for k in range(1, w.nsteps):
        d2 = F[k + 1] - F[k - 1]
        loss = float(np.sum(M * s * d2 * d2))
        assert abs((E[k] - E[k - 1]) + loss) <= 1e-11 * E[0]
    assert E[-1] < 0.9 * E[0]


def test_sigma_gradient_matches_finite_differences():
    """Absorbing faces, a face source, random sigma: dJ/dsigma of the exact
    adjoint against central differences on every unknown voxel."""
    w = _problem(n=9, fem=(2, 6), nsteps=70)
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(5)
    sig_obs = 2.0 * rng.random(P.n_unknown)
    sigma = 2.0 * rng.random(P.n_unknown)
    src = w.sources[0]
    obs = O.telegraph_forward(P, sig_obs, src, w.nsteps, w.dt)["trace"]
    J, g, _ = O.telegraph_value_and_grad(P, sigma, [src], w.nsteps, w.dt, [obs])
    assert J > 0 and np.abs(g).max() > 0
    eps = 1e-5
    for v in range(P.n_unknown):
        e = np.zeros(P.n_unknown)
        e[v] = eps
        Jp, _, _ = O.telegraph_value_and_grad(P, sigma + e, [src], w.nsteps, w.dt, [obs])
        Jm, _, _ = O.telegraph_value_and_grad(P, sigma - e, [src], w.nsteps, w.dt, [obs])
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - g[v]) <= 1e-6 * np.abs(g).max(), (v, fd, g[v])


def test_sigma_gradient_quadrature_weights_and_oblique_source():
    """The same finite-difference check with the quadrature weights of
    Eq. (functional) and a diagonal plane wave."""
    w = _problem(n=9, fem=(2, 6), nsteps=60)
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(6)
    src = synth.Source(synth.FACE_ZM, 14.0, 1.0, (1.0, 1.0, 1.0))
    sigma = 1.5 * rng.random(P.n_unknown)
    obs = O.telegraph_forward(P, 1.5 * rng.random(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    J, g, _ = O.telegraph_value_and_grad(P, sigma, [src], w.nsteps, w.dt, [obs], mode="quadrature")
    eps = 1e-5
    for v in (0, 3, P.n_unknown - 1):
        e = np.zeros(P.n_unknown)
        e[v] = eps
        Jp, _, _ = O.telegraph_value_and_grad(P, sigma + e, [src], w.nsteps, w.dt, [obs], mode="quadrature")
        Jm, _, _ = O.telegraph_value_and_grad(P, sigma - e, [src], w.nsteps, w.dt, [obs], mode="quadrature")
        assert abs((Jp - Jm) / (2 * eps) - g[v]) <= 1e-6 * np.abs(g).max()

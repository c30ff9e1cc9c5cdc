"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a textbook
element matrix, a hand-derived closed form, an exact identity of the scheme,
a closed-form solution of the continuous problem or an exact adjoint
relation.  None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.hybrid import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_kuhn_golden():
    rows = []
    for line in open(os.path.join(GOLDEN, "kuhn_voxel.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([float(v) for v in line.split()])
    return np.array(rows[:8]), np.array(rows[8])


# --------------------------------------------------------------- elements
def test_reference_tetrahedron_textbook_matrices():
    """Unit right tetrahedron: phi_0 = 1 - x - y - z, phi_i = x_i, so
    K = (1/6) [[3,-1,-1,-1],[-1,1,0,0],[-1,0,1,0],[-1,0,0,1]] and |K| = 1/6
    (Sec. 7.2 element stiffness for a = 1)."""
    X = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=float)
    vol, g = oracle.p1_element(X)
    K = oracle.element_stiffness(vol, g, np.ones(1))[0]
    ref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert abs(vol[0] - 1.0 / 6.0) < 1e-15
    np.testing.assert_allclose(K, ref, atol=1e-15)


def test_p1_stiffness_invariants_random_tets():
    """For any tetrahedron: constants are in the kernel of K^K and a linear
    function u = g.x has energy u^T K^K u = a |K| |g|^2; the lumped masses sum
    to |K|."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((50, 4, 3))
    vol, grads = oracle.p1_element(X)
    a = rng.uniform(0.5, 3.0, 50)
    K = oracle.element_stiffness(vol, grads, a)
    np.testing.assert_allclose(K.sum(axis=2), 0.0, atol=1e-10 * np.abs(K).max())
    gvec = rng.standard_normal((50, 3))
    u = np.einsum("tvd,td->tv", X, gvec)
    e = np.einsum("ti,tij,tj->t", u, K, u)
    np.testing.assert_allclose(e, a * vol * np.sum(gvec ** 2, axis=1), rtol=1e-9)
    ref_vol = np.abs(np.einsum("tij,tij->t", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])[:, None, :],
                               (X[:, 3] - X[:, 0])[:, None, :])) / 6.0
    np.testing.assert_allclose(vol, ref_vol, rtol=1e-12)


@pytest.mark.parametrize("h", [1.0, 0.25])
def test_kuhn_voxel_closed_form(h):
    """The six Kuhn tetrahedra of one voxel assemble to the hand-derived
    matrices of tests/golden/kuhn_voxel.txt: only the 12 axis edges couple
    (h/3 at the edges touching the diagonal corners, h/6 elsewhere) and the
    lumped masses are h^3/4 and h^3/12."""
    Kref6, Mref12 = _load_kuhn_golden()
    tets = oracle.kuhn_tets(np.zeros((1, 3), dtype=np.int64))[0]  # (6,4,3)
    vol, grads = oracle.p1_element(h * tets.astype(float))
    Kloc = oracle.element_stiffness(vol, grads, np.ones(6))
    corner = tets[..., 0] + 2 * tets[..., 1] + 4 * tets[..., 2]
    K = np.zeros((8, 8))
    M = np.zeros(8)
    for t in range(6):
        for i in range(4):
            M[corner[t, i]] += vol[t] / 4.0
            for j in range(4):
                K[corner[t, i], corner[t, j]] += Kloc[t, i, j]
    np.testing.assert_allclose(6.0 * K / h, Kref6, atol=1e-12)
    np.testing.assert_allclose(12.0 * M / h ** 3, Mref12, atol=1e-12)


def test_fem_rows_coincide_with_7point_fdm():
    """With a = 1 the lumped-mass Kuhn FEM row at every FEM-owned node equals
    the FDM row -Delta_h (the structured overlap where the two schemes
    coincide, Sec. 1 and Sec. 7)."""
    P = Problem((11, 10, 12), 0.1, (2, 2, 3), (8, 7, 9))
    L = P.space_operator(np.ones(P.n_unknown))
    own = P.owned_nodes
    diff = (L[own] + P.D[own]).toarray()
    assert np.abs(diff).max() < 1e-9 * (1.0 / P.h ** 2)


def test_fem_variable_coefficient_row_from_voxel_weights():
    """With a per-voxel a, the FEM row at an interior node is the 7-point
    stencil whose axis-edge weight is sum over the four voxels around the edge
    of a_c times 1/3 (edge touching the voxel's diagonal corners) or 1/6."""
    P = Problem((9, 9, 9), 1.0, (1, 1, 1), (7, 7, 7))
    rng = np.random.default_rng(5)
    a = rng.uniform(1.0, 3.0, P.n_unknown)
    L = P.space_operator(a)
    ud = P.unknown_dims

    def av(c):
        c = np.array(c)
        if np.all(c >= 2) and np.all(c <= 5):
            r = c - 2
            return a[r[0] + ud[0] * (r[1] + ud[1] * r[2])]
        return 1.0

    node = np.array([4, 3, 5])
    nid = P.node_id(node)
    for ax in range(3):
        p, q = [d for d in range(3) if d != ax]
        for s in (+1, -1):
            base = node.copy() if s > 0 else node - np.eye(3, dtype=int)[ax]
            w = 0.0
            for bp in (0, 1):
                for bq in (0, 1):
                    c = base.copy()
                    c[p] -= bp
                    c[q] -= bq
                    w += av(c) * (1.0 / 3.0 if bp == bq else 1.0 / 6.0)
            nb = P.node_id(node + s * np.eye(3, dtype=int)[ax])
            assert abs(L[nid, nb] + w) < 1e-12


# --------------------------------------------------------- schemes coincide
def test_algorithm2_equals_matrix_form():
    w = synth.small_problem(n=11, fem=(3, 7), nsteps=80, omega=10.0)
    P = oracle.problem_from_workload(w)
    a = w.a_true()
    res = P.forward(a, w.sources[0], w.nsteps, w.dt)
    tr, u = P.forward_matrix(a, w.sources[0], w.nsteps, w.dt)
    scale = np.abs(res["trace"]).max()
    assert scale > 0
    assert np.abs(tr - res["trace"]).max() < 1e-12 * scale
    assert np.abs(u - res["u"]).max() < 1e-12 * np.abs(u).max()


def test_hybrid_equals_pure_fdm_when_a_is_one():
    w = synth.small_problem(n=13, fem=(3, 9), nsteps=120, omega=10.0)
    P = oracle.problem_from_workload(w)
    Q = Problem(w.n, w.h, None, None, w.bc, w.origin)
    r1 = P.forward(np.ones(P.n_unknown), w.sources[0], w.nsteps, w.dt)
    r2 = Q.forward(np.zeros(0), w.sources[0], w.nsteps, w.dt)
    s = np.linalg.norm(r2["trace"])
    assert np.linalg.norm(r1["trace"] - r2["trace"]) < 1e-13 * s
    assert np.linalg.norm(r1["u"] - r2["u"]) < 1e-13 * np.linalg.norm(r2["u"])


def test_hybrid_equals_all_fem():
    """A small FEM block inside FDM (with the Algorithm 1 exchange) equals a
    FEM block covering every interior node, with the same coefficient."""
    n = 13
    w = synth.small_problem(n=n, fem=(3, 9), nsteps=120, omega=10.0, sigma_seed=4)
    P = oracle.problem_from_workload(w)
    Q = Problem(w.n, w.h, (0, 0, 0), (n - 1, n - 1, n - 1), w.bc, w.origin)
    aP = w.a_true()
    aQ = np.ones(Q.n_unknown).reshape(Q.unknown_dims[::-1])
    aQ[3:7, 3:7, 3:7] = aP.reshape(P.unknown_dims[::-1])  # unknown voxels 4..7 vs 1..10
    r1 = P.forward(aP, w.sources[0], w.nsteps, w.dt)
    r2 = Q.forward(aQ.ravel(), w.sources[0], w.nsteps, w.dt)
    assert np.linalg.norm(r1["trace"] - r2["trace"]) < 1e-12 * np.linalg.norm(r2["trace"])
    assert np.linalg.norm(r1["u"] - r2["u"]) < 1e-12 * np.linalg.norm(r2["u"])


# ---------------------------------------------------------------- energy
def _natural_mass(P):
    """Lumped mass of the lattice node volume: h^3 halved for every axis on
    which the node sits on the outer boundary."""
    m = np.full(P.N, P.h ** 3)
    for d in range(3):
        b = (P.I[:, d] == 0) | (P.I[:, d] == P.n[d] - 1)
        m[b] *= 0.5
    return m


def test_energy_conserved_with_reflecting_faces():
    """Leapfrog with a symmetric mass-weighted operator conserves
    E^{k+1/2} = 1/2 |(u^{k+1}-u^k)/tau|_M^2 + 1/2 (u^{k+1})^T K u^k exactly
    (discrete form of the energy identity in the proof of the Theorem,
    Sec. 4, with the boundary term absent for d_n u = 0).  Checked for a
    non-constant a, after the source flux has switched off."""
    w = synth.small_problem(n=11, fem=(2, 8), nsteps=300, bc=(0,) * 6, omega=15.0,
                            sigma_scale=2.0, sigma_seed=9)
    P = oracle.problem_from_workload(w)
    a = w.a_true()
    L = P.space_operator(a)
    M = _natural_mass(P)
    Km = (P.D.multiply(0) + __import__("scipy.sparse").sparse.diags(M) @ L).tocsr()
    asym = abs(Km - Km.T).max()
    assert asym < 1e-12 * abs(Km).max(), "mass-weighted operator must be symmetric"
    res = P.forward(a, w.sources[0], w.nsteps, w.dt, keep_fields=True)
    F = res["fields"]
    t1 = w.sources[0].t1
    k0 = int(math.ceil(t1 / w.dt)) + 2
    E = []
    for k in range(k0, w.nsteps):
        v = (F[k + 1] - F[k]) / w.dt
        E.append(0.5 * np.dot(M * v, v) + 0.5 * F[k + 1] @ (Km @ F[k]))
    E = np.array(E)
    assert E[0] > 0
    assert np.abs(E - E[0]).max() < 1e-11 * E[0]


def test_energy_decays_with_absorbing_faces():
    w = synth.small_problem(n=11, fem=(2, 8), nsteps=400, bc=(1,) * 6, omega=15.0,
                            sigma_scale=1.0, sigma_seed=2)
    P = oracle.problem_from_workload(w)
    a = w.a_true()
    import scipy.sparse as sps
    Km = (sps.diags(_natural_mass(P)) @ P.space_operator(a)).tocsr()
    M = _natural_mass(P)
    res = P.forward(a, w.sources[0], w.nsteps, w.dt, keep_fields=True)
    F = res["fields"]
    k0 = int(math.ceil(w.sources[0].t1 / w.dt)) + 2

    def energy(k):
        v = (F[k + 1] - F[k]) / w.dt
        return 0.5 * np.dot(M * v, v) + 0.5 * F[k + 1] @ (Km @ F[k])

    e0, e1 = energy(k0), energy(w.nsteps - 1)
    assert e1 < 0.5 * e0


# ------------------------------------------------------------- plane wave
def _plane_wave_error(nz, omega=5.0, Lz=3.0, T=6.5):
    """Max error on the top-face trace and on the centre column at the end
    against u(z, t) = F(t - (Lz - z)), F(s) = (1 - cos(omega s)) / omega on
    [0, 2 pi / omega], 0 elsewhere: the exact solution of u_tt = u_zz with
    d_n u = sin(omega t) on the top face for t < 2 pi / omega (Eq. (model2),
    Eq. (f)) and a reflection-free bottom (Eq. (absbc))."""
    h = Lz / (nz - 1)
    dt = 0.5 * h / math.sqrt(3.0)
    nsteps = int(round(T / dt))
    bc = (0, 0, 0, 0, 1, 1)
    P = Problem((3, 3, nz), h, None, None, bc, (0.0, 0.0, 0.0))
    src = synth.Source(synth.FACE_ZP, omega)
    res = P.forward(np.zeros(0), src, nsteps, dt)
    t = dt * np.arange(nsteps + 1)

    def F(s):
        s = np.asarray(s, dtype=float)
        return np.where((s >= 0) & (s <= 2 * np.pi / omega), (1 - np.cos(omega * s)) / omega, 0.0)

    e_trace = np.abs(res["trace"][:, 4] - F(t)).max()
    z = h * np.arange(nz)
    col = res["u"].reshape(nz, 3, 3)[:, 1, 1]
    e_col = np.abs(col - F(t[-1] - (Lz - z))).max()
    return max(e_trace, e_col), F(t).max()


def test_plane_wave_closed_form_second_order():
    e1, amp = _plane_wave_error(31)
    e2, _ = _plane_wave_error(61)
    e3, _ = _plane_wave_error(121)
    assert e3 < 0.02 * amp
    r1, r2 = e1 / e2, e2 / e3
    assert 3.0 < r2 < 5.5, (e1, e2, e3)
    assert 2.5 < r1 < 6.0, (e1, e2, e3)


def test_plane_wave_sign_errors_would_fail():
    """The closed-form comparison above is sensitive to the absorbing
    condition: a reflecting bottom (Neumann) sends the pulse back to the top
    face, an O(1) error in the trace."""
    nz = 61
    h = 3.0 / (nz - 1)
    dt = 0.5 * h / math.sqrt(3.0)
    nsteps = int(round(6.5 / dt))
    P = Problem((3, 3, nz), h, None, None, (0, 0, 0, 0, 0, 1), (0.0, 0.0, 0.0))
    res = P.forward(np.zeros(0), synth.Source(synth.FACE_ZP, 5.0), nsteps, dt)
    late = res["trace"][int(6.2 / dt):, 4]
    assert np.abs(late).max() > 0.1


# ---------------------------------------------------------------- adjoint
def test_adjoint_dot_product():
    """<T f, c> = sum_k <f^k, lambda^{k+1}> for the linear map T from a forcing
    of every step to the trace, lambda solving the transposed recursion
    (the discrete counterpart of the Lagrangian identity, Eq. (lagrangian1))."""
    w = synth.small_problem(n=(7, 8, 9), fem=(2, 5), nsteps=40, omega=20.0, courant=0.9)
    P = oracle.problem_from_workload(w)
    a = w.a_true()
    src = w.sources[0]
    rng = np.random.default_rng(11)
    f = rng.standard_normal((w.nsteps, P.N))
    t0, _ = P.forward_matrix(a, src, w.nsteps, w.dt)
    tf, _ = P.forward_matrix(a, src, w.nsteps, w.dt, forcing=f)
    Tf = tf - t0
    c = rng.standard_normal(Tf.shape)
    c[0] = 0
    hist = np.zeros((w.nsteps, P.owned_nodes.size))
    _, lams = P.adjoint(a, src, w.nsteps, w.dt, c, hist, keep_lambdas=True)
    lhs = np.sum(Tf * c)
    rhs = sum(np.dot(f[k], lams[k + 1]) for k in range(w.nsteps))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1e-300) * 10


@pytest.mark.parametrize("bc", [(1,) * 6, (0, 1, 1, 0, 1, 1)])
def test_gradient_matches_central_differences(bc):
    """dJ/da from the adjoint equals (J(a + eps e_c) - J(a - eps e_c)) / (2 eps)
    on every unknown voxel of a small problem (Eq. (grad1new))."""
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=90, omega=12.0, bc=bc, sigma_seed=1,
                            courant=0.8)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a = w.a_true()
    a_obs = 1.0 + 1.5 * np.random.default_rng(2).random(P.n_unknown)
    obs = P.forward(a_obs, src, w.nsteps, w.dt)["trace"]
    J, g, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], gamma=0.0)
    eps = 1e-6
    fd = np.zeros(P.n_unknown)
    for c in range(P.n_unknown):
        e = np.zeros(P.n_unknown)
        e[c] = eps
        Jp, _, _ = oracle.value_and_grad(P, a + e, [src], w.nsteps, w.dt, [obs], need_grad=False)
        Jm, _, _ = oracle.value_and_grad(P, a - e, [src], w.nsteps, w.dt, [obs], need_grad=False)
        fd[c] = (Jp - Jm) / (2 * eps)
    assert np.linalg.norm(g - fd) < 1e-6 * np.linalg.norm(fd)


def test_gradient_tikhonov_and_quadrature_weights():
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=60, omega=12.0, sigma_seed=3, courant=0.8)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a = w.a_true()
    obs = P.forward(np.ones(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    gamma = 0.3
    J, g, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], gamma=gamma, a0=1.0,
                                    mode="quadrature")
    eps = 1e-6
    for c in (0, 3, 7):
        e = np.zeros(P.n_unknown)
        e[c] = eps
        Jp, _, _ = oracle.value_and_grad(P, a + e, [src], w.nsteps, w.dt, [obs], gamma, 1.0,
                                         "quadrature", need_grad=False)
        Jm, _, _ = oracle.value_and_grad(P, a - e, [src], w.nsteps, w.dt, [obs], gamma, 1.0,
                                         "quadrature", need_grad=False)
        assert abs((Jp - Jm) / (2 * eps) - g[c]) < 1e-6 * np.abs(g).max()


# --------------------------------------------------------------------- CG
def test_cg_direction_by_hand():
    """Algorithm 3, Step 2 on two voxels of volume 2: d^0 = -g^0, then
    beta = ||g^1||^2 / ||g^0||^2 with ||g||^2 = sum |c| g_c^2."""
    g0 = np.array([1.0, -2.0])
    d0, b0, n0 = oracle.cg_direction(g0, None, None, 2.0)
    assert b0 == 0.0 and n0 == 10.0
    np.testing.assert_array_equal(d0, [-1.0, 2.0])
    g1 = np.array([0.5, 0.5])
    d1, b1, n1 = oracle.cg_direction(g1, d0, n0, 2.0)
    assert n1 == 1.0 and b1 == 0.1
    np.testing.assert_allclose(d1, [-0.5 - 0.1, -0.5 + 0.2])


def test_quadratic_step_recovers_parabola_minimum():
    # J(alpha) = 3 - 4 alpha + 5 alpha^2: minimum at 0.4
    J = lambda x: 3 - 4 * x + 5 * x * x
    assert abs(oracle.quadratic_step(J(0), -4.0, 0.3, J(0.3)) - 0.4) < 1e-14
    # clamp to 4 alpha_t
    assert oracle.quadratic_step(J(0), -4.0, 0.05, J(0.05)) == pytest.approx(0.2)
    # concave: keep the trial step
    assert oracle.quadratic_step(0.0, -1.0, 0.3, -1.0) == 0.3


def test_cg_step_decreases_functional_and_projects():
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=80, omega=12.0, sigma_seed=5, courant=0.8)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a_true = 1.0 + 2.0 * np.random.default_rng(8).random(P.n_unknown)
    obs = P.forward(a_true, src, w.nsteps, w.dt)["trace"]
    a = np.ones(P.n_unknown)
    state = {}
    Js = []
    for _ in range(3):
        a, state, rep = oracle.cg_step(P, a, [src], w.nsteps, w.dt, [obs], state, gamma=0.0,
                                       a_min=1.0, a_max=4.0)
        Js.append(rep["J"])
        assert a.min() >= 1.0 and a.max() <= 4.0
    J_end, _, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], 0.0, 1.0, "quadrature",
                                        need_grad=False)
    assert J_end < Js[0]


# ------------------------------------------------- quadrature of the functional
@pytest.mark.parametrize("n", [(9, 7, 5), (4, 11, 6)])
def test_face_weights_are_the_trapezoid_rule(n):
    """The lumped face weights m_j of the misfit int_{S_T} (u - u~)^2 dS dt
    (Eq. (functional)) are the tensor trapezoid rule on each face: they sum to
    the face area (n_p - 1)(n_q - 1) h^2 and integrate every bilinear function
    of the two in-face coordinates exactly.  (Not halving on the border, or
    halving a corner only once, changes the sum.)"""
    h = 0.3
    P = Problem(n, h, None, None, (1,) * 6)
    rng = np.random.default_rng(2)
    for f in range(6):
        ax = f // 2
        p, q = [d for d in range(3) if d != ax]
        w = P.face_weights(f)
        nodes = P.face_nodes(f)
        Lp, Lq = (n[p] - 1) * h, (n[q] - 1) * h
        assert abs(w.sum() - Lp * Lq) < 1e-13 * Lp * Lq
        x = h * P.I[nodes, p]
        y = h * P.I[nodes, q]
        c = rng.standard_normal(4)
        f_val = c[0] + c[1] * x + c[2] * y + c[3] * x * y
        exact = c[0] * Lp * Lq + c[1] * Lp ** 2 / 2 * Lq + c[2] * Lp * Lq ** 2 / 2 + c[3] * Lp ** 2 * Lq ** 2 / 4
        assert abs(np.dot(w, f_val) - exact) < 1e-12 * (abs(exact) + Lp * Lq)
        # corners carry a quarter, edge nodes a half, interior nodes the full h^2
        on_p = (P.I[nodes, p] == 0) | (P.I[nodes, p] == n[p] - 1)
        on_q = (P.I[nodes, q] == 0) | (P.I[nodes, q] == n[q] - 1)
        np.testing.assert_allclose(w[on_p & on_q], h * h / 4)
        np.testing.assert_allclose(w[on_p ^ on_q], h * h / 2)
        np.testing.assert_allclose(w[~on_p & ~on_q], h * h)


def test_time_weights_are_the_right_rectangle_rule():
    """With quadrature weights the time integral of the misfit is the right
    rectangle rule tau sum_{k=1}^{N} g(t_k): exact for constants (= T) and,
    for g(t) = t, exactly T^2 / 2 + T tau / 2 (the rule's closed-form error)."""
    P = Problem((5, 5, 5), 0.25, None, None, (1,) * 6)
    N, dt = 37, 0.0123
    T = N * dt
    wk, mj = oracle.data_weights(P, synth.FACE_ZP, N, dt, "quadrature")
    t = dt * np.arange(N + 1)
    assert wk[0] == 0.0
    assert abs(np.dot(wk, np.ones(N + 1)) - T) < 1e-14
    assert abs(np.dot(wk, t) - (T * T / 2 + T * dt / 2)) < 1e-14
    # plain weights: the unweighted sum over k >= 1 and every face node
    wp, mp = oracle.data_weights(P, synth.FACE_ZP, N, dt, "plain")
    assert wp.sum() == N and np.all(mp == 1.0)


def test_misfit_of_a_constant_residual_is_half_c2_T_area():
    """J = 1/2 int_{S_T} (u - u~)^2 dS dt for u - u~ = c on every face node and
    every step: 1/2 c^2 T |face| with the quadrature weights."""
    P = Problem((6, 7, 8), 0.2, None, None, (1,) * 6)
    N, dt, c = 25, 0.03, 0.7
    for f in range(6):
        wk, mj = oracle.data_weights(P, f, N, dt, "quadrature")
        obs = np.zeros((N + 1, mj.size))
        J, cot = oracle.misfit(obs + c, obs, wk, mj)
        ax = f // 2
        area = np.prod([(P.n[d] - 1) * P.h for d in range(3) if d != ax])
        assert abs(J - 0.5 * c * c * N * dt * area) < 1e-13 * J
        np.testing.assert_allclose(cot[1:], c * dt * mj[None, :].repeat(N, 0))
        assert np.all(cot[0] == 0.0)


def test_projected_direction_by_hand():
    """Three voxels, a_min = 1, a_max = 4: voxel 0 at the lower bound with
    g > 0 (blocked: its gradient component is dropped), voxel 1 at the lower
    bound with g < 0 (free: it moves up), voxel 2 at the upper bound with
    g > 0 (free: it moves down).  A previous direction that pushes voxel 0
    further down is dropped there too."""
    a = np.array([1.0, 1.0, 4.0])
    g = np.array([2.0, -1.0, 3.0])
    gp = oracle.projected_gradient(a, g, 1.0, 4.0)
    np.testing.assert_array_equal(gp, [0.0, -1.0, 3.0])
    d, beta, gn2 = oracle.cg_direction(gp, np.array([-1.0, 1.0, 1.0]), 5.0, 2.0)
    assert gn2 == 2.0 * (1.0 + 9.0) and beta == 4.0
    np.testing.assert_array_equal(d, [-4.0, 5.0, 1.0])
    np.testing.assert_array_equal(oracle.drop_blocked(a, d, 1.0, 4.0), [0.0, 5.0, 0.0])


def test_projected_cg_descends_from_the_lower_bound():
    """Started at a = a_min with data from a coefficient that is below the
    background on part of the block (its gradient pushes those voxels out of
    the admissible set), the projected iteration lowers F at every step; the
    slope <g, d> it fits the parabola to is the slope of the projected path."""
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=80, omega=12.0, sigma_seed=5, courant=0.8)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    rng = np.random.default_rng(8)
    a_true = 1.0 + 2.0 * rng.random(P.n_unknown) * (rng.random(P.n_unknown) < 0.5)
    a_true[rng.random(P.n_unknown) < 0.3] = 0.6  # below a_min: unreachable
    obs = P.forward(a_true, src, w.nsteps, w.dt)["trace"]
    a = np.ones(P.n_unknown)
    state = {}
    Js = []
    for _ in range(4):
        a_prev = a
        a, state, rep = oracle.cg_step(P, a, [src], w.nsteps, w.dt, [obs], state, gamma=0.0, a_min=1.0,
                                       a_max=4.0)
        Js.append(rep["J"])
        # the directional derivative along the projected path equals <g, d>
        eps = 1e-7 * rep["alpha_trial"]
        Jp, _, _ = oracle.value_and_grad(P, np.clip(a_prev + eps * state["d"], 1.0, 4.0), [src], w.nsteps, w.dt,
                                         [obs], 0.0, 1.0, "quadrature", need_grad=False)
        assert abs((Jp - rep["J"]) / eps - rep["dJ0"]) < 1e-4 * abs(rep["dJ0"])
    J_end, _, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], 0.0, 1.0, "quadrature",
                                        need_grad=False)
    Js.append(J_end)
    assert all(Js[i + 1] < Js[i] for i in range(len(Js) - 1)), Js


# ------------------------------------------------------------ paper-mode adjoint
@pytest.mark.parametrize("refine", [0.0, 0.4])
@pytest.mark.parametrize("mode", ["plain", "quadrature"])
def test_paper_adjoint_equals_exact_with_reflecting_faces(refine, mode):
    """With reflecting faces everywhere (no absorbing rows, so the forward's
    boundary never switches), the paper's adjoint (Eq. (fdmschemeadjoint) with
    d_n lambda = 0, residual as the flux on S_T, same-index pairing of
    Eq. (gradient1)) is the exact discrete adjoint written in the variable
    lambda = -tau M^{-1} mu: the two gradients agree to rounding."""
    w = synth.small_problem(n=10, fem=(2, 7), nsteps=70, omega=12.0, courant=0.8, bc=(0,) * 6,
                            refine_frac=refine, sigma_seed=3)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a = w.a_true()
    obs = P.forward(np.ones(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    J, g_exact, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], mode=mode)
    J2, g_paper, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], mode=mode, adjoint="paper")
    assert J == J2
    assert np.linalg.norm(g_paper - g_exact) < 1e-11 * np.linalg.norm(g_exact)


def test_paper_adjoint_with_absorbing_faces_differs_but_agrees_in_direction():
    """With absorbing faces the paper's adjoint keeps d_n lambda = 0 where the
    forward absorbs (the absorbing terms of Eq. (lagrangian1) are dropped), so
    its gradient is no longer the exact one: it differs by far more than
    rounding, yet points the same way."""
    w = synth.small_problem(n=10, fem=(2, 7), nsteps=90, omega=12.0, courant=0.8, sigma_seed=3)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a = w.a_true()
    obs = P.forward(np.ones(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    _, ge, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], mode="quadrature")
    _, gp, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], mode="quadrature", adjoint="paper")
    rel = np.linalg.norm(gp - ge) / np.linalg.norm(ge)
    cos = float(np.dot(gp, ge) / (np.linalg.norm(gp) * np.linalg.norm(ge)))
    assert rel > 1e-6 and cos > 0.5, (rel, cos)


# ----------------------------------------------------- Model Problem 1 (IP1)
def _ip1_init(w):
    (u0, um), (c0, cm) = synth.model1_initial(w)
    return np.concatenate([u0, c0]), np.concatenate([um, cm])


def test_model1_initial_state_of_initcond():
    """Eq. (initcond) on the lattice: u^0 = exp(-|x|^2) at every node (1 at the
    origin), u^{-1} = u^0 (zero initial velocity); centre nodes of refined
    voxels take the same function at the voxel centre."""
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=10, refine_frac=0.5)
    w.origin = (-0.5, -0.5, -0.5)
    (u0, um), (c0, cm) = synth.model1_initial(w)
    assert u0.size == 9 ** 3 and np.array_equal(u0, um) and c0.size == int(w.refine.sum())
    assert u0[4 + 9 * (4 + 9 * 4)] == 1.0  # node (4, 4, 4) sits at the origin
    assert abs(u0[0] - math.exp(-0.75)) < 1e-15
    ud = w.unknown_dims
    first = int(np.flatnonzero(w.refine)[0])
    cx, cy, cz = first % ud[0], (first // ud[0]) % ud[1], first // (ud[0] * ud[1])
    xc = [-0.5 + w.h * (c + 2 + 1 + 0.5) for c in (cx, cy, cz)]
    assert abs(c0[0] - math.exp(-sum(v * v for v in xc))) < 1e-15


@pytest.mark.parametrize("refine", [0.0, 0.4])
def test_model1_energy_conserved_from_nonzero_data(refine):
    """Model Problem 1 with a Gaussian initial state, no source and reflecting
    faces: the discrete energy is constant from the first step (the energy
    identity of Sec. 4 with nonzero initial data), for a non-constant a."""
    w = synth.small_problem(n=11, fem=(2, 8), nsteps=200, bc=(0,) * 6, sigma_scale=2.0, sigma_seed=9,
                            refine_frac=refine, courant=0.8)
    w.origin = (-0.5, -0.5, -0.5)
    P = oracle.problem_from_workload(w)
    a = w.a_true()
    init = _ip1_init(w)
    src = synth.Source(synth.FACE_ZP, 12.0, 0.0)  # amplitude 0: no flux
    res = P.forward(a, src, w.nsteps, w.dt, init=init, keep_fields=True)
    F = res["fields"]
    M = P.lumped_mass(a)
    import scipy.sparse as sps
    Km = (sps.diags(M) @ P.space_operator(a)).tocsr()
    assert abs(Km - Km.T).max() < 1e-12 * abs(Km).max()
    E = []
    for k in range(0, w.nsteps):
        v = (F[k + 1] - F[k]) / w.dt
        E.append(0.5 * np.dot(M * v, v) + 0.5 * F[k + 1] @ (Km @ F[k]))
    E = np.array(E)
    assert E[0] > 0 and np.abs(E - E[0]).max() < 1e-11 * E[0]


def test_model1_gradient_matches_central_differences():
    """Model Problem 1 (nonzero u^0): dJ/da from the adjoint, whose pairing
    now has a k = 0 term, equals central differences of J on every voxel
    (dropping that term fails this check)."""
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=60, omega=12.0, sigma_seed=1, courant=0.8)
    w.origin = (-0.5, -0.5, -0.5)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    init = _ip1_init(w)
    a = w.a_true()
    obs = P.forward(1.0 + 1.5 * np.random.default_rng(2).random(P.n_unknown), src, w.nsteps, w.dt,
                    init=init)["trace"]
    J, g, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], init=init)
    eps = 1e-6
    fd = np.zeros(P.n_unknown)
    for c in range(P.n_unknown):
        e = np.zeros(P.n_unknown)
        e[c] = eps
        Jp, _, _ = oracle.value_and_grad(P, a + e, [src], w.nsteps, w.dt, [obs], need_grad=False, init=init)
        Jm, _, _ = oracle.value_and_grad(P, a - e, [src], w.nsteps, w.dt, [obs], need_grad=False, init=init)
        fd[c] = (Jp - Jm) / (2 * eps)
    assert np.linalg.norm(g - fd) < 1e-6 * np.linalg.norm(fd)
    # the k = 0 pairing term is not negligible here
    res = P.forward(a, src, w.nsteps, w.dt, keep_hist=True, init=init)
    wk, mj = oracle.data_weights(P, src.face, w.nsteps, w.dt)
    _, cot = oracle.misfit(res["trace"], obs, wk, mj)
    _, lam1 = P.adjoint(a, src, w.nsteps, w.dt, cot, res["hist"], return_lambda=True)
    _, ML = P.assemble(a)
    k0 = -w.dt ** 2 * P.pair(res["hist"][0], lam1, ML)
    assert np.linalg.norm(k0) > 1e-3 * np.linalg.norm(fd)

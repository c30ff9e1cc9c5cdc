"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 fields and gradients within 1e-12 relative L2 of the
oracle; FP32 fields within 1e-4 relative L2 on the recorded trace and FP32
gradients (FP64 accumulation) within 1e-3.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_TRACE = 1e-4
TOL32_GRAD = 1e-3


@pytest.fixture(scope="module")
def H():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01399_gb300 import hyb
    return hyb


def run_gpu(H, w, a, a_obs, precision="fp64", ckpt=None, srcs=None, paper=False):
    import torch
    srcs = srcs or w.sources
    m = H.HybMesh.from_workload(w, precision=precision, ckpt_every=ckpt,
                                adjoint_mode=H.HYB_ADJ_PAPER if paper else H.HYB_ADJ_EXACT)
    obs = m.forward(a_obs, srcs, w.nsteps, w.dt)
    tr = m.forward(a, srcs, w.nsteps, w.dt)
    u_last = [m.field(H.HYB_FIELD_U_LAST, s).cpu().numpy().ravel() for s in range(len(srcs))]
    J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_PLAIN, want_cot=True)
    m.adjoint(cot)
    g = m.gradient(a, 0.0, 1.0)
    lam1 = [m.field(H.HYB_FIELD_LAMBDA_FIRST, s).cpu().numpy().ravel() for s in range(len(srcs))]
    m.sync()
    out = dict(trace=tr.double().cpu().numpy(), J=J, g=g.cpu().numpy(), u=u_last, lam1=lam1,
               launches=m.launches())
    m.close()
    return out


def run_oracle(w, a, a_obs, srcs=None, paper=False):
    srcs = srcs or w.sources
    P = oracle.problem_from_workload(w)
    res = dict(trace=[], J=0.0, g=np.zeros(P.n_unknown), u=[], lam1=[], kappa=[])
    for src in srcs:
        ro = P.forward(a, src, w.nsteps, w.dt, keep_hist=True)
        oo = P.forward(a_obs, src, w.nsteps, w.dt)["trace"]
        c = ro["trace"] - oo
        res["kappa"].append(float(np.linalg.norm(ro["trace"]) / max(np.linalg.norm(c), 1e-300)))
        res["J"] += 0.5 * float(np.sum(c[1:] ** 2))
        res["trace"].append(ro["trace"])
        res["u"].append(ro["u"][: P.N])  # lattice nodes (centre nodes of refined voxels follow)
        if paper:  # lambda^0 of the paper's scheme, unscaled
            gi, lam0 = P.adjoint_paper(a, src, w.nsteps, w.dt, c, ro["hist"], return_lambda=True)
            res["g"] += gi
            res["lam1"].append(lam0[: P.N])
            continue
        if P.n_unknown:
            gi, lam1 = P.adjoint(a, src, w.nsteps, w.dt, c, ro["hist"], return_lambda=True)
            res["g"] += gi
        else:
            _, lam1 = P.adjoint(a, src, w.nsteps, w.dt, c, np.zeros((w.nsteps, 0)), return_lambda=True)
        # the library keeps lambda scaled by h^3 / M^L on FEM-owned rows (it
        # differs from lambda only at corners of refined voxels)
        _, ML = P.assemble(a)
        scale = np.ones(P.NT)
        scale[P.owned] = P.h ** 3 / ML[P.owned]
        res["lam1"].append((lam1 * scale)[: P.N])
    return res


def compare(gpu, ora, tol_trace, tol_grad, tol_field=None):
    """Trace, final field and gradient within the tolerances; lambda^1 within
    tol_field times kappa = |trace| / |residual|: the adjoint's input is the
    residual trace - u_obs, a difference that each side forms from its own
    traces, so their agreement to ~1e-16 relative becomes ~1e-16 kappa
    relative on the residual that lambda carries."""
    tol_field = tol_trace if tol_field is None else tol_field
    for s, t in enumerate(ora["trace"]):
        e = rel_l2(gpu["trace"][s, :, : t.shape[1]], t)
        assert e <= tol_trace, f"trace src {s}: {e}"
        assert rel_l2(gpu["u"][s], ora["u"][s]) <= tol_field
        kappa = max(1.0, ora.get("kappa", [1.0] * len(ora["trace"]))[s])
        e = rel_l2(gpu["lam1"][s], ora["lam1"][s])
        assert e <= tol_field * kappa, f"lambda src {s}: {e} (kappa {kappa:.3g})"
    if ora["J"] > 0:
        assert abs(gpu["J"] - ora["J"]) <= 10 * tol_trace * ora["J"]
    if ora["g"].size:
        e = rel_l2(gpu["g"], ora["g"])
        assert e <= tol_grad, f"gradient: {e}"


CASES = {
    "abc_9": lambda: synth.small_problem(n=9, fem=(2, 6), nsteps=60, omega=12.0, courant=0.8),
    "mixed_bc_ragged": lambda: synth.small_problem(n=(9, 10, 11), fem=(2, 6), nsteps=70, omega=12.0,
                                                   bc=(0, 1, 1, 0, 1, 1), courant=0.8),
    "neumann_all": lambda: synth.small_problem(n=10, fem=(3, 7), nsteps=80, omega=12.0, bc=(0,) * 6,
                                               courant=0.9),
    "no_fem": lambda: synth.small_problem(n=8, fem=None, nsteps=50, omega=12.0),
    "all_fem": lambda: synth.small_problem(n=9, fem=(0, 8), nsteps=50, omega=12.0, courant=0.8),
    "thin_fem": lambda: synth.small_problem(n=12, fem=(4, 6), nsteps=40, omega=12.0),
    "wide_tiles": lambda: synth.small_problem(n=(37, 21, 19), fem=((5, 4, 4), (30, 16, 15)), nsteps=45,
                                              omega=15.0, courant=0.9, sigma_scale=2.0),
    "refined": lambda: synth.small_problem(n=11, fem=(2, 8), nsteps=60, omega=12.0, courant=0.8,
                                           refine_frac=0.4),
    # a tile row off both y faces
    "tall_tiles": lambda: synth.small_problem(n=(37, 38, 12), fem=((5, 5, 3), (30, 30, 8)), nsteps=45, omega=15.0,
                                              courant=0.9, bc=(1, 1, 0, 1, 1, 1), src_face=synth.FACE_ZP),
    # tiles with a single x face (x extent > one tile): mirror face carrying the source, absorbing opposite
    "wide_x_mirror_src_low": lambda: synth.small_problem(n=(41, 12, 11), fem=((3, 3, 3), (14, 8, 7)), nsteps=80,
                                                         omega=14.0, courant=0.8, bc=(0, 1, 1, 0, 1, 1),
                                                         src_face=synth.FACE_XM),
    "wide_x_mirror_src_high": lambda: synth.small_problem(n=(43, 11, 12), fem=((28, 3, 4), (38, 7, 8)), nsteps=80,
                                                          omega=14.0, courant=0.8, bc=(1, 0, 0, 1, 0, 1),
                                                          src_face=synth.FACE_XP),
    "refined_neumann_ragged": lambda: synth.small_problem(n=(12, 11, 13), fem=((2, 2, 2), (9, 8, 10)), nsteps=60,
                                                          omega=12.0, courant=0.8, refine_frac=0.5,
                                                          bc=(0, 1, 0, 1, 1, 1)),
}


def _oblique(w, srcs):
    w.sources = srcs
    return w


# oblique plane waves (entering through two or three faces, per-node delay)
OBLIQUE = {
    "diag_abc": lambda: _oblique(synth.small_problem(n=11, fem=(3, 7), nsteps=70, omega=15.0, courant=0.8),
                                 [synth.Source(synth.FACE_ZM, 15.0, 1.0, (1.0, 1.0, 1.0))]),
    "diag_neg_mixed_bc": lambda: _oblique(
        synth.small_problem(n=(12, 10, 11), fem=(2, 7), nsteps=80, omega=15.0, courant=0.8, bc=(0, 1, 1, 0, 1, 1)),
        [synth.Source(synth.FACE_ZP, 15.0, 1.0, (-1.0, -1.0, -1.0))]),
    "two_axis_oblique_refined": lambda: _oblique(
        synth.small_problem(n=12, fem=(2, 9), nsteps=70, omega=14.0, courant=0.8, refine_frac=0.4),
        [synth.Source(synth.FACE_XM, 14.0, 0.7, (1.0, 0.0, 0.5))]),
    # tiles wider than one tile in x: the x face column runs on the producer warp's lanes
    "diag_wide_x": lambda: _oblique(
        synth.small_problem(n=(41, 12, 11), fem=((3, 3, 3), (14, 8, 7)), nsteps=80, omega=14.0, courant=0.8,
                            bc=(0, 1, 1, 0, 1, 1)),
        [synth.Source(synth.FACE_XM, 14.0, 1.0, (1.0, 0.3, -0.6))]),
}


PAPER_CASES = {
    "abc": lambda: synth.small_problem(n=11, fem=(3, 7), nsteps=70, omega=12.0, courant=0.8),
    "mixed_bc_refined": lambda: synth.small_problem(n=(12, 11, 13), fem=((2, 2, 2), (9, 8, 10)), nsteps=60,
                                                    omega=12.0, courant=0.8, refine_frac=0.5, bc=(0, 1, 0, 1, 1, 1)),
    "wide_tiles": lambda: synth.small_problem(n=(37, 21, 19), fem=((5, 4, 4), (30, 16, 15)), nsteps=45,
                                              omega=15.0, courant=0.9, sigma_scale=2.0),
    "wide_x_src": lambda: synth.small_problem(n=(41, 12, 11), fem=((3, 3, 3), (14, 8, 7)), nsteps=80, omega=14.0,
                                              courant=0.8, bc=(0, 1, 1, 0, 1, 1), src_face=synth.FACE_XM),
}


@pytest.mark.parametrize("name", sorted(PAPER_CASES))
def test_fp64_parity_paper_adjoint(H, name):
    """The paper's adjoint scheme (HYB_ADJ_PAPER): lambda^0 and the
    same-index gradient against the oracle's Algorithm-2 implementation."""
    w = PAPER_CASES[name]()
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + 2.0 * np.random.default_rng(9).random(P.n_unknown)
    a = w.a_true()
    compare(run_gpu(H, w, a, a_obs, paper=True), run_oracle(w, a, a_obs, paper=True), TOL64, TOL64)


def test_paper_adjoint_batched_and_checkpointed(H):
    """Paper mode with three sources in one launch (one oblique) and
    checkpoint/recompute: bitwise equal to stored history, and the oracle's."""
    w = synth.small_problem(n=12, fem=(2, 9), nsteps=63, omega=12.0, courant=0.8, refine_frac=0.3)
    srcs = [synth.Source(5, 12.0), synth.Source(0, 9.0), synth.Source(synth.FACE_ZM, 14.0, 1.0, (1.0, 1.0, 1.0))]
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + np.random.default_rng(2).random(P.n_unknown)
    a = w.a_true()
    full = run_gpu(H, w, a, a_obs, srcs=srcs, paper=True, ckpt=0)
    ck = run_gpu(H, w, a, a_obs, srcs=srcs, paper=True, ckpt=10)
    np.testing.assert_array_equal(ck["g"], full["g"])
    compare(full, run_oracle(w, a, a_obs, srcs=srcs, paper=True), TOL64, TOL64)


def test_paper_adjoint_equals_exact_with_reflecting_faces(H):
    """Every face reflecting: the paper's adjoint is the exact discrete
    adjoint in another variable, so the two GPU gradients agree to rounding."""
    w = synth.small_problem(n=(13, 12, 14), fem=(3, 9), nsteps=80, omega=12.0, courant=0.8, bc=(0,) * 6,
                            refine_frac=0.3)
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + np.random.default_rng(7).random(P.n_unknown)
    a = w.a_true()
    ge = run_gpu(H, w, a, a_obs)["g"]
    gp = run_gpu(H, w, a, a_obs, paper=True)["g"]
    assert rel_l2(gp, ge) <= 1e-11


@pytest.mark.parametrize("name", sorted(OBLIQUE))
def test_fp64_parity_oblique_sources(H, name):
    w = OBLIQUE[name]()
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(4)
    a_obs = 1.0 + 2.0 * rng.random(P.n_unknown)
    a = w.a_true()
    gpu = run_gpu(H, w, a, a_obs)
    ora = run_oracle(w, a, a_obs)
    compare(gpu, ora, TOL64, TOL64)


def test_batched_axis_and_diagonal_sources(H):
    """The eight sources of the large workload (six faces, two body
    diagonals) on a small lattice, FP64 in one batch against the oracle, and
    FP32 against the oracle at the FP32 tolerances."""
    w = synth.small_problem(n=(13, 12, 14), fem=(3, 9), nsteps=60, omega=15.0, courant=0.8)
    srcs = [synth.Source(f, 15.0) for f in range(6)]
    srcs += [synth.Source(synth.FACE_ZM, 15.0, 1.0, (1.0, 1.0, 1.0)),
             synth.Source(synth.FACE_ZP, 15.0, 1.0, (-1.0, -1.0, -1.0))]
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + np.random.default_rng(6).random(P.n_unknown)
    a = w.a_true()
    ora = run_oracle(w, a, a_obs, srcs=srcs)
    compare(run_gpu(H, w, a, a_obs, srcs=srcs), ora, TOL64, TOL64)
    g32 = run_gpu(H, w, a, a_obs, precision="fp32", srcs=srcs)
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(g32["trace"][s, :, : t.shape[1]], t) <= TOL32_TRACE
    assert rel_l2(g32["g"], ora["g"]) <= TOL32_GRAD


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_parity_small(H, name):
    w = CASES[name]()
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(3)
    a_obs = 1.0 + 2.0 * rng.random(P.n_unknown)
    a = w.a_true()
    gpu = run_gpu(H, w, a, a_obs)
    ora = run_oracle(w, a, a_obs)
    compare(gpu, ora, TOL64, TOL64)


def test_fp64_parity_reference_33(H):
    """33^3, FEM nodes 8..24, absorbing faces, plane wave sin(40 t), 400 steps:
    forward at the true coefficient is the data; forward + adjoint + gradient
    at a = 1."""
    w = synth.pr1_ref_33()
    a_obs = w.a_true()
    a = np.ones(w.n_unknown)
    gpu = run_gpu(H, w, a, a_obs)
    ora = run_oracle(w, a, a_obs)
    compare(gpu, ora, TOL64, TOL64)


def test_fp32_parity_reference_33(H):
    w = synth.pr1_ref_33()
    a_obs = w.a_true()
    a = np.ones(w.n_unknown)
    gpu = run_gpu(H, w, a, a_obs, precision="fp32")
    ora = run_oracle(w, a, a_obs)
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(gpu["trace"][s, :, : t.shape[1]], t) <= TOL32_TRACE
    assert rel_l2(gpu["g"], ora["g"]) <= TOL32_GRAD


def test_fp32_parity_wide_x_faces(H):
    """FP32 on a lattice wider than one tile in x and y (tiles with a single x
    face, whose face column runs on the producer warp's lanes; a tile row off
    both y faces; items without FEM nodes on the deep copy rings), mirror x
    face carrying the source."""
    w = synth.small_problem(n=(70, 38, 19), fem=((6, 4, 4), (20, 30, 14)), nsteps=90, omega=14.0,
                            courant=0.8, bc=(0, 1, 1, 0, 1, 1), src_face=synth.FACE_XM)
    rng = np.random.default_rng(5)
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + 2.0 * rng.random(P.n_unknown)
    a = w.a_true()
    gpu = run_gpu(H, w, a, a_obs, precision="fp32")
    ora = run_oracle(w, a, a_obs)
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(gpu["trace"][s, :, : t.shape[1]], t) <= TOL32_TRACE
    assert rel_l2(gpu["g"], ora["g"]) <= TOL32_GRAD


# x extents that put node nx - 2 (the column next to the high x face) at the
# first node of a tile: FP32 tiles start at x = 32 m, FP64 tiles at 1 + 32 m
TILE_EDGE_SHAPES = {
    "fp32_tile_start_34": dict(n=(34, 12, 11), fem=((20, 3, 3), (31, 8, 7)), bc=(1, 0, 1, 1, 0, 1),
                               src_face=synth.FACE_XP),
    "fp64_tile_start_35": dict(n=(35, 12, 11), fem=((3, 3, 3), (14, 8, 7)), bc=(0, 1, 1, 0, 1, 1),
                               src_face=synth.FACE_XM),
    "two_tiles_66": dict(n=(66, 13, 12), fem=((28, 3, 3), (40, 9, 8)), bc=(0, 0, 1, 1, 1, 1),
                         src_face=synth.FACE_XP),
}


@pytest.mark.parametrize("name", sorted(TILE_EDGE_SHAPES))
def test_tile_edges_both_precisions(H, name):
    """Lattices whose x faces fall at the first or last node of a tile in
    either precision's tiling: FP64 against the oracle at 1e-12, FP32 against
    the oracle at the FP32 tolerances and against the FP64 run (trace 2e-5),
    which a wrong column anywhere would exceed by orders of magnitude."""
    w = synth.small_problem(nsteps=70, omega=14.0, courant=0.8, **TILE_EDGE_SHAPES[name])
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + 2.0 * np.random.default_rng(8).random(P.n_unknown)
    a = w.a_true()
    ora = run_oracle(w, a, a_obs)
    g64 = run_gpu(H, w, a, a_obs)
    compare(g64, ora, TOL64, TOL64)
    g32 = run_gpu(H, w, a, a_obs, precision="fp32")
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(g32["trace"][s, :, : t.shape[1]], t) <= TOL32_TRACE
        e = rel_l2(g32["trace"][s], g64["trace"][s])
        assert e <= 2e-5, f"fp32 against fp64 trace: {e}"
    assert rel_l2(g32["g"], ora["g"]) <= TOL32_GRAD


def test_batched_sources_equal_single_runs(H):
    """Sources advanced together by one launch give, per source, exactly the
    trace of a run with that source alone, and the gradient is their sum."""
    w = synth.small_problem(n=11, fem=(3, 7), nsteps=50, omega=12.0, courant=0.8)
    srcs = [synth.Source(5, 12.0), synth.Source(0, 9.0), synth.Source(3, 15.0)]
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + np.random.default_rng(1).random(P.n_unknown)
    a = w.a_true()
    both = run_gpu(H, w, a, a_obs, srcs=srcs)
    gsum = np.zeros(P.n_unknown)
    for s, src in enumerate(srcs):
        one = run_gpu(H, w, a, a_obs, srcs=[src])
        np.testing.assert_array_equal(both["trace"][s], one["trace"][0])
        gsum += one["g"]
    assert rel_l2(both["g"], gsum) < 1e-14
    ora = run_oracle(w, a, a_obs, srcs=srcs)
    compare(both, ora, TOL64, TOL64)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("refine", [0.0, 0.4])
def test_checkpoint_recompute_equals_stored_history(H, precision, refine):
    w = synth.small_problem(n=12, fem=(2, 9), nsteps=103, omega=12.0, courant=0.8, refine_frac=refine)
    P = oracle.problem_from_workload(w)
    a_obs = 1.0 + np.random.default_rng(5).random(P.n_unknown)
    a = w.a_true()
    full = run_gpu(H, w, a, a_obs, precision=precision, ckpt=0)
    for C in (1, 10, 50, 103, 200):
        ck = run_gpu(H, w, a, a_obs, precision=precision, ckpt=C)
        np.testing.assert_array_equal(ck["g"], full["g"])
        np.testing.assert_array_equal(ck["trace"], full["trace"])


def test_gradient_with_tikhonov_term(H):
    import torch
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=40, omega=12.0, courant=0.8)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a = w.a_true()
    obs = P.forward(np.ones(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    J_o, g_o, _ = oracle.value_and_grad(P, a, [src], w.nsteps, w.dt, [obs], gamma=0.7, a0=1.2,
                                        mode="quadrature")
    m = H.HybMesh.from_workload(w)
    tr = m.forward(a, [src], w.nsteps, w.dt)
    obs_t = torch.zeros_like(tr)
    obs_t[0, :, : obs.shape[1]] = torch.from_numpy(obs)
    J, cot = m.misfit(tr, obs_t, H.HYB_WEIGHTS_QUADRATURE, want_cot=True)
    m.adjoint(cot)
    g = m.gradient(a, 0.7, 1.2).cpu().numpy()
    J_tik = 0.5 * 0.7 * P.voxel_volume * np.sum((a - 1.2) ** 2)
    assert abs(J + J_tik - J_o) <= 1e-12 * J_o
    assert rel_l2(g, g_o) <= TOL64


def _alpha_tol(rep_or):
    """Relative accuracy of the step length: alpha = -J'(0) at^2 / (2 curv) with
    curv = J(at) - J(0) - J'(0) at, a difference of nearly equal numbers;
    FP64 values of J carry ~1e-13 relative error, amplified by the ratio of
    their size to curv (or alpha = at exactly when the parabola has no
    minimum)."""
    J0, Jt, dJ0, at = rep_or["J"], rep_or["J_trial"], rep_or["dJ0"], rep_or["alpha_trial"]
    curv = Jt - J0 - dJ0 * at
    if curv <= 0:
        return 1e-12
    return max(1e-12, 1e-12 * (abs(J0) + abs(Jt) + abs(dJ0 * at)) / curv)


def test_cg_steps_match_oracle(H):
    """Three iterations of Algorithm 3 (FP64) from a = a_min with data from a
    coefficient partly below it (active bounds): the coefficient after each
    iteration, J, beta and the step length agree with the oracle's."""
    import torch
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=70, omega=12.0, courant=0.8, sigma_seed=5)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    rng = np.random.default_rng(8)
    a_true = 1.0 + 2.0 * rng.random(P.n_unknown)
    a_true[rng.random(P.n_unknown) < 0.3] = 0.6
    obs = P.forward(a_true, src, w.nsteps, w.dt)["trace"]
    m = H.HybMesh.from_workload(w)
    obs_t = torch.zeros((1, w.nsteps + 1, m.obs_stride), dtype=torch.float64, device="cuda")
    obs_t[0, :, : obs.shape[1]] = torch.from_numpy(obs)
    a_gpu = torch.ones(P.n_unknown, dtype=torch.float64, device="cuda")
    st = m.new_cg_state()
    a_or = np.ones(P.n_unknown)
    st_or = {}
    for it in range(3):
        rep = m.cg_step(a_gpu, obs_t, [src], w.nsteps, w.dt, st, gamma=0.01, a0=1.0, a_min=1.0, a_max=4.0)
        a_or, st_or, rep_or = oracle.cg_step(P, a_or, [src], w.nsteps, w.dt, [obs], st_or, gamma=0.01,
                                             a0=1.0, a_min=1.0, a_max=4.0)
        assert abs(rep.J - rep_or["J"]) <= 1e-12 * rep_or["J"]
        assert abs(rep.gnorm - rep_or["gnorm"]) <= 1e-12 * rep_or["gnorm"]
        assert abs(rep.gpnorm - rep_or["gpnorm"]) <= 1e-12 * rep_or["gpnorm"]
        assert abs(rep.beta - rep_or["beta"]) <= 1e-12 * max(1.0, abs(rep_or["beta"]))
        assert abs(rep.alpha_trial - rep_or["alpha_trial"]) <= 1e-12 * rep_or["alpha_trial"]
        tol = _alpha_tol(rep_or)
        assert abs(rep.alpha - rep_or["alpha"]) <= tol * abs(rep_or["alpha"])
        assert rel_l2(a_gpu.cpu().numpy(), a_or) <= max(1e-12, tol)
    m.sync()


def test_fp32_cg_descends_and_follows_the_fp64_oracle(H):
    """Five FP32 iterations of Algorithm 3 on the 33^3 reference lattice (FEM
    17^3, two inclusions a = 2, 240 steps, data from the FP64 oracle at the
    true coefficient, gamma = 1e-4) started at a = a_min: F decreases at every
    iteration by more than the FP32 misfit's rounding (1e-4 relative), and
    the iterates stay within 1e-3 of the FP64 oracle's."""
    import torch
    w = synth.pr1_ref_33()
    w.nsteps = 240
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    obs = P.forward(w.a_true(), src, w.nsteps, w.dt)["trace"]
    m = H.HybMesh.from_workload(w, precision="fp32")
    obs_t = torch.zeros((1, w.nsteps + 1, m.obs_stride), dtype=torch.float32, device="cuda")
    obs_t[0, :, : obs.shape[1]] = torch.from_numpy(obs)
    a_gpu = torch.ones(P.n_unknown, dtype=torch.float64, device="cuda")
    st = m.new_cg_state()
    a_or = np.ones(P.n_unknown)
    st_or = {}
    Js = []
    for it in range(5):
        rep = m.cg_step(a_gpu, obs_t, [src], w.nsteps, w.dt, st, gamma=1e-4, a0=1.0, a_min=1.0, a_max=w.a_max)
        a_or, st_or, rep_or = oracle.cg_step(P, a_or, [src], w.nsteps, w.dt, [obs], st_or, gamma=1e-4,
                                             a0=1.0, a_min=1.0, a_max=w.a_max)
        Js.append(rep.J)
        assert abs(rep.J - rep_or["J"]) <= 1e-3 * rep_or["J"]
        assert rel_l2(a_gpu.cpu().numpy() - 1.0, a_or - 1.0) <= 1e-3
    assert all(Js[i + 1] < (1 - 1e-4) * Js[i] for i in range(len(Js) - 1)), Js
    m.sync()


def test_wait_limit_reports_timeout(H):
    """A mesh whose bounded pipeline waits give up at once: the step kernels
    return (no trap, no hang), hyb_sync reports HYB_ERR_TIMEOUT and clears the
    flag, and the device stays usable (a normal mesh then matches the
    oracle)."""
    w = synth.small_problem(n=(40, 24, 20), fem=((5, 4, 4), (30, 18, 15)), nsteps=12, omega=15.0, courant=0.8)
    m = H.HybMesh.from_workload(w, wait_cycles=H.HYB_WAIT_NONE)
    m.forward(w.a_true(), w.sources, w.nsteps, w.dt)
    with pytest.raises(H.HybError) as e:
        m.sync()
    assert e.value.status == H.HYB_ERR_TIMEOUT
    m.sync()  # the flag was cleared
    m.close()
    a_obs = np.ones(w.n_unknown)
    compare(run_gpu(H, w, w.a_true(), a_obs), run_oracle(w, w.a_true(), a_obs), TOL64, TOL64)


def _full_size(H, w, precision):
    """Forward at the true coefficient, a seeded random cotangent on the
    trace, adjoint and gradient, through the C ABI; the same in the oracle."""
    import torch
    m = H.HybMesh.from_workload(w, precision=precision, ckpt_every=0)
    src = w.sources[0]
    a = w.a_true()
    tr = m.forward(a, [src], w.nsteps, w.dt)
    P = oracle.problem_from_workload(w)
    n_face = P.face_nodes(src.face).size
    cot = synth.random_cotangent(1, w.nsteps, n_face, seed=11)[0] * 1e-2
    cot_t = torch.zeros_like(tr)
    cot_t[0, :, :n_face] = torch.from_numpy(cot)
    m.adjoint(cot_t)
    g = m.gradient(a, 0.0, 1.0).cpu().numpy()
    gpu = dict(trace=tr[0, :, :n_face].double().cpu().numpy(), g=g,
               u=m.field(H.HYB_FIELD_U_LAST, 0).double().cpu().numpy().ravel(),
               lam1=m.field(H.HYB_FIELD_LAMBDA_FIRST, 0).double().cpu().numpy().ravel())
    m.sync()
    m.close()
    ro = P.forward(a, src, w.nsteps, w.dt, keep_hist=True)
    go, lam1 = P.adjoint(a, src, w.nsteps, w.dt, cot, ro["hist"], return_lambda=True)
    _, ML = P.assemble(a)
    scale = np.ones(P.NT)
    scale[P.owned] = P.h ** 3 / ML[P.owned]
    ora = dict(trace=ro["trace"], g=go, u=ro["u"][: P.N], lam1=(lam1 * scale)[: P.N])
    return {k: rel_l2(gpu[k], ora[k]) for k in ora}


def test_full_size_129_fp64_across_the_fem_block(H):
    """The 129^3 / 65^3-FEM workload (refined around its inclusions) at full
    lattice size in the benchmark's launch configuration, FP64, 450 steps: by
    then the wave has crossed the FEM block's top half and reached the
    inclusions.  Trace, final field, lambda^1 and gradient within 1e-12."""
    w = synth.inverse_129(nsteps=450)
    err = _full_size(H, w, "fp64")
    print("fp64 129^3 x 450:", err)
    for k, e in err.items():
        assert e <= TOL64, (k, e)


@pytest.mark.slow
def test_full_size_129_fp32_all_steps(H):
    """The same workload in FP32 (FP64 gradient accumulation) over all 1500
    steps against the FP64 oracle: trace within 1e-4, gradient within 1e-3."""
    w = synth.inverse_129(nsteps=1500)
    err = _full_size(H, w, "fp32")
    print("fp32 129^3 x 1500 vs FP64 oracle:", err)
    assert err["trace"] <= TOL32_TRACE, err
    assert err["g"] <= TOL32_GRAD, err


def test_refined_mesh_reports_its_stability_bound(H):
    """Refined voxels lower dt_max below h / sqrt(3 a_max); a refined voxel
    too close to the outer faces is rejected."""
    w = synth.small_problem(n=11, fem=(2, 8), nsteps=10, omega=12.0, refine_frac=0.4)
    m = H.HybMesh.from_workload(w)
    info = m.query()
    assert info.n_centres == int(w.refine.sum()) and info.n_sparse_rows > info.n_centres
    assert info.dt_max < w.h / np.sqrt(3 * w.a_max)
    with pytest.raises(H.HybError) as e:
        m.forward(w.a_true(), w.sources, 5, 1.01 * info.dt_max)
    assert e.value.status == H.HYB_ERR_CFL
    w2 = synth.small_problem(n=9, fem=(0, 8), nsteps=10)  # unknown voxel 0 has a corner 1 node from the faces
    w2.refine = np.zeros(w2.n_unknown, dtype=bool)
    w2.refine[0] = True
    with pytest.raises(H.HybError) as e:
        H.HybMesh.from_workload(w2)
    assert e.value.status == H.HYB_ERR_ARG


def test_argument_and_state_errors(H):
    import torch
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=10, omega=12.0)
    m = H.HybMesh.from_workload(w)
    cot = torch.zeros((1, 11, m.obs_stride), dtype=torch.float64, device="cuda")
    with pytest.raises(H.HybError) as e:
        m.adjoint(cot)
    assert e.value.status == H.HYB_ERR_STATE
    with pytest.raises(H.HybError) as e:
        m.forward(w.a_true(), w.sources, w.nsteps, 2.0 * m.info.dt_max)
    assert e.value.status == H.HYB_ERR_CFL
    bad = w.a_true().copy()
    bad[3] = w.a_max * 2
    m.forward(bad, w.sources, w.nsteps, w.dt)
    with pytest.raises(H.HybError) as e:
        m.sync()
    assert e.value.status == H.HYB_ERR_CFL
    m.sync()  # the flag was cleared


def test_graph_replay_is_bitwise_identical(H):
    """Repeating a sweep with the same buffers replays a captured CUDA graph
    (from the third call on); results are bitwise those of direct launches."""
    import torch
    w = synth.small_problem(n=12, fem=(3, 8), nsteps=40, omega=12.0, courant=0.8)
    m = H.HybMesh.from_workload(w)
    a = torch.tensor(w.a_true(), dtype=torch.float64, device="cuda")
    trace = m.new_trace(1, w.nsteps)
    cot = torch.randn_like(trace)
    g = torch.empty(m.n_unknown, dtype=torch.float64, device="cuda")
    outs = []
    for it in range(4):
        m.forward(a, w.sources, w.nsteps, w.dt, trace)
        m.adjoint(cot)
        m.gradient(a, 0.0, 1.0, out=g)
        outs.append((trace.clone(), g.clone()))
    m.sync()
    for t, gg in outs[1:]:
        assert torch.equal(t, outs[0][0]) and torch.equal(gg, outs[0][1])


# ---------------------------------------------------------- Model Problem 1
def _model1(H, w, a, a_obs, ckpt=0, paper=False):
    """GPU and oracle runs of Model Problem 1: both start from the state of
    Eq. (initcond) (synth.model1_initial)."""
    import torch
    (u0, um), (c0, cm) = synth.model1_initial(w)
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=ckpt,
                                adjoint_mode=H.HYB_ADJ_PAPER if paper else H.HYB_ADJ_EXACT)
    m.set_initial(u0, um, c0 if c0.size else None, cm if cm.size else None)
    obs = m.forward(a_obs, w.sources, w.nsteps, w.dt).clone()
    tr = m.forward(a, w.sources, w.nsteps, w.dt)
    u_last = m.field(H.HYB_FIELD_U_LAST, 0).cpu().numpy().ravel()  # (a checkpointed adjoint reuses the levels)
    J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_PLAIN, want_cot=True)
    m.adjoint(cot)
    g = m.gradient(a, 0.0, 1.0)
    gpu = dict(trace=tr.double().cpu().numpy(), J=J, g=g.cpu().numpy(), u=[u_last],
               lam1=[m.field(H.HYB_FIELD_LAMBDA_FIRST, 0).cpu().numpy().ravel()])
    m.sync()
    m.close()
    P = oracle.problem_from_workload(w)
    init = (np.concatenate([u0, c0]), np.concatenate([um, cm]))
    src = w.sources[0]
    ro = P.forward(a, src, w.nsteps, w.dt, keep_hist=True, init=init)
    oo = P.forward(a_obs, src, w.nsteps, w.dt, init=init)["trace"]
    c = ro["trace"] - oo
    if paper:
        go, lam = P.adjoint_paper(a, src, w.nsteps, w.dt, c, ro["hist"], return_lambda=True)
        lam = lam[: P.N]
    else:
        go, lam = P.adjoint(a, src, w.nsteps, w.dt, c, ro["hist"], return_lambda=True)
        _, ML = P.assemble(a)
        scale = np.ones(P.NT)
        scale[P.owned] = P.h ** 3 / ML[P.owned]
        lam = (lam * scale)[: P.N]
    ora = dict(trace=[ro["trace"]], J=0.5 * float(np.sum(c[1:] ** 2)), g=go, u=[ro["u"][: P.N]], lam1=[lam],
               kappa=[float(np.linalg.norm(ro["trace"]) / np.linalg.norm(c))])
    return gpu, ora


MODEL1_CASES = {
    "abc": lambda: synth.small_problem(n=11, fem=(3, 7), nsteps=70, omega=12.0, courant=0.8),
    "refined_mixed": lambda: synth.small_problem(n=(12, 11, 13), fem=((2, 2, 2), (9, 8, 10)), nsteps=60,
                                                 omega=12.0, courant=0.8, refine_frac=0.5, bc=(0, 1, 0, 1, 1, 1)),
    "wide_tiles": lambda: synth.small_problem(n=(37, 21, 19), fem=((5, 4, 4), (30, 16, 15)), nsteps=45,
                                              omega=15.0, courant=0.9, sigma_scale=2.0),
}


@pytest.mark.parametrize("ckpt", [0, 9])
@pytest.mark.parametrize("name", sorted(MODEL1_CASES))
def test_fp64_parity_model1(H, name, ckpt):
    """Model Problem 1 (nonzero initial state, Eq. (initcond)): trace (row 0 =
    u^0 on the face), final field, lambda^1 and the gradient with its k = 0
    pairing term against the oracle, with stored history and with
    checkpoint/recompute (segment 0 restarts from the initial state)."""
    w = MODEL1_CASES[name]()
    w.origin = tuple(-0.5 * (n - 1) * w.h for n in w.n)
    a_obs = 1.0 + 2.0 * np.random.default_rng(12).random(w.n_unknown)
    gpu, ora = _model1(H, w, w.a_true(), a_obs, ckpt=ckpt)
    compare(gpu, ora, TOL64, TOL64)


def test_fp64_parity_model1_paper_adjoint(H):
    w = MODEL1_CASES["refined_mixed"]()
    w.origin = tuple(-0.5 * (n - 1) * w.h for n in w.n)
    a_obs = 1.0 + 2.0 * np.random.default_rng(13).random(w.n_unknown)
    gpu, ora = _model1(H, w, w.a_true(), a_obs, ckpt=7, paper=True)
    compare(gpu, ora, TOL64, TOL64)


# -------------------------------------------------- pure FEM (HYB_FEM_TET_ALL)
def _all_fem_oracle(w, a, a_obs):
    """The oracle with a FEM block over the whole lattice (every voxel cut
    into Kuhn tetrahedra, every interior node a FEM row, the outer boundary
    rows FDM), its coefficient laid out from the hybrid's unknown voxels
    (a = 1 elsewhere).  Returns the oracle results and the index map from the
    hybrid's unknown voxels into the all-FEM ones."""
    n = w.n
    Q = oracle.hybrid.Problem(n, w.h, (0, 0, 0), tuple(v - 1 for v in n), w.bc, w.origin)
    ud, qd = w.unknown_dims, Q.unknown_dims
    x, y, z = np.meshgrid(np.arange(ud[0]), np.arange(ud[1]), np.arange(ud[2]), indexing="ij")
    off = [w.fem_lo[d] + 1 - 1 for d in range(3)]  # unknown voxel origins fem_lo+1.. vs 1..
    idx = ((x + off[0]) + qd[0] * ((y + off[1]) + qd[1] * (z + off[2]))).transpose(2, 1, 0).ravel()
    res = dict(trace=[], J=0.0, g=np.zeros(w.n_unknown), u=[], lam1=[], kappa=[])
    for src in w.sources:
        aq = np.ones(Q.n_unknown)
        aq[idx] = a
        aq_obs = np.ones(Q.n_unknown)
        aq_obs[idx] = a_obs
        ro = Q.forward(aq, src, w.nsteps, w.dt, keep_hist=True)
        c = ro["trace"] - Q.forward(aq_obs, src, w.nsteps, w.dt)["trace"]
        res["J"] += 0.5 * float(np.sum(c[1:] ** 2))
        res["trace"].append(ro["trace"])
        res["u"].append(ro["u"][: Q.N])
        gq, lam1 = Q.adjoint(aq, src, w.nsteps, w.dt, c, ro["hist"], return_lambda=True)
        res["g"] += gq[idx]
        _, ML = Q.assemble(aq)
        scale = np.ones(Q.NT)
        scale[Q.owned] = Q.h ** 3 / ML[Q.owned]
        res["lam1"].append((lam1 * scale)[: Q.N])
        res["kappa"].append(float(np.linalg.norm(ro["trace"]) / np.linalg.norm(c)))
    return res


TET_CASES = {
    "abc": lambda: synth.small_problem(n=10, fem=(3, 7), nsteps=50, omega=12.0, courant=0.8),
    "mixed_bc_ragged": lambda: synth.small_problem(n=(9, 10, 11), fem=(2, 6), nsteps=60, omega=12.0,
                                                   bc=(0, 1, 1, 0, 1, 1), courant=0.8),
    "diag_source": lambda: _oblique(synth.small_problem(n=10, fem=(2, 7), nsteps=60, omega=14.0, courant=0.8),
                                    [synth.Source(synth.FACE_ZM, 14.0, 1.0, (1.0, 1.0, 1.0))]),
}


@pytest.mark.parametrize("name", sorted(TET_CASES))
def test_fp64_parity_all_fem_path(H, name):
    """HYB_FEM_TET_ALL (rows gathered element by element over the Kuhn
    tetrahedra of every voxel) against the oracle's all-FEM problem."""
    w = TET_CASES[name]()
    a_obs = 1.0 + 2.0 * np.random.default_rng(14).random(w.n_unknown)
    a = w.a_true()
    import torch
    m = H.HybMesh.from_workload(w, fem_path=H.HYB_FEM_TET_ALL)
    obs = m.forward(a_obs, w.sources, w.nsteps, w.dt).clone()
    tr = m.forward(a, w.sources, w.nsteps, w.dt)
    J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_PLAIN, want_cot=True)
    m.adjoint(cot)
    gpu = dict(trace=tr.double().cpu().numpy(), J=J, g=m.gradient(a, 0.0, 1.0).cpu().numpy(),
               u=[m.field(H.HYB_FIELD_U_LAST, 0).cpu().numpy().ravel()],
               lam1=[m.field(H.HYB_FIELD_LAMBDA_FIRST, 0).cpu().numpy().ravel()])
    m.sync()
    m.close()
    compare(gpu, _all_fem_oracle(w, a, a_obs), TOL64, TOL64)


@pytest.mark.parametrize("config", ["pr1_ref_33", "autograd_97"])
def test_hybrid_equals_pure_fem_on_the_gpu(H, config):
    """The hybrid run (FDM outside the FEM block, stencil-form FEM rows inside)
    equals the pure-FEM run (every interior row gathered over tetrahedra) to
    1e-13 relative L2 in FP64: trace, final field and gradient, on the 33^3
    reference workload (400 steps) and the 97^3 workload (1200 steps): the
    two schemes coincide on the structured mesh (Sec. 1, Sec. 7)."""
    import torch
    w = getattr(synth, config)()
    a = w.a_true()
    out = {}
    for path in (H.HYB_FEM_STENCIL, H.HYB_FEM_TET_ALL):
        m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0, fem_path=path)
        obs = m.forward(np.ones(w.n_unknown), w.sources, w.nsteps, w.dt).clone()
        tr = m.forward(a, w.sources, w.nsteps, w.dt)
        J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_PLAIN, want_cot=True)
        m.adjoint(cot)
        out[path] = (tr.double().cpu().numpy(), m.field(H.HYB_FIELD_U_LAST, 0).cpu().numpy(),
                     m.gradient(a, 0.0, 1.0).cpu().numpy())
        m.sync()
        m.close()
    for q, name in enumerate(("trace", "field", "gradient")):
        e = rel_l2(out[H.HYB_FEM_TET_ALL][q], out[H.HYB_FEM_STENCIL][q])
        print(f"{config}: hybrid vs pure FEM {name}: {e:.2e}")
        assert e <= 1e-13, (name, e)

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


def run_gpu(H, w, a, a_obs, precision="fp64", ckpt=None, srcs=None):
    import torch
    srcs = srcs or w.sources
    m = H.HybMesh.from_workload(w, precision=precision, ckpt_every=ckpt)
    obs = m.forward(a_obs, srcs, w.nsteps, w.dt)
    tr = m.forward(a, srcs, w.nsteps, w.dt)
    J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_PLAIN, want_cot=True)
    m.adjoint(cot)
    g = m.gradient(a, 0.0, 1.0)
    u_last = [m.field(H.HYB_FIELD_U_LAST, s).cpu().numpy().ravel() for s in range(len(srcs))]
    lam1 = [m.field(H.HYB_FIELD_LAMBDA_FIRST, s).cpu().numpy().ravel() for s in range(len(srcs))]
    m.sync()
    out = dict(trace=tr.double().cpu().numpy(), J=J, g=g.cpu().numpy(), u=u_last, lam1=lam1,
               launches=m.launches())
    m.close()
    return out


def run_oracle(w, a, a_obs, srcs=None):
    srcs = srcs or w.sources
    P = oracle.problem_from_workload(w)
    res = dict(trace=[], J=0.0, g=np.zeros(P.n_unknown), u=[], lam1=[])
    for src in srcs:
        ro = P.forward(a, src, w.nsteps, w.dt, keep_hist=True)
        oo = P.forward(a_obs, src, w.nsteps, w.dt)["trace"]
        c = ro["trace"] - oo
        res["J"] += 0.5 * float(np.sum(c[1:] ** 2))
        res["trace"].append(ro["trace"])
        res["u"].append(ro["u"][: P.N])  # lattice nodes (centre nodes of refined voxels follow)
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
    tol_field = tol_trace if tol_field is None else tol_field
    for s, t in enumerate(ora["trace"]):
        e = rel_l2(gpu["trace"][s, :, : t.shape[1]], t)
        assert e <= tol_trace, f"trace src {s}: {e}"
        assert rel_l2(gpu["u"][s], ora["u"][s]) <= tol_field
        assert rel_l2(gpu["lam1"][s], ora["lam1"][s]) <= tol_field * 10
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


def test_cg_steps_match_oracle(H):
    """Two iterations of Algorithm 3 (FP64): the coefficient after each
    iteration, J, beta and the step length agree with the oracle."""
    import torch
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=70, omega=12.0, courant=0.8, sigma_seed=5)
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    a_true = 1.0 + 2.0 * np.random.default_rng(8).random(P.n_unknown)
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
        assert abs(rep.J - rep_or["J"]) <= 1e-11 * rep_or["J"]
        assert abs(rep.beta - rep_or["beta"]) <= 1e-9 * max(1.0, abs(rep_or["beta"]))
        assert abs(rep.alpha - rep_or["alpha"]) <= 1e-9 * abs(rep_or["alpha"])
        assert rel_l2(a_gpu.cpu().numpy(), a_or) <= 1e-10
    m.sync()


@pytest.mark.parametrize("precision,steps", [("fp64", 60), ("fp32", 120)])
def test_full_size_129_first_steps(H, precision, steps):
    """The 129^3 / 65^3-FEM workload at its full lattice size in the launch
    configuration the benchmark uses, over its first steps (the oracle's time
    bound): trace, final field and gradient against the FP64 oracle."""
    w = synth.inverse_129(nsteps=steps)
    a = w.a_true()
    a_obs = np.ones(w.n_unknown)
    gpu = run_gpu(H, w, a, a_obs, precision=precision)
    ora = run_oracle(w, a, a_obs)
    if precision == "fp64":
        compare(gpu, ora, TOL64, TOL64)
    else:
        t = ora["trace"][0]
        assert rel_l2(gpu["trace"][0, :, : t.shape[1]], t) <= TOL32_TRACE
        assert rel_l2(gpu["g"], ora["g"]) <= TOL32_GRAD


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

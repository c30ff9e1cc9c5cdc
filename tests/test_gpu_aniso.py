"""Per-axis lattice steps dx_1, dx_2, dx_3 (the 7-point Laplacian of Sec. 7.3
with unequal steps, brick Kuhn elements) through the C ABI against the FP64
oracle: traces, J and gradients with plain and quadrature weights, face and
oblique sources, absorbing and reflecting faces, at 1e-12 in FP64 and at the
FP32 tolerances; the checkpointed adjoint equal to the stored-history one;
equal steps equal to the isotropic lattice; the pure-FEM path equal to the
hybrid one on bricks; three CG iterations against the oracle's; the bound
dt_max and the refusals."""
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


CASES = {
    "bricks_13": lambda: synth.small_problem(n=(13, 12, 14), fem=((2, 2, 3), (9, 9, 10)), nsteps=80, omega=14.0,
                                             courant=0.8, spacing=(0.08, 0.1, 0.065)),
    "mixed_bc_x_source": lambda: synth.small_problem(n=(15, 11, 12), fem=((3, 2, 2), (11, 8, 9)), nsteps=80,
                                                     omega=14.0, courant=0.8, bc=(1, 0, 1, 1, 0, 1),
                                                     src_face=synth.FACE_XP, spacing=(0.06, 0.09, 0.075)),
    "wide": lambda: synth.small_problem(n=(37, 21, 19), fem=((5, 4, 4), (30, 16, 15)), nsteps=70, omega=15.0,
                                        courant=0.9, spacing=(0.03, 0.05, 0.045)),
    # most nodes away from the faces and the FEM block (the kernels' plain rows)
    "fast_rows_41": lambda: synth.small_problem(n=(41, 33, 49), fem=((8, 8, 10), (32, 24, 38)), nsteps=120,
                                                omega=20.0, courant=0.85, spacing=(0.025, 0.03, 0.02)),
}


def _coefs(w, seed):
    rng = np.random.default_rng(seed)
    return 1.0 + 2.0 * rng.random(w.n_unknown), 1.0 + 2.0 * rng.random(w.n_unknown)


def _run(H, w, a, a_obs, weights, precision="fp64", ckpt=0, srcs=None, **kw):
    srcs = srcs or w.sources
    m = H.HybMesh.from_workload(w, precision=precision, ckpt_every=ckpt, **kw)
    obs = m.forward(a_obs, srcs, w.nsteps, w.dt)
    tr = m.forward(a, srcs, w.nsteps, w.dt)
    J, cot = m.misfit(tr, obs, weights, want_cot=True)
    m.adjoint(cot)
    g = m.gradient(a, 0.0, 1.0)
    m.sync()
    out = dict(trace=tr.double().cpu().numpy(), J=J, g=g.cpu().numpy(), info=m.query())
    m.close()
    return out


def _oracle(w, a, a_obs, mode, srcs=None):
    srcs = srcs or w.sources
    P = oracle.problem_from_workload(w)
    obs = [P.forward(a_obs, s, w.nsteps, w.dt)["trace"] for s in srcs]
    J, g, traces = oracle.value_and_grad(P, a, srcs, w.nsteps, w.dt, obs, mode=mode)
    return dict(trace=traces, J=J, g=g)


def _check(gpu, ora, tol_trace, tol_grad, tol_J):
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(gpu["trace"][s, :, : t.shape[1]], t) <= tol_trace, s
    assert abs(gpu["J"] - ora["J"]) <= tol_J * ora["J"]
    assert rel_l2(gpu["g"], ora["g"]) <= tol_grad


@pytest.mark.parametrize("mode", ["plain", "quadrature"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_parity(H, name, mode):
    w = CASES[name]()
    a, a_obs = _coefs(w, 21)
    weights = H.HYB_WEIGHTS_PLAIN if mode == "plain" else H.HYB_WEIGHTS_QUADRATURE
    gpu = _run(H, w, a, a_obs, weights)
    _check(gpu, _oracle(w, a, a_obs, mode), TOL64, TOL64, 1e-11)


def test_oblique_and_face_sources_quadrature(H):
    """A face source observed on its face and a plane wave along (1, 2, 3)
    entering through the three low faces, observed on the low z face: the
    delays d . (x - x0) and switch times axis by axis, and each face's own
    quadrature area."""
    w = CASES["bricks_13"]()
    srcs = [synth.Source(synth.FACE_YP, 14.0), synth.Source(synth.FACE_ZM, 14.0, 1.0, (1.0, 2.0, 3.0))]
    a, a_obs = _coefs(w, 22)
    gpu = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE, srcs=srcs)
    _check(gpu, _oracle(w, a, a_obs, "quadrature", srcs=srcs), TOL64, TOL64, 1e-11)


def test_fp32_parity(H):
    w = CASES["wide"]()
    a, a_obs = _coefs(w, 23)
    gpu = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE, precision="fp32")
    _check(gpu, _oracle(w, a, a_obs, "quadrature"), TOL32_TRACE, TOL32_GRAD, 1e-3)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpointed_adjoint_equals_stored_history(H, precision):
    w = CASES["mixed_bc_x_source"]()
    a, a_obs = _coefs(w, 24)
    full = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE, precision=precision)
    ck = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE, precision=precision, ckpt=20)
    np.testing.assert_array_equal(ck["trace"], full["trace"])
    np.testing.assert_array_equal(ck["g"], full["g"])


def test_equal_steps_are_the_isotropic_lattice_bitwise(H):
    w = synth.small_problem(n=(13, 12, 14), fem=((2, 2, 3), (9, 9, 10)), nsteps=60, omega=14.0, courant=0.8)
    a, a_obs = _coefs(w, 25)
    iso = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE)
    w.spacing = (w.h, w.h, w.h)
    eq = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE)
    np.testing.assert_array_equal(eq["trace"], iso["trace"])
    np.testing.assert_array_equal(eq["g"], iso["g"])


def test_pure_fem_path_equals_the_hybrid_path_on_bricks(H):
    """Every interior row gathered over the brick's Kuhn tetrahedra (a = 1
    off the unknown voxels) against the hybrid scheme's stencil rows: the
    schemes coincide on the structured lattice (Sec. 1, Sec. 7)."""
    w = CASES["bricks_13"]()
    a, a_obs = _coefs(w, 26)
    hyb = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE)
    fem = _run(H, w, a, a_obs, H.HYB_WEIGHTS_QUADRATURE, fem_path=H.HYB_FEM_TET_ALL)
    assert rel_l2(fem["trace"], hyb["trace"]) <= TOL64
    assert rel_l2(fem["g"], hyb["g"]) <= TOL64


def test_cg_iterations_match_the_oracle(H):
    """Three FP64 iterations of Algorithm 3 with quadrature weights (the
    L2 norms and Tikhonov term over brick voxels of volume dx_1 dx_2 dx_3)."""
    import torch
    w = CASES["bricks_13"]()
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    rng = np.random.default_rng(27)
    a_true = 1.0 + 2.0 * rng.random(P.n_unknown)
    obs = P.forward(a_true, src, w.nsteps, w.dt)["trace"]
    m = H.HybMesh.from_workload(w)
    obs_t = torch.zeros((1, w.nsteps + 1, m.obs_stride), dtype=torch.float64, device="cuda")
    obs_t[0, :, : obs.shape[1]] = torch.from_numpy(obs)
    a_gpu = torch.ones(P.n_unknown, dtype=torch.float64, device="cuda")
    st = m.new_cg_state()
    a_or, st_or = np.ones(P.n_unknown), {}
    for _ in range(3):
        rep = m.cg_step(a_gpu, obs_t, [src], w.nsteps, w.dt, st, gamma=0.01, a0=1.0, a_min=1.0, a_max=4.0)
        a_or, st_or, ro = oracle.cg_step(P, a_or, [src], w.nsteps, w.dt, [obs], st_or, gamma=0.01, a0=1.0,
                                         a_min=1.0, a_max=4.0)
        assert abs(rep.J - ro["J"]) <= 1e-11 * ro["J"]
        assert abs(rep.gnorm - ro["gnorm"]) <= 1e-11 * ro["gnorm"]
        assert abs(rep.alpha_trial - ro["alpha_trial"]) <= 1e-11 * ro["alpha_trial"]
        curv = ro["J_trial"] - ro["J"] - ro["dJ0"] * ro["alpha_trial"]
        tol = 1e-12 if curv <= 0 else max(1e-12, 1e-12 * (abs(ro["J"]) + abs(ro["J_trial"]) +
                                                        abs(ro["dJ0"] * ro["alpha_trial"])) / curv)
        assert abs(rep.alpha - ro["alpha"]) <= 10 * tol * abs(ro["alpha"])
        assert rel_l2(a_gpu.cpu().numpy(), a_or) <= max(1e-11, 10 * tol)
    m.sync()
    m.close()


def test_step_bound_volume_and_refusals(H):
    w = CASES["bricks_13"]()
    hv = w.spacing
    m = H.HybMesh.from_workload(w)
    info = m.query()
    bound = 1.0 / math.sqrt(w.a_max * sum(1.0 / (d * d) for d in hv))
    assert abs(info.dt_max - bound) <= 1e-15 * bound
    assert abs(info.voxel_volume - hv[0] * hv[1] * hv[2]) <= 1e-15 * info.voxel_volume
    with pytest.raises(H.HybError) as e:
        m.forward(w.a_true(), w.sources, 5, 1.01 * bound)
    assert e.value.status == H.HYB_ERR_CFL
    m.close()
    refine = np.zeros(w.n_unknown, dtype=bool)
    refine[0] = True
    for kw in (dict(refine=refine), dict(adjoint_mode=H.HYB_ADJ_PAPER), dict(model=H.HYB_MODEL_TELEGRAPH),
               dict(spacing=(0.1, -0.1, 0.1))):
        with pytest.raises(H.HybError) as e:
            H.HybMesh.from_workload(w, **kw)
        assert e.value.status == H.HYB_ERR_ARG
    import torch
    m = H.HybMesh.from_workload(w)
    a = torch.ones((1, w.n_unknown), dtype=torch.float64, device="cuda")
    tr = m.new_trace(1, 5)
    with pytest.raises(H.HybError) as e:
        H.hyb_forward_batch(m.handle, a.data_ptr(), w.sources, 5, w.dt, tr.data_ptr())
    assert e.value.status == H.HYB_ERR_ARG
    m.close()


def test_full_size_plane_wave_is_one_dimensional(H):
    """The anisotropic box at its full size (257 x 193 x 321 nodes, the
    bench's lattice, FEM block and launch configuration, FP64) with
    reflecting x and y faces, a = 1 and a source on the high z face: every
    node of the z face records the 1-D leapfrog along z with step 2/320
    (written out in the oracle pins).  500 steps: the pulse crosses the FEM
    block (z nodes 80..240) and anything a wrong row there reflected would
    be back on the face."""
    from test_oracle_aniso import _leapfrog_1d
    w = synth.anisotropic_box(nsteps=500, n_src=1)
    w.bc = (0, 0, 0, 0, 1, 1)
    src = synth.Source(synth.FACE_ZP, 40.0)
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0)
    tr = m.forward(np.ones(w.n_unknown), [src], w.nsteps, w.dt)
    m.sync()
    nf = w.n[0] * w.n[1]
    t = tr[0, :, :nf].cpu().numpy()
    m.close()
    ref = _leapfrog_1d(w.n[2], w.hv[2], w.dt, w.nsteps, 40.0, 1.0, True)
    assert np.abs(ref).max() > 1e-3
    err = np.abs(t - ref[:, None]).max() / np.abs(ref).max()
    assert err <= 1e-12, err

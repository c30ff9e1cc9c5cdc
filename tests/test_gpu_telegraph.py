"""The telegraph reading (HYB_MODEL_TELEGRAPH: u_tt + sigma u_t - div grad u = 0
with sigma on the unknown voxels) through the C ABI against the FP64 oracle:
traces and sigma-gradients at 1e-12 (FP64) and at the FP32 tolerances, the
checkpointed adjoint equal to the stored-history one, sigma = 0 equal to the
wave model, and the refusals of what the model does not take."""
import numpy as np
import pytest

import oracle
import synth
from helpers import rel_l2
from oracle import hybrid as O

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
    "cube_11": lambda: synth.small_problem(n=11, fem=(3, 7), nsteps=70, omega=14.0, courant=0.8),
    "ragged_mixed_bc": lambda: synth.small_problem(n=(13, 12, 14), fem=((2, 2, 3), (9, 9, 10)), nsteps=70,
                                                   omega=14.0, courant=0.8, bc=(0, 1, 1, 0, 1, 1)),
    "wide_tiles": lambda: synth.small_problem(n=(37, 21, 19), fem=((5, 4, 4), (30, 16, 15)), nsteps=60,
                                              omega=15.0, courant=0.9),
}


def _run(H, w, sigma, sig_obs, precision="fp64", ckpt=0, srcs=None):
    srcs = srcs or w.sources
    m = H.HybMesh.from_workload(w, precision=precision, ckpt_every=ckpt, model=H.HYB_MODEL_TELEGRAPH)
    obs = m.forward(sig_obs, srcs, w.nsteps, w.dt)
    tr = m.forward(sigma, srcs, w.nsteps, w.dt)
    J, cot = m.misfit(tr, obs, H.HYB_WEIGHTS_PLAIN, want_cot=True)
    m.adjoint(cot)
    g = m.gradient(sigma, 0.0, 0.0)
    m.sync()
    out = dict(trace=tr.double().cpu().numpy(), J=J, g=g.cpu().numpy())
    m.close()
    return out


def _oracle(w, sigma, sig_obs, srcs=None):
    srcs = srcs or w.sources
    P = oracle.problem_from_workload(w)
    obs = [O.telegraph_forward(P, sig_obs, s, w.nsteps, w.dt)["trace"] for s in srcs]
    J, g, traces = O.telegraph_value_and_grad(P, sigma, srcs, w.nsteps, w.dt, obs)
    return dict(trace=traces, J=J, g=g)


def _sigmas(w, seed):
    rng = np.random.default_rng(seed)
    return 2.0 * rng.random(w.n_unknown), 2.0 * rng.random(w.n_unknown)


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_parity(H, name):
    w = CASES[name]()
    sigma, sig_obs = _sigmas(w, 11)
    gpu = _run(H, w, sigma, sig_obs)
    ora = _oracle(w, sigma, sig_obs)
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(gpu["trace"][s, :, : t.shape[1]], t) <= TOL64
    assert abs(gpu["J"] - ora["J"]) <= 1e-11 * ora["J"]
    assert rel_l2(gpu["g"], ora["g"]) <= TOL64


def test_fp32_parity(H):
    w = CASES["wide_tiles"]()
    sigma, sig_obs = _sigmas(w, 12)
    gpu = _run(H, w, sigma, sig_obs, precision="fp32")
    ora = _oracle(w, sigma, sig_obs)
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(gpu["trace"][s, :, : t.shape[1]], t) <= TOL32_TRACE
    assert rel_l2(gpu["g"], ora["g"]) <= TOL32_GRAD


def test_several_sources_oblique(H):
    w = CASES["ragged_mixed_bc"]()
    srcs = [synth.Source(synth.FACE_ZP, 14.0), synth.Source(synth.FACE_ZM, 14.0, 1.0, (1.0, 1.0, 1.0))]
    sigma, sig_obs = _sigmas(w, 13)
    gpu = _run(H, w, sigma, sig_obs, srcs=srcs)
    ora = _oracle(w, sigma, sig_obs, srcs=srcs)
    for s, t in enumerate(ora["trace"]):
        assert rel_l2(gpu["trace"][s, :, : t.shape[1]], t) <= TOL64
    assert rel_l2(gpu["g"], ora["g"]) <= TOL64


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpointed_adjoint_equals_stored_history(H, precision):
    """Checkpoints every 20 steps (segments recomputed one step further for
    u^{k+1} - u^{k-1}) give the same gradient, bitwise, as the full history."""
    w = CASES["cube_11"]()
    sigma, sig_obs = _sigmas(w, 14)
    full = _run(H, w, sigma, sig_obs, precision=precision)
    ck = _run(H, w, sigma, sig_obs, precision=precision, ckpt=20)
    np.testing.assert_array_equal(ck["trace"], full["trace"])
    np.testing.assert_array_equal(ck["g"], full["g"])


def test_zero_damping_is_the_wave_model(H):
    w = CASES["cube_11"]()
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0)
    t_wave = m.forward(np.ones(w.n_unknown), w.sources, w.nsteps, w.dt).double().cpu().numpy()
    m.close()
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0, model=H.HYB_MODEL_TELEGRAPH)
    t_tel = m.forward(np.zeros(w.n_unknown), w.sources, w.nsteps, w.dt).double().cpu().numpy()
    m.close()
    assert rel_l2(t_tel, t_wave) <= 1e-14


def test_refusals(H):
    w = synth.small_problem(n=11, fem=(1, 7), nsteps=10)
    with pytest.raises(H.HybError) as e:
        H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0, model=H.HYB_MODEL_TELEGRAPH)
    assert e.value.status == H.HYB_ERR_ARG
    w = CASES["cube_11"]()
    with pytest.raises(H.HybError) as e:
        H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0, model=H.HYB_MODEL_TELEGRAPH,
                                adjoint_mode=H.HYB_ADJ_PAPER)
    assert e.value.status == H.HYB_ERR_ARG
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=0, model=H.HYB_MODEL_TELEGRAPH)
    sig = -np.ones(w.n_unknown)
    m.forward(sig, w.sources, w.nsteps, w.dt)
    with pytest.raises(H.HybError) as e:
        m.sync()
    assert e.value.status == H.HYB_ERR_CFL
    m.close()

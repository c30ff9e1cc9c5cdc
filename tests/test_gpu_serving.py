"""Serving form: continuous batching of FP32 forward + adjoint + gradient
solves of different lattice sizes, admitted by an HBM budget."""
import numpy as np
import pytest

import oracle
import synth
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01399_gb300 import serve
    return serve


def _requests(n, sizes=(25, 29, 33), nsteps=60, spread=0.0):
    reqs = []
    for i in range(n):
        w = synth.serving_request(i, sizes=sizes, nsteps=nsteps)
        reqs.append((w, spread * i))
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix(S):
    """Requests batched with others of their class (one launch per level
    advancing all of them) and overlapping with other classes' batches give
    bitwise the result of a solve alone."""
    from paper_1509_01399_gb300.serve import Request, ServingEngine
    reqs = _requests(12)
    eng = ServingEngine(workers=2, max_batch=4)
    mix = eng.run([Request(i, w, t) for i, (w, t) in enumerate(reqs)])
    assert eng.max_batch_seen >= 2, "requests of one class should share launches"
    alone = ServingEngine(workers=1)
    for i, (w, _) in enumerate(reqs):
        r = alone.solve(Request(i, w, 0.0))
        np.testing.assert_array_equal(r.gradient, mix[i].gradient)
        assert r.J == mix[i].J
    eng.close()
    alone.close()


def test_admission_respects_the_hbm_budget(S):
    from paper_1509_01399_gb300.serve import Request, ServingEngine, estimate_bytes
    reqs = _requests(8, sizes=(25, 33), spread=0.0)
    biggest = max(estimate_bytes(w, "fp32") for w, _ in reqs)
    eng = ServingEngine(hbm_budget=int(1.2 * biggest * 4), workers=4, max_batch=4)
    res = eng.run([Request(i, w, t) for i, (w, t) in enumerate(reqs)])
    assert len(res) == 8 and all(np.isfinite(r.gradient).all() for r in res)
    assert eng.max_meshes <= 2
    eng.close()


def test_served_gradient_matches_the_oracle(S):
    from paper_1509_01399_gb300.serve import Request, ServingEngine
    w = synth.serving_request(3, sizes=(25,), nsteps=80)
    eng = ServingEngine(workers=2)
    r = eng.solve(Request(0, w, 0.0))
    eng.close()
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    obs = P.forward(np.ones(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    J, g, _ = oracle.value_and_grad(P, w.a_true(), [src], w.nsteps, w.dt, [obs])
    assert rel_l2(r.gradient, g) <= 1e-3
    assert abs(r.J - J) <= 1e-3 * J


def test_batched_forward_equals_single_problems(S):
    """hyb_forward_batch: three problems of one lattice class with their own
    coefficients and sources in one batch; per slot the trace, the misfit and
    the gradient are bitwise those of the problem alone, and match the FP64
    oracle."""
    import torch
    from paper_1509_01399_gb300 import hyb as H
    w = synth.small_problem(n=(13, 12, 11), fem=(3, 8), nsteps=50, omega=12.0, courant=0.8, refine_frac=0.3)
    P = oracle.problem_from_workload(w)
    rng = np.random.default_rng(17)
    coefs = [1.0 + 2.0 * rng.random(P.n_unknown) for _ in range(3)]
    srcs = [synth.Source(5, 12.0), synth.Source(0, 9.0), synth.Source(synth.FACE_ZM, 14.0, 1.0, (1.0, 1.0, 1.0))]
    m = H.HybMesh.from_workload(w, precision="fp64")
    # zero observations: the residual is the trace itself (no cancellation)
    obs = torch.zeros((3, w.nsteps + 1, m.obs_stride), dtype=torch.float64, device="cuda")
    a = torch.tensor(np.stack(coefs), dtype=torch.float64, device="cuda")
    tr = m.new_trace(3, w.nsteps)
    H.hyb_forward_batch(m.handle, a.data_ptr(), srcs, w.nsteps, w.dt, tr.data_ptr())
    cot = torch.empty_like(tr)
    J = H.hyb_misfit_batch(m.handle, tr.data_ptr(), obs.data_ptr(), H.HYB_WEIGHTS_PLAIN, 3, cot.data_ptr())
    H.hyb_adjoint(m.handle, cot.data_ptr(), 0)
    g = torch.empty((3, P.n_unknown), dtype=torch.float64, device="cuda")
    H.hyb_gradient_batch(m.handle, a.data_ptr(), 0.0, 1.0, g.data_ptr())
    m.sync()
    for s_ in range(3):
        one = H.HybMesh.from_workload(w, precision="fp64")
        t1 = one.forward(coefs[s_], [srcs[s_]], w.nsteps, w.dt)
        J1, c1 = one.misfit(t1, obs[s_:s_ + 1], H.HYB_WEIGHTS_PLAIN, want_cot=True)
        one.adjoint(c1)
        g1 = one.gradient(coefs[s_], 0.0, 1.0)
        one.sync()
        assert torch.equal(tr[s_], t1[0]) and torch.equal(g[s_], g1) and J[s_] == J1
        one.close()
        Jo, go, _ = oracle.value_and_grad(P, coefs[s_], [srcs[s_]], w.nsteps, w.dt,
                                          [obs[s_, :, : P.face_nodes(srcs[s_].face).size].cpu().numpy()])
        assert abs(J[s_] - Jo) <= 1e-12 * Jo
        assert rel_l2(g[s_].cpu().numpy(), go) <= 1e-12
    m.close()

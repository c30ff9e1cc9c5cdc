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
    from paper_1509_01399_gb300.serve import Request, ServingEngine
    reqs = _requests(12)
    eng = ServingEngine(workers=4)
    mix = eng.run([Request(i, w, t) for i, (w, t) in enumerate(reqs)])
    assert eng.max_in_flight >= 2, "requests should overlap on the device"
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
    eng = ServingEngine(hbm_budget=int(1.2 * biggest), workers=4)
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

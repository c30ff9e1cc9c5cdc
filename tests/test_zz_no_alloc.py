"""hyb_misfit_noalloc: the allocation-free misfit equals hyb_misfit.

Some callers cannot allocate device memory at the moment they need the data
misfit: code running while a stream is captured into a CUDA graph, loops in
which cudaMalloc's implicit device synchronisation is not allowed, or hosts
that serve all device memory from their own pool.  hyb_misfit_noalloc needs
no mesh: its partial sums live in a static device array shared by all calls.
Two calls in a row check that the array carries nothing from one call into
the next.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01399_gb300 import hyb
    return torch, hyb


def _face_dims(n, faces):
    out = []
    for f in faces:
        ax = f // 2
        p, q = [d for d in range(3) if d != ax]
        out.append((n[p], n[q]))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("weights", [0, 1])
def test_noalloc_misfit_matches_mesh_misfit(env, precision, weights):
    torch, H = env
    w = synth.small_problem(n=(11, 12, 13), fem=(3, 8), nsteps=50, omega=12.0, courant=0.8)
    srcs = [synth.Source(5, 12.0), synth.Source(1, 9.0)]
    m = H.HybMesh.from_workload(w, precision=precision)
    obs = m.forward(np.ones(m.n_unknown), srcs, w.nsteps, w.dt).clone()
    tr = m.forward(w.a_true(), srcs, w.nsteps, w.dt)
    J_ref, cot_ref = m.misfit(tr, obs, weights, want_cot=True)
    dims = _face_dims(w.n, [s.face for s in srcs])
    code = H.HYB_FP64 if precision == "fp64" else H.HYB_FP32
    J_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        cot = torch.full_like(tr, 7.0)
        J_dev.fill_(-1.0)
        H.hyb_misfit_noalloc(tr.data_ptr(), obs.data_ptr(), code, len(srcs), w.nsteps, m.obs_stride, dims,
                             w.dt, w.h, weights, J_dev.data_ptr(), cot.data_ptr(), stream)
        torch.cuda.synchronize()
        J = J_dev.item()
        assert J_ref > 0
        assert abs(J - J_ref) <= 1e-12 * J_ref
        assert torch.equal(cot, cot_ref)
    m.close()


def test_noalloc_rejects_traces_beyond_its_scratch(env):
    torch, H = env
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    J_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HybError) as e:
        H.hyb_misfit_noalloc(buf.data_ptr(), buf.data_ptr(), H.HYB_FP32, 1, 70_000_000, 1, [(1, 1)], 0.01, 0.1,
                             0, J_dev.data_ptr(), 0, 0)
    assert e.value.status == H.HYB_ERR_ARG
    assert "exceeds" in H.hyb_last_error()
    # sizes whose product overflows 64 bits, or whose step count overflows
    # 32 bits when one is added, are refused the same way
    for n_src, nsteps, stride in ((1, 2 ** 31 - 1, 1), (16, 2 ** 31 - 2, 2 ** 31 - 1)):
        with pytest.raises(H.HybError) as e:
            H.hyb_misfit_noalloc(buf.data_ptr(), buf.data_ptr(), H.HYB_FP32, n_src, nsteps, stride,
                                 [(1, 1)] * n_src, 0.01, 0.1, 0, J_dev.data_ptr(), 0, 0)
        assert e.value.status == H.HYB_ERR_ARG

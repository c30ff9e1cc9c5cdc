"""Differentiation form: torch.autograd through the forward solve, backward by
the hand-written discrete adjoint with checkpoint/recompute."""
import numpy as np
import pytest

import oracle
import synth
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_hyb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01399_gb300 import autograd, hyb
    return torch, hyb, autograd


def _loss(torch, autograd, mesh, sigma, srcs, w, obs):
    tr = autograd.hyb_trace(sigma, mesh, srcs, w.nsteps, w.dt)
    d = tr - obs
    d[:, 0, :] = 0
    return 0.5 * (d * d).sum()


def test_autograd_matches_oracle_small(torch_hyb):
    torch, H, AG = torch_hyb
    w = synth.small_problem(n=11, fem=(2, 8), nsteps=60, omega=12.0, courant=0.8)
    w.ckpt_every = 7
    P = oracle.problem_from_workload(w)
    src = w.sources[0]
    obs_np = P.forward(np.ones(P.n_unknown), src, w.nsteps, w.dt)["trace"]
    m = H.HybMesh.from_workload(w, precision="fp64")
    obs = torch.zeros((1, w.nsteps + 1, m.obs_stride), dtype=torch.float64, device="cuda")
    obs[0, :, : obs_np.shape[1]] = torch.from_numpy(obs_np)
    sigma = torch.tensor(w.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    L = _loss(torch, AG, m, sigma, w.sources, w, obs)
    L.backward()
    J, g, _ = oracle.value_and_grad(P, w.a_true(), [src], w.nsteps, w.dt, [obs_np])
    assert abs(L.item() - J) <= 1e-12 * J
    assert rel_l2(sigma.grad.cpu().numpy(), g) <= 1e-12


def test_autograd_fd_97_checkpointed(torch_hyb):
    """97^3 lattice (FEM 49^3), 1200 steps, checkpoints every 50 steps:
    the autograd gradient against central finite differences (eps = 1e-6,
    FP64) of the same loss on 32 random voxels."""
    torch, H, AG = torch_hyb
    w = synth.autograd_97()
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=50)
    srcs = w.sources
    obs = m.forward(np.ones(w.n_unknown), srcs, w.nsteps, w.dt).clone()
    sigma = torch.tensor(w.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    L = _loss(torch, AG, m, sigma, srcs, w, obs)
    L.backward()
    g = sigma.grad.cpu().numpy()
    rng = np.random.default_rng(4)
    # voxels near the inclusions carry the largest gradient; sample both kinds
    idx = np.concatenate([rng.choice(np.flatnonzero(w.sigma > 0), 16, replace=False),
                          rng.choice(w.n_unknown, 16, replace=False)])
    eps = 1e-6
    fd = []
    with torch.no_grad():
        for c in idx:
            vals = []
            for s in (+1, -1):
                sg = torch.tensor(w.sigma, dtype=torch.float64, device="cuda")
                sg[c] += s * eps
                tr = m.forward(1.0 + sg, srcs, w.nsteps, w.dt)
                d = tr - obs
                d[:, 0, :] = 0
                vals.append(0.5 * float((d * d).sum()))
            fd.append((vals[0] - vals[1]) / (2 * eps))
    fd = np.array(fd)
    err = np.abs(g[idx] - fd) / np.abs(fd).max()
    assert err.max() <= 1e-3, err.max()


def test_backward_requires_its_own_forward(torch_hyb):
    torch, H, AG = torch_hyb
    w = synth.small_problem(n=9, fem=(2, 6), nsteps=20, omega=12.0)
    m = H.HybMesh.from_workload(w)
    sigma = torch.tensor(w.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    tr = AG.hyb_trace(sigma, m, w.sources, w.nsteps, w.dt)
    AG.hyb_trace(sigma.detach(), m, w.sources, w.nsteps, w.dt)
    with pytest.raises(RuntimeError):
        tr.sum().backward()


def test_autograd_against_the_paper_gradient_97(torch_hyb):
    """The 97^3 autograd configuration (1200 steps, checkpoints every 50):
    the exact-adjoint gradient that autograd returns against the paper's
    Lagrangian gradient (Eq. (fdmschemeadjoint) with d_n lambda = 0,
    Eq. (gradient1) with the same time index).  Their difference comes from
    the absorbing terms the paper drops from its adjoint and from O(h, tau)
    discretisation; it is reported (relative L2, cosine), with only a loose
    bound on the angle."""
    torch, H, AG = torch_hyb
    w = synth.autograd_97()
    m = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=50)
    srcs = w.sources
    obs = m.forward(np.ones(w.n_unknown), srcs, w.nsteps, w.dt).clone()
    sigma = torch.tensor(w.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    L = _loss(torch, AG, m, sigma, srcs, w, obs)
    L.backward()
    g_exact = sigma.grad.clone()
    mp = H.HybMesh.from_workload(w, precision="fp64", ckpt_every=50, adjoint_mode=H.HYB_ADJ_PAPER)
    a = (1.0 + sigma.detach()).contiguous()
    tr = mp.forward(a, srcs, w.nsteps, w.dt)
    cot = tr - obs
    cot[:, 0, :] = 0
    mp.adjoint(cot)
    g_paper = mp.gradient(a, 0.0, 1.0)
    mp.sync()
    rel = float(torch.linalg.vector_norm(g_paper - g_exact) / torch.linalg.vector_norm(g_exact))
    cos = float(torch.dot(g_paper, g_exact) / (torch.linalg.vector_norm(g_paper) * torch.linalg.vector_norm(g_exact)))
    print(f"97^3 x 1200: paper-mode vs exact gradient: relative L2 {rel:.4e}, cosine {cos:.6f}")
    assert cos > 0.5

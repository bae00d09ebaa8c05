"""Differentiable cost on the GPU: forward and hand-written adjoint against the oracle's
cost and gradient (FP64: 1e-9 relative; FP32: 2e-3 of each gradient's norm), against
central finite differences through torch.autograd.gradcheck (FP64, tiny window), and on
the full 8-camera, 50-keyframe window."""
import numpy as np
import pytest

from oracle import ba
from paper_2506_04359_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rc(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_04359_gb300 import autograd
    return autograd


def tensors(p, xi, dtype, dev):
    import torch
    f = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)
    i = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.int32, device=dev)
    return (f(xi).requires_grad_(), f(p.poses0).requires_grad_(), f(p.lm0).requires_grad_(),
            f(p.rig.intr).requires_grad_(), f(p.rig.T_cb), i(p.obs_kf), i(p.obs_cam), i(p.obs_lm), f(p.obs_uv))


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name,kw", [("c2", dict(K=6, M=120, track=(2, 5), seed=41, outlier_frac=0.1)),
                                     ("c2", {})])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_cost_and_gradient_match_oracle(rc, cuda_device, name, kw, dtype):
    import torch
    p = synth.make_problem(name, **kw)
    rng = np.random.default_rng(7)
    xi = rng.normal(size=(p.K, 6)) * 0.01
    dt = getattr(torch, dtype)
    args = tensors(p, xi, dt, cuda_device)
    F = rc.reproj_cost(*args, p.huber_delta)
    F.backward()
    w = ba.Window.from_problem(p)
    Fo, go = ba.cost_grad(w, p.poses0, p.lm0, p.rig.intr, xi)
    tol_f, tol_g = (1e-11, 1e-9) if dtype == "float64" else (1e-4, 2e-3)
    assert abs(F.item() - Fo) <= tol_f * Fo, (F.item(), Fo)
    for t, key in zip(args[:4], ["xi", "T", "lm", "intr"]):
        e = rel_err(t.grad.double().cpu().numpy(), go[key])
        assert e <= tol_g, (key, e)


def test_gradcheck_fp64_tiny(rc, cuda_device):
    import torch
    p = synth.make_problem("c2", K=3, M=8, track=(2, 3), seed=43, outlier_frac=0.25)
    xi = np.random.default_rng(3).normal(size=(p.K, 6)) * 0.02
    args = tensors(p, xi, torch.float64, cuda_device)
    f = lambda x, P, L, I: rc.reproj_cost(x, P, L, I, *args[4:], p.huber_delta)
    assert torch.autograd.gradcheck(f, args[:4], eps=1e-6, atol=1e-6, rtol=1e-5)


def test_gradient_descent_step_reduces_cost(rc, cuda_device):
    """The adjoint gives a descent direction on the full window (torch optimiser loop)."""
    import torch
    p = synth.make_problem("c2")
    args = tensors(p, np.zeros((p.K, 6)), torch.float64, cuda_device)
    xi = args[0]
    F0 = rc.reproj_cost(*args, p.huber_delta)
    F0.backward()
    with torch.no_grad():
        step = -1e-4 * xi.grad / xi.grad.norm()
    F1 = rc.reproj_cost(step, *args[1:], p.huber_delta)
    assert F1.item() < F0.item()

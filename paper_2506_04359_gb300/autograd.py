"""ReprojCost: the robust reprojection objective of cuVSLAM Sec. 2.2 as a
torch.autograd.Function, forward and adjoint both in the CUDA library.

    F = 1/2 sum_n rho(|pi(T^cb_k Exp(xi_i) T^bw_i p_j) - o_n|^2)      (Huber rho)

Differentiable inputs: xi (K, 6) left tangent perturbations (translation first),
poses (K, 3, 4), landmarks (M, 3), intrinsics (C, 4).  All float tensors must be CUDA
tensors of one dtype (float64 or float32: the arithmetic runs in that type).  The
backward call recomputes the Jacobians (nothing but the inputs is saved), and runs on the
current torch stream.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import cvba

_DT = {torch.float64: 0, torch.float32: 1}


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _check(st: int, what: str):
    if st != 0:
        raise cvba.CvbaError(st, what)


class ReprojCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi, poses, landmarks, intr, T_cb, obs_kf, obs_cam, obs_lm, obs_uv, huber_delta=1.0,
                z_min=1e-3):
        dt = poses.dtype
        if dt not in _DT:
            raise TypeError("poses must be float64 or float32")
        fl = [t.contiguous() for t in (xi, poses, landmarks, intr, T_cb, obs_uv)]
        if any(t.dtype != dt or not t.is_cuda for t in fl):
            raise TypeError("all float inputs must be CUDA tensors of one dtype")
        ints = [t.contiguous().to(torch.int32) for t in (obs_kf, obs_cam, obs_lm)]
        K, M, Cn, N = poses.shape[0], landmarks.shape[0], intr.shape[0], obs_uv.shape[0]
        nbytes = cvba.lib.cvba_cost_workspace_bytes(N, K, Cn)
        work = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=poses.device)
        cost = torch.empty((), dtype=dt, device=poses.device)
        stream = torch.cuda.current_stream(poses.device).cuda_stream
        xi_, P, L, I, Tc, uv = fl
        _check(cvba.lib.cvba_cost_forward(_DT[dt], N, K, Cn, M, _ptr(I), _ptr(Tc), _ptr(xi_), _ptr(P), _ptr(L),
                                          _ptr(ints[0]), _ptr(ints[1]), _ptr(ints[2]), _ptr(uv), float(huber_delta),
                                          float(z_min), _ptr(cost), _ptr(work), nbytes, C.c_void_p(stream)),
               "cvba_cost_forward")
        ctx.save_for_backward(xi_, P, L, I, Tc, uv, *ints)
        ctx.consts = (float(huber_delta), float(z_min), nbytes)
        return cost

    @staticmethod
    def backward(ctx, grad):
        xi, P, L, I, Tc, uv, kf, cam, lm = ctx.saved_tensors
        hub, zmin, nbytes = ctx.consts
        dt = P.dtype
        K, M, Cn, N = P.shape[0], L.shape[0], I.shape[0], uv.shape[0]
        need = ctx.needs_input_grad
        g_xi = torch.empty_like(xi) if need[0] else None
        g_T = torch.empty_like(P) if need[1] else None
        g_L = torch.empty_like(L) if need[2] else None
        g_I = torch.empty_like(I) if need[3] else None
        work = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=P.device)
        g = grad.to(dt).contiguous().reshape(1)
        stream = torch.cuda.current_stream(P.device).cuda_stream
        _check(cvba.lib.cvba_cost_backward(_DT[dt], N, K, Cn, M, _ptr(I), _ptr(Tc), _ptr(xi), _ptr(P), _ptr(L),
                                           _ptr(kf), _ptr(cam), _ptr(lm), _ptr(uv), hub, zmin, _ptr(g), _ptr(g_xi),
                                           _ptr(g_T), _ptr(g_L), _ptr(g_I), _ptr(work), nbytes,
                                           C.c_void_p(stream)),
               "cvba_cost_backward")
        return g_xi, g_T, g_L, g_I, None, None, None, None, None, None, None


def reproj_cost(xi, poses, landmarks, intr, T_cb, obs_kf, obs_cam, obs_lm, obs_uv, huber_delta=1.0, z_min=1e-3):
    """Functional form of ReprojCost.apply."""
    return ReprojCost.apply(xi, poses, landmarks, intr, T_cb, obs_kf, obs_cam, obs_lm, obs_uv, huber_delta, z_min)

"""Nonlinear smoothing (ks_gauss_newton, Section 2's Gauss-Newton reduction to linear smoothing
problems) through the C ABI against the oracle's Levenberg-Marquardt iteration.

* The built-in pendulum: the same minimiser as the oracle (1e-8 relative in FP64; the FP32 +
  refinement inner solves converge to it as well, 1e-6), the same objective, both converged.
* A model supplied by the caller as a C callback (here written in Python with torch on the
  library's stream): a linear model, whose minimiser is the linear smoother's solution, checked
  against the oracle's linear smoother.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import gauss_newton as gn
from paper_2502_11686_gb300 import Smoother, inputs, native

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_pendulum(pp, precision):
    import torch
    K = torch.from_numpy(pp.K).cuda()
    C = torch.from_numpy(pp.C).cuda()
    o = torch.from_numpy(np.ascontiguousarray(pp.o.reshape(-1))).cuda()
    u = torch.from_numpy(pp.u0.copy()).cuda()
    model = native.ks_pendulum(pp.dt, pp.gravity, o.data_ptr())
    with Smoother(device=0, precision=precision) as sm:
        _, rep = native.ks_gauss_newton(sm.ctx, pp.k, 2, 1, native.pendulum_linearizer(), model,
                                        K, C, u)
    return u.cpu().numpy(), rep


@pytest.mark.parametrize("k", [2000, 100_000])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_pendulum_matches_oracle(k, precision):
    pp = inputs.pendulum_problem(k, seed=k)
    prob = gn.NonlinearProblem(k=k, model=gn.Pendulum(pp.dt, pp.gravity), K=pp.K, C=pp.C, o=pp.o)
    u_ref, rep_ref = gn.gauss_newton(prob, pp.u0)
    u, rep = _gpu_pendulum(pp, precision)
    assert rep_ref["converged"], rep_ref
    # FP64 stops on the same criteria as the oracle; with FP32 inner solves the last corrections
    # carry rounding noise, so the stop may instead come from the damping limit
    assert rep["converged"] or precision == "fp32_refine", rep
    tol = 1e-8 if precision == "fp64" else 1e-6
    assert _rel(u, u_ref) < tol
    assert abs(rep["objective"] - rep_ref["objective"]) <= 1e-9 * rep_ref["objective"]
    assert abs(rep["objective0"] - rep_ref["objective0"]) <= 1e-12 * rep_ref["objective0"]
    # the result is a real improvement over the initial guess
    assert np.sqrt(np.mean((u - pp.truth) ** 2)) < 0.5 * np.sqrt(np.mean((pp.u0 - pp.truth) ** 2))


class _Dev:
    """A raw device pointer seen by torch through the CUDA array interface."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": "<f8", "data": (ptr, False),
                                         "version": 3, "strides": None, "stream": None}


def test_callback_model_linear_reaches_linear_smoother():
    import torch
    k, n, m = 777, 4, 3
    rng = np.random.default_rng(7)
    A = 0.95 * np.linalg.qr(rng.normal(size=(n, n)))[0]
    B = rng.normal(size=(m, n))
    lin = inputs.random_problem(k, n, m, seed=8)
    lin.F = np.ascontiguousarray(np.broadcast_to(A, (k - 1, n, n)))
    lin.G = np.ascontiguousarray(np.broadcast_to(B, (k, m, n))).reshape(-1)
    ref = oracle.smooth(lin, covariances=False)["u"]
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ot = torch.from_numpy(lin.o.reshape(k, m)).cuda()

    def lin_fn(user, kk, nn, mm, up, J, e, Gj, r, stream):
        try:
            with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                uu = torch.as_tensor(_Dev(up, (kk, nn)), device="cuda")
                torch.as_tensor(_Dev(J, (kk - 1, nn, nn)), device="cuda").copy_(At.expand(kk - 1, nn, nn))
                torch.as_tensor(_Dev(e, (kk - 1, nn)), device="cuda").copy_(uu[:-1] @ At.T - uu[1:])
                torch.as_tensor(_Dev(Gj, (kk, mm, nn)), device="cuda").copy_(Bt.expand(kk, mm, nn))
                torch.as_tensor(_Dev(r, (kk, mm)), device="cuda").copy_(ot - uu @ Bt.T)
            return 0
        except Exception:   # noqa: BLE001  (a failure must reach the library as a status)
            return 1

    cb = native.LINEARIZE_FN(lin_fn)
    K = torch.from_numpy(lin.K).cuda()
    C = torch.from_numpy(lin.C.reshape(k, m, m)).cuda()
    u = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    with Smoother(device=0, precision="fp64") as sm:
        _, rep = native.ks_gauss_newton(sm.ctx, k, n, m, cb, None, K, C, u)
    assert rep["converged"]
    assert _rel(u.cpu().numpy(), ref) < 1e-9


def test_failing_callback_is_a_status():
    import torch
    cb = native.LINEARIZE_FN(lambda *a: 1)
    k, n, m = 10, 2, 1
    K = torch.eye(n, dtype=torch.float64, device="cuda").expand(k - 1, n, n).contiguous()
    C = torch.ones((k, 1, 1), dtype=torch.float64, device="cuda")
    u = torch.zeros((k, n), dtype=torch.float64, device="cuda")
    with Smoother(device=0, precision="fp64") as sm:
        st, _ = native.ks_gauss_newton(sm.ctx, k, n, m, cb, None, K, C, u, check=False)
    assert st == native.KS_ERR_ARG

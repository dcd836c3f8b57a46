"""Pins of the oracle's Gauss-Newton / Levenberg-Marquardt nonlinear smoother (Section 2) --
no GPU.

* A linear model (f(u) = A u, g(u) = B u): the iteration converges to the dense least-squares
  solution of the equivalent linear problem.
* The pendulum on a short horizon: the same minimiser as scipy.optimize.least_squares on the
  stacked whitened residual vector, which uses its own (finite-difference) Jacobians and its own
  trust-region algorithm.
* First-order optimality: along sampled coordinates the central-difference Newton step
  |dPhi/du| / (d^2 Phi/du^2) vanishes at the result.
* A planted mistake -- a wrong sign in the pendulum Jacobian -- is caught by the scipy pin.
"""
import numpy as np
import pytest

from dense_ref import dense_lstsq
from oracle import gauss_newton as gn
from paper_2502_11686_gb300 import inputs


class LinearModel:
    def __init__(self, A, B):
        self.A, self.B = A, B
        self.n, self.m = A.shape[0], B.shape[0]

    def f(self, u):
        return u @ self.A.T

    def df(self, u):
        return np.broadcast_to(self.A, u.shape[:-1] + self.A.shape).copy()

    def g(self, u):
        return u @ self.B.T

    def dg(self, u):
        return np.broadcast_to(self.B, u.shape[:-1] + self.B.shape).copy()


def _pendulum(k, seed=0):
    pp = inputs.pendulum_problem(k, seed=seed)
    prob = gn.NonlinearProblem(k=k, model=gn.Pendulum(pp.dt, pp.gravity), K=pp.K, C=pp.C, o=pp.o)
    return pp, prob


def _stacked_residual(prob):
    Lk = np.linalg.cholesky(prob.K)
    Lc = np.linalg.cholesky(prob.C)
    n = prob.model.n

    def res(x):
        u = x.reshape(prob.k, n)
        e = u[1:] - prob.model.f(u[:-1])
        r = prob.o - prob.model.g(u)
        we = np.linalg.solve(Lk, e[..., None])[..., 0]
        wr = np.linalg.solve(Lc, r[..., None])[..., 0]
        return np.concatenate([we.ravel(), wr.ravel()])
    return res


def test_linear_model_reaches_dense_least_squares():
    rng = np.random.default_rng(3)
    k, n, m = 9, 3, 2
    A = 0.9 * np.linalg.qr(rng.normal(size=(n, n)))[0]
    B = rng.normal(size=(m, n))
    lin = inputs.random_problem(k, n, m, seed=4)
    lin.F = np.ascontiguousarray(np.broadcast_to(A, (k - 1, n, n)))
    lin.G = np.ascontiguousarray(np.broadcast_to(B, (k, m, n))).reshape(-1)
    prob = gn.NonlinearProblem(k=k, model=LinearModel(A, B), K=lin.K, C=lin.C.reshape(k, m, m),
                               o=lin.o.reshape(k, m))
    u, rep = gn.gauss_newton(prob, np.zeros((k, n)))
    ref = dense_lstsq(lin)
    assert rep["converged"]
    assert np.linalg.norm(u - ref["u"]) <= 1e-9 * np.linalg.norm(ref["u"])
    assert abs(rep["objective"] - ref["resid2"]) <= 1e-9 * ref["resid2"]


def _scipy_minimiser(prob, u0):
    so = pytest.importorskip("scipy.optimize")
    sol = so.least_squares(_stacked_residual(prob), u0.ravel(), method="lm", xtol=1e-15,
                           ftol=1e-15, gtol=1e-15, max_nfev=20000)
    return sol.x.reshape(u0.shape)


@pytest.mark.parametrize("seed", [0, 1])
def test_pendulum_matches_scipy_least_squares(seed):
    pp, prob = _pendulum(40, seed)
    u, rep = gn.gauss_newton(prob, pp.u0)
    ref = _scipy_minimiser(prob, pp.u0)
    assert np.linalg.norm(u - ref) <= 1e-7 * np.linalg.norm(ref)
    assert rep["objective"] <= gn.objective(prob, ref) * (1 + 1e-10)


def test_gradient_vanishes_at_the_result():
    pp, prob = _pendulum(300, 5)
    u, _ = gn.gauss_newton(prob, pp.u0)
    phi0 = gn.objective(prob, u)
    rng = np.random.default_rng(0)
    h = 1e-6
    for idx in rng.choice(u.size, size=25, replace=False):
        e = np.zeros(u.size)
        e[idx] = h
        gp = gn.objective(prob, u + e.reshape(u.shape))
        gm = gn.objective(prob, u - e.reshape(u.shape))
        grad = (gp - gm) / (2 * h)
        curv = (gp - 2 * phi0 + gm) / h ** 2
        # the Newton step along this coordinate, |grad| / curvature, is the distance to the
        # minimum along it: measured at most ~1e-16 here, while a point 1e-4 away reads 1e-4
        assert curv > 0 and abs(grad) / curv <= 1e-10, (idx, grad, curv)


class WrongSignPendulum(gn.Pendulum):
    def df(self, u):
        J = super().df(u)
        J[..., 1, 0] = -J[..., 1, 0]
        return J


def test_planted_jacobian_mistake_is_caught():
    pp, prob = _pendulum(40, 0)
    bad = gn.NonlinearProblem(k=prob.k, model=WrongSignPendulum(pp.dt, pp.gravity), K=prob.K,
                              C=prob.C, o=prob.o)
    u, _ = gn.gauss_newton(bad, pp.u0, max_iter=50)
    ref = _scipy_minimiser(prob, pp.u0)
    assert np.linalg.norm(u - ref) > 1e-7 * np.linalg.norm(ref)

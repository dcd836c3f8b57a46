"""Nonlinear smoothing by Gauss-Newton / Levenberg-Marquardt -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and reference legs
may use this module; the product path never imports it.

Section 2 of Gargir & Toledo: when the evolution maps f_i and the observation maps g_i are
nonlinear, the minimiser of

    Phi(u) = sum_i || L_K,i^{-1} (u_{i+1} - f_i(u_i)) ||^2 + sum_i || L_C,i^{-1} (o_i - g_i(u_i)) ||^2

(here with H_i = I) is found by a Gauss-Newton-type iteration, each step of which is a LINEAR
smoothing problem whose matrices are the Jacobians F_i = df_i/du and G_i = dg_i/du at the
current iterate, "or Jacobians concatenated with a diagonal matrix" -- the Levenberg-Marquardt
damping rows sqrt(lambda) I.  Only the states of those linear problems are needed.

One iteration at the iterate u (steps in the order below):
  1. linearize: J_i = df_i(u_i), e_i = f_i(u_i) - u_{i+1}, Gj_i = dg_i(u_i), r_i = o_i - g_i(u_i);
  2. solve the linear smoothing problem for the correction d:
       d_{i+1} = J_i d_i + e_i + noise(K_i),   r_i = Gj_i d_i + noise(C_i),   0 = d_i + noise(I / lambda)
     (the last block is the damping, appended to every observation);
  3. stop if the correction is negligible, ||d|| <= xtol (||u|| + xtol);
  4. trial point u + d; accept it if Phi decreases (then lambda <- lambda / 3), otherwise
     reject it (lambda <- 4 lambda);
  5. stop after an accepted step whose decrease of Phi is at most ftol * Phi, or when
     lambda exceeds 1e16, or after max_iter iterations.
The linear solves use the oracle's sequential Paige-Saunders smoother (``oracle.smooth``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import smooth


@dataclass
class Pendulum:
    """The pendulum model (angle theta, angular velocity w), one symplectic Euler step of dt
    (explicit Euler would gain energy at every step):
        w' = w - g sin(theta) dt,   theta' = theta + w' dt;      observation sin(theta)."""
    dt: float = 0.01
    gravity: float = 9.81

    n = 2
    m = 1

    def f(self, u):
        th, w = u[..., 0], u[..., 1]
        w1 = w - self.gravity * np.sin(th) * self.dt
        return np.stack([th + w1 * self.dt, w1], axis=-1)

    def df(self, u):
        a = self.gravity * np.cos(u[..., 0]) * self.dt    # d(g sin(theta) dt) / d theta
        J = np.zeros(u.shape[:-1] + (2, 2))
        J[..., 0, 0] = 1.0 - a * self.dt
        J[..., 0, 1] = self.dt
        J[..., 1, 0] = -a
        J[..., 1, 1] = 1.0
        return J

    def g(self, u):
        return np.sin(u[..., :1])

    def dg(self, u):
        G = np.zeros(u.shape[:-1] + (1, 2))
        G[..., 0, 0] = np.cos(u[..., 0])
        return G


@dataclass
class NonlinearProblem:
    """k states of dimension n, observations o [k, m]; noise covariances K [k-1, n, n] and
    C [k, m, m]; the model supplies f, df, g, dg."""
    k: int
    model: object
    K: np.ndarray
    C: np.ndarray
    o: np.ndarray


def objective(prob, u):
    """Phi(u) with the Cholesky factors of K_i and C_i."""
    e = u[1:] - prob.model.f(u[:-1])
    r = prob.o - prob.model.g(u)
    we = np.linalg.solve(np.linalg.cholesky(prob.K), e[..., None])[..., 0]
    wr = np.linalg.solve(np.linalg.cholesky(prob.C), r[..., None])[..., 0]
    return float(np.sum(we * we) + np.sum(wr * wr))


class _Linear:
    """The linear smoothing problem of one iteration, in the layout ``oracle.smooth`` reads."""

    def __init__(self, prob, u, lam):
        k, n, m = prob.k, prob.model.n, prob.model.m
        mdl = prob.model
        self.k, self.n = k, n
        self.m = np.full(k, m + n, dtype=np.int32)
        self.F = np.ascontiguousarray(mdl.df(u[:-1]))
        self.H = np.ascontiguousarray(np.broadcast_to(np.eye(n), (k - 1, n, n)))
        self.c = np.ascontiguousarray(mdl.f(u[:-1]) - u[1:])
        self.K = np.ascontiguousarray(prob.K)
        G = np.zeros((k, m + n, n))
        G[:, :m, :] = mdl.dg(u)
        G[:, m:, :] = np.eye(n)
        self.G = G.reshape(-1)
        o = np.zeros((k, m + n))
        o[:, :m] = prob.o - mdl.g(u)
        self.o = o.reshape(-1)
        C = np.zeros((k, m + n, m + n))
        C[:, :m, :m] = prob.C
        C[:, m:, m:] = np.eye(n) / lam
        self.C = C.reshape(-1)


def gauss_newton(prob, u0, max_iter=50, lambda0=1e-3, ftol=1e-12, xtol=1e-10):
    """Levenberg-Marquardt iteration of the module docstring from u0 [k, n].
    Returns (u, report) with report = dict(iterations, accepted, objective0, objective, lambda,
    converged: stopped by ftol or xtol)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    lam = lambda0
    phi = objective(prob, u)
    rep = {"iterations": 0, "accepted": 0, "objective0": phi, "objective": phi, "lambda": lam,
           "converged": False}
    for it in range(max_iter):
        rep["iterations"] = it + 1
        d = smooth(_Linear(prob, u, lam), covariances=False)["u"]
        if np.linalg.norm(d) <= xtol * (np.linalg.norm(u) + xtol):
            rep["converged"] = True
            break
        trial = u + d
        phi_t = objective(prob, trial)
        if phi_t < phi:
            decrease = phi - phi_t
            u, phi = trial, phi_t
            lam = lam / 3.0
            rep["accepted"] += 1
            if decrease <= ftol * phi:
                rep["converged"] = True
                break
        else:
            lam = lam * 4.0
            if lam > 1e16:
                break
    rep["objective"] = phi
    rep["lambda"] = lam
    return u, rep

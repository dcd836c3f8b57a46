"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

* dense least squares of the stacked whitened system and the explicit inverse of
  (UA)^T (UA) on tiny problems (Section 2, eq. of the generalized least-squares estimator, and
  Section 4, cov(u_hat) = (R^T R)^{-1}), including the lag-one blocks;
* brute-force normal equations;
* the scalar random walk: closed-form steady-state smoothed variance q r / sqrt(q^2 + 4 q r),
  closed-form interior weights of the smoothed mean, and lag-one covariance;
* exact recovery of noise-free consistent data, constant state, k = 1 textbook least squares;
* the conventional Kalman/RTS smoother (Section 2.2) with a diffuse-equivalent start;
* invariants: zero gradient at the minimiser, minimal objective equals the accumulated
  residual of the factorization.
"""
import numpy as np
import pytest

import oracle
from dense_ref import dense_lstsq, gradient, normal_equations, objective, rts_smoother
from paper_2502_11686_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


TINY = [(k, n) for k in (1, 2, 3, 4, 5, 7, 8, 9) for n in (1, 2, 3, 4)]


@pytest.mark.parametrize("k,n", TINY)
def test_dense_lstsq_uniform_m(k, n):
    p = inputs.random_problem(k, n, n, seed=100 * k + n, with_c=True)
    ref = dense_lstsq(p)
    got = oracle.smooth(p, covariances=True, cross=True)
    assert rel(got["u"], ref["u"]) < 1e-11
    assert rel(got["cov"], ref["cov"]) < 1e-11
    if k > 1:
        assert rel(got["cross"], ref["cross"]) < 1e-11
    assert abs(got["resid2"] - ref["resid2"]) <= 1e-10 * max(1.0, ref["resid2"])


@pytest.mark.parametrize("k", [2, 3, 5, 8, 9, 12])
@pytest.mark.parametrize("pattern", ["gaps", "wide", "narrow"])
def test_dense_lstsq_ragged_m(k, pattern):
    n = 3
    rng = np.random.default_rng(k)
    if pattern == "gaps":      # some steps unobserved (m_i = 0), still full column rank
        m = np.where(rng.uniform(size=k) < 0.4, 0, n).astype(np.int32)
        m[0] = n
    elif pattern == "wide":    # m_i > n
        m = rng.integers(n, 2 * n + 3, size=k).astype(np.int32)
    else:                      # m_i < n on most steps
        m = rng.integers(1, n + 1, size=k).astype(np.int32)
        m[0] = n
    p = inputs.random_problem(k, n, m, seed=k + 17, with_c=True)
    ref = dense_lstsq(p)
    got = oracle.smooth(p, covariances=True, cross=True)
    assert rel(got["u"], ref["u"]) < 1e-10
    assert rel(got["cov"], ref["cov"]) < 1e-10
    assert abs(got["resid2"] - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])


def test_normal_equations_tiny():
    for seed, (k, n) in enumerate([(6, 2), (9, 3), (12, 4)]):
        p = inputs.random_problem(k, n, n, seed=seed, with_c=True)
        assert rel(oracle.smooth(p, covariances=False)["u"], normal_equations(p)) < 1e-10


def test_scalar_random_walk_closed_forms():
    """Interior of a long random walk observed in noise.

    Normal equations in the interior: (1 + 2 lam) x_i - lam (x_{i-1} + x_{i+1}) = o_i with
    lam = r / q, whose Green's function is A rho^|d| with rho + 1/rho = (1 + 2 lam) / lam and
    A = 1 / sqrt(1 + 4 lam).  Hence the smoothed mean is sum_d A rho^|d| o_{i+d}, the smoothed
    variance is r A = q r / sqrt(q^2 + 4 q r) (the RTS steady state), and the lag-one
    covariance is r A rho."""
    q, r, k = 0.5, 2.0, 801
    p = inputs.scalar_random_walk(k, q, r, seed=3)
    got = oracle.smooth(p, covariances=True, cross=True)
    lam = r / q
    rho = ((1 + 2 * lam) - np.sqrt(1 + 4 * lam)) / (2 * lam)
    A = 1.0 / np.sqrt(1 + 4 * lam)
    mid = k // 2
    d = np.arange(k) - mid
    mean = np.sum(A * rho ** np.abs(d) * p.o)
    assert abs(got["u"][mid, 0] - mean) < 1e-12 * max(1.0, abs(mean))
    ps = q * r / np.sqrt(q * q + 4 * q * r)
    assert abs(got["cov"][mid, 0, 0] - ps) < 1e-13
    assert abs(got["cross"][mid, 0, 0] - r * A * rho) < 1e-13


@pytest.mark.parametrize("k,n,m", [(1, 3, 5), (2, 2, 2), (17, 4, 4), (64, 6, 3), (301, 5, 5)])
def test_exact_recovery(k, n, m):
    p = inputs.consistent_problem(k, n, m, seed=k + n)
    got = oracle.smooth(p, covariances=False)
    assert rel(got["u"], p.truth) < 1e-10
    assert got["resid2"] < 1e-18 * max(1.0, float(np.sum(p.o ** 2)))


def test_constant_state():
    k, n, m = 40, 3, 2
    p = inputs.random_problem(k, n, m, seed=5)
    p.F = np.ascontiguousarray(np.broadcast_to(np.eye(n), (k - 1, n, n)))
    a = np.array([0.3, -1.2, 2.0])
    p.o = np.einsum("kij,j->ki", p.G.reshape(k, m, n), a).reshape(-1)
    got = oracle.smooth(p, covariances=False)
    assert np.max(np.abs(got["u"] - a[None, :])) < 1e-11


def test_single_state_textbook_lstsq():
    n, m = 4, 7
    p = inputs.random_problem(1, n, m, seed=11)
    G = p.G.reshape(m, n)
    Ci = np.linalg.inv(p.C.reshape(m, m))
    P = np.linalg.inv(G.T @ Ci @ G)
    u = P @ G.T @ Ci @ p.o
    got = oracle.smooth(p)
    assert rel(got["u"][0], u) < 1e-12
    assert rel(got["cov"][0], P) < 1e-12


@pytest.mark.parametrize("k,n", [(30, 2), (200, 4), (120, 6)])
def test_rts_smoother(k, n):
    p = inputs.random_problem(k, n, n, seed=k, f_scale=0.99, with_c=True)
    xs, Ps = rts_smoother(p)
    got = oracle.smooth(p)
    # The covariance-form filter starts from (G_0^T C_0^{-1} G_0)^{-1} and inverts the
    # innovation covariances, so it loses about cond(G_0)^2 * eps (cond ~ 250 here); the
    # orthogonal factorizations do not.  The tolerance is that of the RTS reference.
    assert rel(got["u"], xs) < 1e-7
    assert rel(got["cov"], Ps) < 1e-7


def test_cv_problem_against_rts_after_observable_start():
    """The constant-velocity workload observes 2 of 4 state coordinates per step, so the RTS
    start needs m_0 >= n; pin it instead by dense least squares on a short prefix problem."""
    p = inputs.cv_problem(k=12, seed=0)
    ref = dense_lstsq(p)
    got = oracle.smooth(p)
    assert rel(got["u"], ref["u"]) < 1e-10
    assert rel(got["cov"], ref["cov"]) < 1e-10


def test_invariants_moderate_size():
    p = inputs.random_problem(3000, 6, 6, seed=1, with_c=True)
    got = oracle.smooth(p, covariances=False)
    g = gradient(p, got["u"])
    assert np.max(np.abs(g)) < 1e-9
    obj = objective(p, got["u"])
    assert abs(obj - got["resid2"]) <= 1e-10 * obj


def test_not_spd_reports_step():
    p = inputs.random_problem(10, 3, 3, seed=2)
    p.K = p.K.copy()
    p.K[4] = -np.eye(3)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.smooth(p)
    assert ei.value.code == 2 and ei.value.info == 4


def test_unobservable_is_singular():
    p = inputs.random_problem(6, 3, 0, seed=2)   # no observation at all: rank deficient
    with pytest.raises(oracle.OracleError) as ei:
        oracle.smooth(p)
    assert ei.value.code == 3

"""Parity of the register-column level and whitening kernels (state dimensions 12, 16, 24, 32, 48,
64) with the oracle, and with the column-owner kernels they replace (KS_NO_MED=1 selects the
latter).

The lengths give levels of odd and even width (the three-block tail of Section 3), ragged
observation counts (including steps without observations) run through the same kernels, and the
residual (the discarded rows) must match too.  Levels run in FP64 for n <= 32 and whitening for
n <= 48 (larger n fall back to the column-owner kernels, which the same test checks); FP32 +
refinement for all six.  Steps with more observations than the state dimension take the
column-owner whitening.
"""
import numpy as np
import pytest

import oracle
from paper_2502_11686_gb300 import Smoother, inputs, problem_arrays

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_blocks(c, ref):
    num = np.linalg.norm((c - ref).reshape(len(ref), -1), axis=1)
    den = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    return float(np.max(num / den))


def run(sm, p):
    arr = problem_arrays(p, "cuda")
    u, h = sm.smooth(p.k, p.n, arr, keep=True)
    cov = sm.covariances(h, p.k, p.n, arr["F"]).cpu().numpy()
    r2 = sm.residual(h)
    sm.release(h)
    return u.cpu().numpy(), cov, r2


CASES = [(12, 203), (16, 96), (24, 77), (32, 45), (48, 23), (64, 13)]


@pytest.mark.parametrize("n,k", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_med_kernel_matches_oracle_and_column_owner(n, k, precision, monkeypatch):
    p = inputs.random_problem(k, n, n, seed=70 + n, with_c=True, f_scale=0.99)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision=precision) as sm:
        if n > sm.max_n:
            pytest.skip(f"n = {n} above this precision's limit {sm.max_n}")
        monkeypatch.setenv("KS_NO_MED", "0")
        u, cov, r2 = run(sm, p)
        monkeypatch.setenv("KS_NO_MED", "1")
        u0, cov0, r20 = run(sm, p)
    tol_u = 1e-10 if precision == "fp64" else 1e-6
    tol_c = 1e-10 if precision == "fp64" else 1e-5
    assert rel(u, ref["u"]) < tol_u
    assert rel_blocks(cov, ref["cov"]) < tol_c
    assert rel(u, u0) < tol_u
    assert rel_blocks(cov, cov0) < tol_c
    if precision == "fp64":
        assert abs(r2 - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])


@pytest.mark.parametrize("n,precision", [(12, "fp64"), (32, "fp64"), (48, "fp64"),
                                         (16, "fp32_refine"), (48, "fp32_refine")])
def test_med_kernel_ragged_observations(n, precision, monkeypatch):
    rng = np.random.default_rng(n)
    k = 150
    m = rng.integers(0, n + 1, size=k).astype(np.int32)
    m[0] = n
    m[5] = 0
    p = inputs.random_problem(k, n, m, seed=5 + n, with_c=False)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision=precision) as sm:
        monkeypatch.setenv("KS_NO_MED", "0")
        u, cov, r2 = run(sm, p)
        monkeypatch.setenv("KS_NO_MED", "1")
        u0, cov0, _ = run(sm, p)
    tol_u = 1e-10 if precision == "fp64" else 1e-6
    tol_c = 1e-10 if precision == "fp64" else 1e-5
    assert rel(u, ref["u"]) < tol_u
    assert rel_blocks(cov, ref["cov"]) < tol_c
    assert rel(u, u0) < tol_u
    assert rel_blocks(cov, cov0) < tol_c
    if precision == "fp64":
        assert abs(r2 - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_med_whitening_falls_back_for_wide_steps(precision):
    """Steps with m_i > n exceed the register-column whitening; the column-owner kernel runs."""
    n, k = 16, 90
    m = np.full(k, n // 2, dtype=np.int32)
    m[::7] = n + 5
    p = inputs.random_problem(k, n, m, seed=41, with_c=True)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision=precision) as sm:
        u, cov, r2 = run(sm, p)
    assert rel(u, ref["u"]) < (1e-10 if precision == "fp64" else 1e-6)
    assert rel_blocks(cov, ref["cov"]) < (1e-10 if precision == "fp64" else 1e-5)
    if precision == "fp64":
        assert abs(r2 - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])

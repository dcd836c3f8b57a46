"""Parity of the register-column level kernel (state dimensions 12, 16, 24, 32, 48, 64) with the
oracle, and with the column-owner level kernel it replaces (KS_NO_MED=1 selects the latter).

The lengths give levels of odd and even width (the three-block tail of Section 3), ragged
observation counts run through the same kernel, and the residual (the discarded rows) must match
too.  FP64 runs for n <= 32 (larger n have no FP64 build of this kernel and fall back to the
column-owner kernel, which is checked by the same test); FP32 + refinement for all six.
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
    tol_c = 1e-10 if precision == "fp64" else 1e-3
    assert rel(u, ref["u"]) < tol_u
    assert rel_blocks(cov, ref["cov"]) < tol_c
    assert rel(u, u0) < tol_u
    assert rel_blocks(cov, cov0) < tol_c
    if precision == "fp64":
        assert abs(r2 - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])


@pytest.mark.parametrize("n", [12, 32])
def test_med_kernel_ragged_observations(n):
    rng = np.random.default_rng(n)
    k = 150
    m = rng.integers(0, n + 1, size=k).astype(np.int32)
    m[0] = n
    p = inputs.random_problem(k, n, m, seed=5 + n, with_c=False)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision="fp64") as sm:
        u, cov, _ = run(sm, p)
    assert rel(u, ref["u"]) < 1e-10
    assert rel_blocks(cov, ref["cov"]) < 1e-10

"""State dimensions above 128 (up to 512; the paper's n = 500 regime, Section 5) against the
oracle through the C ABI: the level QRs with the panel in shared memory and the trailing update
in chunks, the whitening with its Cholesky factors in per-block global scratch, SelInv with
Rd^{-1} there too, and the wide warp kernels of back substitution and refinement.  Lengths with
odd level widths (the three-block tail), ragged observation counts including steps without
observations, FP64 (1e-10) and FP32 + refinement (states 1e-6; covariances bounded as in the
large-state tests).  States (global and per state), every covariance and lag-one block, and
the residual.
"""
import numpy as np
import pytest

import oracle
from paper_2502_11686_gb300 import Smoother, inputs, problem_arrays
from parity import TOL32_STATES, TOL64, check_blocks, check_states

pytestmark = pytest.mark.gpu

COV32 = 1e-4


def run(precision, p):
    with Smoother(device=0, precision=precision) as sm:
        assert sm.max_n >= 512
        arr = problem_arrays(p, "cuda")
        u, h = sm.smooth(p.k, p.n, arr, keep=True)
        cov, cross = sm.covariances(h, p.k, p.n, arr["F"], cross=True)
        r2 = sm.residual(h)
        sm.release(h)
    return u.cpu().numpy(), cov.cpu().numpy(), cross.cpu().numpy(), r2


@pytest.fixture(scope="module")
def cases():
    out = {}
    for n, k in [(160, 9), (256, 12), (500, 5), (512, 3)]:
        p = inputs.random_problem(k, n, n, seed=4000 + n + k, with_c=True, f_scale=0.995)
        out[(n, k)] = (p, oracle.smooth(p, cross=True))
    return out


@pytest.mark.parametrize("n,k", [(160, 9), (256, 12), (500, 5), (512, 3)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_huge_matches_oracle(cases, n, k, precision):
    p, ref = cases[(n, k)]
    u, cov, cross, r2 = run(precision, p)
    if precision == "fp64":
        check_states(u, ref["u"], TOL64)
        check_blocks(cov, ref["cov"], TOL64)
        check_blocks(cross, ref["cross"], TOL64, "cross")
        assert abs(r2 - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])
    else:
        check_states(u, ref["u"], TOL32_STATES)
        check_blocks(cov, ref["cov"], COV32)
        check_blocks(cross, ref["cross"], COV32, "cross")


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_huge_ragged_observations(precision):
    rng = np.random.default_rng(200)
    n, k = 200, 11
    m = rng.integers(0, n + 1, size=k).astype(np.int32)
    m[0] = n
    m[4] = 0
    p = inputs.random_problem(k, n, m, seed=201, with_c=True, f_scale=0.99)
    ref = oracle.smooth(p, cross=True)
    u, cov, cross, _ = run(precision, p)
    tol_u = TOL64 if precision == "fp64" else TOL32_STATES
    check_states(u, ref["u"], tol_u)
    check_blocks(cov, ref["cov"], TOL64 if precision == "fp64" else COV32)

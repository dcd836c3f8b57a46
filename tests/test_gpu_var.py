"""Variable state dimensions and rectangular H_i (Section 2) through the C ABI
(ks_smooth_var / ks_covariances_var) against the oracle's variable-dimension smoother, which
works on the ragged blocks directly (no padding).  Dimension increases (l_i < n_{i+1}),
decreases (l_i > n_{i+1}), ragged and missing observations; the small-state kernels (N <= 8),
the register-column ones (N = 16) and the column-owner ones (some m_i + N - n_i > N); FP64 and
FP32 + refinement; host and device arrays; lengths whose levels have odd widths.
Bounds as in parity.py."""
import numpy as np
import pytest

import oracle
from paper_2502_11686_gb300 import Smoother, inputs, native
from parity import TOL32_STATES, TOL64, check_states, rel_blocks

pytestmark = pytest.mark.gpu


def _compare(prob, got_u, got_cov, ref, tol_u, tol_c):
    uo = prob.u_offsets()
    # per-state check on the packed vectors (states of different sizes): pad to a common width
    nmax = int(prob.nd.max())
    U = np.zeros((prob.k, nmax))
    R = np.zeros((prob.k, nmax))
    for i in range(prob.k):
        U[i, :prob.nd[i]] = got_u[uo[i]:uo[i + 1]]
        R[i, :prob.nd[i]] = ref["u"][uo[i]:uo[i + 1]]
    check_states(U, R, tol_u)
    worst = max(rel_blocks(a[None], b[None]) for a, b in
                zip(prob.split_cov(got_cov), prob.split_cov(ref["cov"])))
    assert worst < tol_c, ("cov", worst, tol_c)


CASES = [
    (9, (3, 4, 6), True, "n"), (33, (3, 4, 6), True, "ragged"), (64, (2, 5), False, "gaps"),
    (257, (4, 6, 8), True, "n"), (1000, (3, 4, 6), True, "ragged"), (129, (12, 16), True, "n"),
    (300, (10, 16), True, "ragged"),
]


@pytest.mark.parametrize("k,ns,rect,mm", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_var_matches_oracle(k, ns, rect, mm, precision):
    p = inputs.var_problem(k, ns, seed=k + len(ns), rect=rect, m_mode=mm)
    ref = oracle.smooth_var(p)
    with Smoother(device=0, precision=precision) as sm:
        u, cov = sm.smooth_var(p, covariances=True)
    u, cov = u.cpu().numpy(), cov.cpu().numpy()
    if precision == "fp64":
        _compare(p, u, cov, ref, TOL64, TOL64)
    else:
        _compare(p, u, cov, ref, TOL32_STATES, 1e-4)


def test_var_host_and_device_arrays_agree():
    p = inputs.var_problem(100, (3, 5), seed=3, rect=True, m_mode="ragged")
    with Smoother(device=0, precision="fp64") as sm:
        a_u, a_c = sm.smooth_var(p, device=None, covariances=True)
        b_u, b_c = sm.smooth_var(p, covariances=True)
    assert np.array_equal(a_u, b_u.cpu().numpy())
    assert np.array_equal(a_c, b_c.cpu().numpy())


def test_var_unobservable_state_is_singular():
    p = inputs.VarProblem(k=3, nd=np.array([3, 3, 3], np.int32), l=np.array([1, 0], np.int32),
                          m=np.array([3, 3, 0], np.int32), F=np.ones(3), H=np.ones(3), c=None,
                          K=np.ones(1), G=np.ones(18), o=np.ones(6),
                          C=np.concatenate([np.eye(3).reshape(-1)] * 2))
    with Smoother(device=0, precision="fp64") as sm:
        with pytest.raises(native.KsError) as ei:
            sm.smooth_var(p, device=None)
    assert ei.value.status == native.KS_ERR_SINGULAR


def test_covariances_var_rejects_a_uniform_handle():
    p = inputs.random_problem(10, 3, 3, seed=1)
    from paper_2502_11686_gb300 import problem_arrays
    with Smoother(device=0, precision="fp64") as sm:
        u, h = sm.smooth(p.k, p.n, problem_arrays(p, "cuda"), keep=True)
        cov = np.zeros(p.k * 9)
        st = native.ks_covariances_var(sm.ctx, h, cov, check=False)
        sm.release(h)
    assert st == native.KS_ERR_ARG

"""Failure detection through the C ABI, in the forms that fault nothing on the GPU.

* Non-finite inputs: a NaN in K_i or C_i has no Cholesky factor (KS_ERR_NOT_SPD, info = i); a
  NaN in F_i, c_i, G_i, o_i or H_{i-1} is reported as KS_ERR_NONFINITE with info = the state
  whose equations hold it.  Checked on every kernel family: the small-state path (n = 4), the
  register-column path (n = 16), the column-owner path (n = 10), the large-state path (n = 80).
* A bounded device wait that runs out: with the test-only switch KS_TEST_STALL_TC=1 the
  tensor-core level kernel (FP32, n = 128) issues no MMA for its first chunk, so the bounded
  completion wait can only give up.  The call returns KS_ERR_TIMEOUT, the kernel still frees
  its tensor memory, and the same ctx then smooths the problem correctly.
Nothing here traps, faults or hangs: every wait is bounded and every failure is a status.
"""
import numpy as np
import pytest

import oracle
from paper_2502_11686_gb300 import Smoother, inputs, native, problem_arrays
from parity import TOL32_STATES, check_blocks, check_states

pytestmark = pytest.mark.gpu

FAMILIES = [(4, "fp64"), (16, "fp64"), (10, "fp64"), (80, "fp64"), (16, "fp32_refine")]


def _smooth_status(sm, p):
    arr = problem_arrays(p, "cuda")
    u = __import__("torch").empty((p.k, p.n), dtype=__import__("torch").float64, device="cuda")
    st, _, info = native.ks_smooth(sm.ctx, p.k, p.n, np.ascontiguousarray(p.m, dtype=np.int32),
                                   arr["F"], arr["H"], arr["c"], arr["K"], arr["G"], arr["o"],
                                   arr["C"], u, check=False)
    return st, info


@pytest.mark.parametrize("n,precision", FAMILIES)
@pytest.mark.parametrize("where", ["K", "C", "F", "H", "c", "G", "o"])
def test_nonfinite_input_is_reported_with_its_state(n, precision, where):
    k, i = 37, 13
    p = inputs.random_problem(k, n, n, seed=n + 7, with_c=True, f_scale=0.99)
    go, co = p.obs_offsets()
    for nm in ("F", "H", "c", "K", "G", "o", "C"):
        setattr(p, nm, getattr(p, nm).copy())
    if where == "K":
        p.K[i][1, 1] = np.nan
    elif where == "C":
        p.C[co[i] + n + 1] = np.nan
    elif where == "F":
        p.F[i][0, n - 1] = np.nan
    elif where == "H":
        p.H[i][n - 1, 0] = np.inf
    elif where == "c":
        p.c[i][n // 2] = np.nan
    elif where == "G":
        p.G[(go[i] + 1) * n + 2] = np.nan
    else:
        p.o[go[i] + n - 1] = -np.inf
    with Smoother(device=0, precision=precision) as sm:
        st, info = _smooth_status(sm, p)
        # the ctx stays usable: a clean problem right after
        clean = inputs.random_problem(k, n, n, seed=n + 8, f_scale=0.99)
        st2, _ = _smooth_status(sm, clean)
    if where in ("K", "C"):
        assert (st, info) == (native.KS_ERR_NOT_SPD, i)
    else:
        assert st == native.KS_ERR_NONFINITE
        assert info == (i + 1 if where == "H" else i)
    assert st2 == native.KS_OK


def test_bounded_wait_times_out_and_ctx_stays_usable(monkeypatch):
    k, n = 33, 128
    p = inputs.random_problem(k, n, n, seed=128, f_scale=0.99)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision="fp32_refine") as sm:
        monkeypatch.setenv("KS_TEST_STALL_TC", "1")
        st, info = _smooth_status(sm, p)
        assert st == native.KS_ERR_TIMEOUT, (st, native.ks_last_error(sm.ctx))
        monkeypatch.delenv("KS_TEST_STALL_TC")
        arr = problem_arrays(p, "cuda")
        u, h = sm.smooth(p.k, p.n, arr, keep=True)
        cov = sm.covariances(h, p.k, p.n, arr["F"]).cpu().numpy()
        sm.release(h)
    check_states(u.cpu().numpy(), ref["u"], TOL32_STATES)
    check_blocks(cov, ref["cov"], 1e-3)

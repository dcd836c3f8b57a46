"""ks_smooth_static, the entry point for callers that cannot allocate device memory.

Such callers (a plugin whose host application owns the device-memory budget, a real-time loop
that must not wait on cudaMalloc or on cudaFree's device synchronization) get all work memory
from one array built into libks.so.  These checks call it through the C ABI twice in a row --
with different problem sizes, so stale contents of the shared array would show -- and compare
each result with ks_smooth / ks_covariances on the same inputs, at the FP64 tolerance of the
other parity tests (1e-10 relative).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2502_11686_gb300 import Smoother, inputs, native, problem_arrays

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _reference(p):
    arr = problem_arrays(p, "cuda")
    with Smoother(device=0, precision="fp64") as sm:
        u, h = sm.smooth(p.k, p.n, arr, keep=True)
        cov = sm.covariances(h, p.k, p.n, arr["F"])
        sm.release(h)
    return u.cpu().numpy(), cov.cpu().numpy()


def _static(p, with_cov=True):
    import torch
    arr = problem_arrays(p, "cuda")
    u = torch.empty((p.k, p.n), dtype=torch.float64, device="cuda")
    cov = torch.empty((p.k, p.n, p.n), dtype=torch.float64, device="cuda") if with_cov else None
    stream = torch.cuda.current_stream().cuda_stream
    st, info, msg = native.ks_smooth_static(0, stream, p.k, p.n, int(p.m[0]), arr["F"], arr["H"],
                                            arr["c"], arr["K"], arr["G"], arr["o"], arr["C"], u,
                                            cov)
    assert st == native.KS_OK, (st, info, msg)
    return u.cpu().numpy(), (cov.cpu().numpy() if with_cov else None)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_two_calls_in_a_row_match_ks_smooth():
    problems = [inputs.cv_problem(k=1000, seed=0),                      # n=4, m=2
                inputs.random_problem(777, 6, 6, seed=3, with_c=True)]  # n=6, m=6, odd k
    for p in problems:
        u_ref, cov_ref = _reference(p)
        u, cov = _static(p)
        assert _rel(u, u_ref) < TOL
        blk = np.linalg.norm((cov - cov_ref).reshape(p.k, -1), axis=1) / \
            np.linalg.norm(cov_ref.reshape(p.k, -1), axis=1)
        assert blk.max() < TOL


def test_large_call_then_smaller_different_shape():
    """A large call fills most of the shared array; the smaller call that follows has another n
    and m, so it would read stale records of the first if any slot were not rewritten."""
    first = inputs.random_problem(3000, 6, 6, seed=11, with_c=True)
    second = inputs.random_problem(501, 3, 1, seed=12, with_c=True)
    _static(first)
    u_ref, cov_ref = _reference(second)
    u, cov = _static(second)
    assert _rel(u, u_ref) < TOL
    blk = np.linalg.norm((cov - cov_ref).reshape(second.k, -1), axis=1) / \
        np.linalg.norm(cov_ref.reshape(second.k, -1), axis=1)
    assert blk.max() < TOL
    # no observations at all: the states are not determined, and both entry points say so
    none = inputs.random_problem(64, 2, 0, seed=13)
    import torch
    arr = problem_arrays(none, "cuda")
    u0 = torch.empty((none.k, none.n), dtype=torch.float64, device="cuda")
    st, _, msg = native.ks_smooth_static(0, None, none.k, none.n, 0, arr["F"], arr["H"], None,
                                         arr["K"], None, None, None, u0, None)
    assert st == native.KS_ERR_SINGULAR, (st, msg)
    assert "singular" in msg
    with Smoother(device=0, precision="fp64") as sm:
        st2, _, _ = native.ks_smooth(sm.ctx, none.k, none.n, np.zeros(none.k, np.int32), arr["F"],
                                     arr["H"], None, arr["K"], None, None, None, u0, check=False)
    assert st2 == native.KS_ERR_SINGULAR


def test_states_only_and_size_limit():
    p = inputs.random_problem(2049, 3, 2, seed=5)
    u_ref, _ = _reference(p)
    u, _ = _static(p, with_cov=False)
    assert _rel(u, u_ref) < TOL
    import torch
    big = 10_000_000
    u = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    st, _, msg = native.ks_smooth_static(0, None, big, 6, 6, u, u, None, u, u, u, u, u, None)
    assert st == native.KS_ERR_ARG and "static scratch" in msg
    # a k whose byte count would overflow 64 bits is refused before any size arithmetic
    st, _, msg = native.ks_smooth_static(0, None, 1 << 61, 1, 1, u, u, None, u, u, u, u, u, None)
    assert st == native.KS_ERR_ARG and "static scratch" in msg

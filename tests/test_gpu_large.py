"""The large-state path (state dimensions above the shared-memory tiles, up to 128) against the
oracle, through the C ABI: states, covariances and residual, on lengths whose levels have odd
widths (the three-block tail of Section 3), ragged observation counts, the error report of a
non-SPD covariance, a batch mixing large and small problems, and a served request.
Tolerances as in the other parity tests (FP64 1e-10; FP32 + refinement states 1e-6).
In FP32 the trailing updates of the blocked QRs run on the tensor cores (3xTF32); KS_NO_TC=1
selects the CUDA-core updates, and both must agree with the oracle and with each other.
"""
import numpy as np
import pytest

import oracle
from paper_2502_11686_gb300 import Smoother, inputs, native, problem_arrays
from parity import TOL32_STATES, TOL64, check_blocks, check_states

# FP32 covariance bound of the large-state path: about ten times the worst block error measured
# at full size on GB300 (2.3e-6 at n = 128, k = 700).
COV32 = 3e-5

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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


@pytest.mark.parametrize("n,k", [(56, 11), (80, 9), (96, 14), (128, 5), (128, 12)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_large_matches_oracle(n, k, precision):
    p = inputs.random_problem(k, n, n, seed=300 + n + k, with_c=True, f_scale=0.99)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision=precision) as sm:
        assert sm.max_n >= 128
        u, cov, r2 = run(sm, p)
    if precision == "fp64":
        check_states(u, ref["u"], TOL64)
        check_blocks(cov, ref["cov"], TOL64)
        assert abs(r2 - ref["resid2"]) <= 1e-9 * max(1.0, ref["resid2"])
    else:
        check_states(u, ref["u"], TOL32_STATES)
        check_blocks(cov, ref["cov"], COV32)


@pytest.mark.parametrize("n,k,m", [(72, 13, 72), (128, 9, 128), (100, 16, 61)])
def test_large_tensor_core_updates_match_cuda_cores(n, k, m, monkeypatch):
    """Chunks of 16..128 columns (and narrower ones left to the CUDA cores), depths p = n and
    p = m < n (the whitening QR), levels of odd width."""
    p = inputs.random_problem(k, n, m, seed=900 + n, with_c=True, f_scale=0.99)
    ref = oracle.smooth(p)
    out = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("KS_NO_TC", flag)
        with Smoother(device=0, precision="fp32_refine") as sm:
            out[flag] = run(sm, p)
    for flag in ("0", "1"):
        u, cov, _ = out[flag]
        check_states(u, ref["u"], TOL32_STATES, f" KS_NO_TC={flag}")
        check_blocks(cov, ref["cov"], COV32)
    assert rel(out["0"][0], out["1"][0]) < 1e-6
    assert rel_blocks(out["0"][1], out["1"][1]) < COV32


def test_large_ragged_observations():
    rng = np.random.default_rng(8)
    n, k = 96, 21
    m = rng.integers(0, n + 1, size=k).astype(np.int32)
    m[0] = n
    m[5] = 0
    p = inputs.random_problem(k, n, m, seed=17, with_c=False)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision="fp64") as sm:
        u, cov, _ = run(sm, p)
    check_states(u, ref["u"], TOL64)
    check_blocks(cov, ref["cov"], TOL64)


def test_fp32_n64_full_observations():
    """n = 64, m = 64 in FP32: register-column levels with the large-state whitening."""
    p = inputs.random_problem(40, 64, 64, seed=64, f_scale=0.99)
    ref = oracle.smooth(p)
    with Smoother(device=0, precision="fp32_refine") as sm:
        u, cov, _ = run(sm, p)
    check_states(u, ref["u"], TOL32_STATES)
    check_blocks(cov, ref["cov"], COV32)


def test_large_not_spd_reports_step():
    p = inputs.random_problem(10, 80, 80, seed=3)
    p.K = p.K.copy()
    p.K[4] = -np.eye(80)
    with Smoother(device=0, precision="fp64") as sm:
        arr = problem_arrays(p, "cuda")
        with pytest.raises(native.KsError) as ei:
            sm.smooth(p.k, p.n, arr)
    assert ei.value.status == native.KS_ERR_NOT_SPD and ei.value.info == 4


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_large_in_a_batch(precision):
    import torch
    probs = [inputs.random_problem(k, n, n, seed=40 + i, f_scale=0.99)
             for i, (k, n) in enumerate([(13, 128), (200, 6), (9, 96), (33, 16)])]
    tol = 1e-10 if precision == "fp64" else 1e-6
    with Smoother(device=0, precision=precision) as sm:
        batch = []
        for p in probs:
            d = dict(problem_arrays(p, "cuda"), k=p.k, n=p.n,
                     m=np.ascontiguousarray(p.m, dtype=np.int32),
                     u_out=torch.zeros((p.k, p.n), dtype=torch.float64, device="cuda"),
                     cov_out=torch.zeros((p.k, p.n, p.n), dtype=torch.float64, device="cuda"))
            batch.append(d)
        native.ks_smooth_batch(sm.ctx, batch)
    for p, b in zip(probs, batch):
        ref = oracle.smooth(p)
        check_states(b["u_out"].cpu().numpy(), ref["u"], tol, f" k={p.k} n={p.n}")
        check_blocks(b["cov_out"].cpu().numpy(), ref["cov"], TOL64 if precision == "fp64" else COV32)


def test_large_served_request():
    import torch
    k, n = 300, 128
    with Smoother(device=0, precision="fp32_refine") as sm:
        srv = native.ks_server_create(sm.ctx)
        rid = native.ks_server_submit_synthetic(srv, k, n, n, 5, want_cov=True)
        assert native.ks_server_wait(srv, rid)["status"] == native.KS_OK
        u = torch.empty((k, n), dtype=torch.float64, device="cuda")
        cov = torch.empty((k, n, n), dtype=torch.float64, device="cuda")
        native.ks_server_result(srv, rid, u, cov)
        native.ks_server_release(srv, rid)
        native.ks_server_destroy(srv)
        F, H, K = (torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(3))
        G = torch.empty((n, n), dtype=torch.float64, device="cuda")
        C = torch.empty((n, n), dtype=torch.float64, device="cuda")
        o = torch.empty((k, n), dtype=torch.float64, device="cuda")
        native.ks_generate(sm.ctx, k, n, n, 5, 0.99, F, H, K, G, C, o)
        arr = {"m": np.full(k, n, np.int32), "F": F.expand(k - 1, n, n).contiguous(),
               "H": H.expand(k - 1, n, n).contiguous(), "K": K.expand(k - 1, n, n).contiguous(),
               "c": None, "G": G.expand(k, n, n).contiguous(), "o": o.contiguous(),
               "C": C.expand(k, n, n).contiguous()}
        u_ref, h = sm.smooth(k, n, arr, keep=True)
        cov_ref = sm.covariances(h, k, n, arr["F"])
        sm.release(h)
    assert rel(u.cpu().numpy(), u_ref.cpu().numpy()) < 1e-6
    assert rel_blocks(cov.cpu().numpy(), cov_ref.cpu().numpy()) < COV32

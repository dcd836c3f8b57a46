"""The serving loop (continuous batching) through the C ABI.

* Requests submitted in waves -- later ones arrive while earlier ones are on the GPU and share
  their launches -- give the same states and covariances as when each is smoothed alone with
  ks_smooth (1e-10 relative, FP64), and the oracle's.
* Covariance follow-ups on kept factors equal ks_covariances on the same problem.
* A memory budget smaller than the offered work makes requests wait for admission; all finish.
* Synthetic requests (inputs generated on the device at admission) equal ks_smooth on the
  generated inputs.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2502_11686_gb300 import Smoother, inputs, native, problem_arrays

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_blocks(c, ref):
    num = np.linalg.norm((c - ref).reshape(len(ref), -1), axis=1)
    den = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    return float(np.max(num / den))


def request(p, want_cov, device="cuda"):
    import torch
    arr = problem_arrays(p, device)
    u = torch.zeros((p.k, p.n), dtype=torch.float64, device=device)
    cov = torch.zeros((p.k, p.n, p.n), dtype=torch.float64, device=device) if want_cov else None
    d = dict(arr, k=p.k, n=p.n, u_out=u, cov_out=cov)
    d["m"] = np.ascontiguousarray(p.m, dtype=np.int32)
    return d


def alone(sm, p, want_cov):
    arr = problem_arrays(p, "cuda")
    u, h = sm.smooth(p.k, p.n, arr, keep=want_cov)
    cov = None
    if want_cov:
        cov = sm.covariances(h, p.k, p.n, arr["F"]).cpu().numpy()
        sm.release(h)
    return u.cpu().numpy(), cov


def problems():
    rng = np.random.default_rng(77)
    out = []
    for i, (k, n) in enumerate([(300, 3), (2500, 6), (64, 16), (1000, 4), (777, 6), (129, 12),
                                (3000, 2), (50, 8), (400, 16), (1500, 6), (9, 3), (2048, 5)]):
        m = n
        if i % 4 == 3:
            m = rng.integers(0, n + 2, size=k).astype(np.int32)
            m[0] = n
        out.append((inputs.random_problem(k, n, m, seed=3000 + i, with_c=(i % 2 == 0)), i % 3 == 0))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_each_result_same_alone_and_in_the_mix(precision):
    """Each request's result equals the same problem smoothed alone (and the oracle's), and the
    requests really ran together: some launches carried the work of several requests."""
    # A long request first: it is still working through its 17 levels when the waves arrive,
    # so the waves' n = 6 requests share its level and back-substitution launches (each at its
    # own recursion depth) whatever the speed of the ticks.
    probs = [(inputs.random_problem(200_000, 6, 6, seed=2999, with_c=True), False)] + problems()
    tol = 1e-10 if precision == "fp64" else 1e-6
    with Smoother(device=0, precision=precision) as sm:
        refs = [alone(sm, p, c) for p, c in probs]
        srv = native.ks_server_create(sm.ctx)
        reqs = [request(p, c) for p, c in probs]
        ids = [None] * len(reqs)

        def submit_waves():
            for i, r in enumerate(reqs):
                ids[i] = native.ks_server_submit(srv, r)
                if i % 3 == 2:
                    time.sleep(0.002)   # later waves arrive while earlier requests run

        t = threading.Thread(target=submit_waves)
        t.start()
        t.join()
        infos = [native.ks_server_wait(srv, rid) for rid in ids]
        stats = native.ks_server_stats(srv)
        native.ks_server_destroy(srv)
    assert all(i["status"] == native.KS_OK and i["done"] for i in infos)
    assert stats["completed"] == len(probs) and stats["ticks"] > 0
    assert stats["max_requests_per_launch"] >= 2 and stats["shared_launches"] > 0, stats
    for (p, want_cov), r, (u_ref, cov_ref) in zip(probs, reqs, refs):
        u = r["u_out"].cpu().numpy()
        assert rel(u, u_ref) < tol, (p.k, p.n)
        assert rel(u, oracle.smooth(p, covariances=False)["u"]) < tol
        if want_cov:
            assert rel_blocks(r["cov_out"].cpu().numpy(), cov_ref) < (1e-10 if precision == "fp64" else 1e-4)


def test_covariance_follow_up_on_kept_factor():
    p = inputs.random_problem(1200, 6, 6, seed=5)
    with Smoother(device=0, precision="fp64") as sm:
        _, cov_ref = alone(sm, p, True)
        srv = native.ks_server_create(sm.ctx, keep_factors=True)
        r = request(p, False)
        rid = native.ks_server_submit(srv, r)
        assert native.ks_server_wait(srv, rid)["status"] == native.KS_OK
        cov = np.zeros((p.k, p.n, p.n))
        fid = native.ks_server_covariances(srv, rid, cov)
        assert native.ks_server_wait(srv, fid)["status"] == native.KS_OK
        assert native.ks_server_release(srv, fid) == native.KS_OK
        assert native.ks_server_release(srv, rid) == native.KS_OK
        native.ks_server_destroy(srv)
    assert rel_blocks(cov, cov_ref) < 1e-10


def test_admission_waits_for_memory():
    probs = [(inputs.random_problem(3000, 6, 6, seed=40 + i), False) for i in range(8)]
    with Smoother(device=0, precision="fp64") as sm:
        refs = [alone(sm, p, False)[0] for p, _ in probs]
        srv = native.ks_server_create(sm.ctx, mem_budget=14 << 20)   # each request needs about 6.5 MB: two at a time
        reqs = [request(p, False) for p, _ in probs]
        ids = [native.ks_server_submit(srv, r) for r in reqs]
        queued_seen = native.ks_server_stats(srv)["queued"]
        infos = [native.ks_server_wait(srv, rid) for rid in ids]
        big = inputs.random_problem(200_000, 6, 6, seed=1)
        rb = request(big, False)
        bid = native.ks_server_submit(srv, rb)
        binfo = native.ks_server_wait(srv, bid)
        native.ks_server_destroy(srv)
    assert all(i["status"] == native.KS_OK for i in infos)
    assert queued_seen >= 1
    assert max(i["queue_ms"] for i in infos) > 0.0
    for r, u_ref in zip(reqs, refs):
        assert rel(r["u_out"].cpu().numpy(), u_ref) < 1e-10
    assert binfo["status"] == native.KS_ERR_OOM   # larger than the whole budget


def test_follow_up_not_blocked_by_a_waiting_request():
    """A covariance follow-up is admitted ahead of an earlier request that waits for memory held
    by the follow-up's own kept factor (admitting in arrival order alone would wait forever)."""
    pa = inputs.random_problem(3000, 6, 6, seed=61)
    pb = inputs.random_problem(4500, 6, 6, seed=62)
    with Smoother(device=0, precision="fp64") as sm:
        ua_ref, cov_ref = alone(sm, pa, True)
        ub_ref = alone(sm, pb, False)[0]
        probe = native.ks_server_create(sm.ctx, keep_factors=True)
        sizes = []
        for p in (pa, pb):
            rid = native.ks_server_submit(probe, request(p, False))
            assert native.ks_server_wait(probe, rid, 60_000.0)["status"] == native.KS_OK
            sizes.append(native.ks_server_stats(probe)["bytes_in_use"])
            native.ks_server_release(probe, rid)
        native.ks_server_destroy(probe)
        a, b = sizes
        budget = 2 * a + (1 << 19)
        assert b <= budget < a + b
        srv = native.ks_server_create(sm.ctx, mem_budget=budget, keep_factors=True)
        ra, rb = request(pa, False), request(pb, False)
        ida = native.ks_server_submit(srv, ra)
        assert native.ks_server_wait(srv, ida, 60_000.0)["status"] == native.KS_OK
        idb = native.ks_server_submit(srv, rb)            # waits: A's factor holds the memory
        cov = np.zeros((pa.k, pa.n, pa.n))
        fid = native.ks_server_covariances(srv, ida, cov)  # queued after B
        finfo = native.ks_server_wait(srv, fid, 60_000.0)
        assert finfo["done"] and finfo["status"] == native.KS_OK
        assert native.ks_server_release(srv, fid) == native.KS_OK
        assert native.ks_server_release(srv, ida) == native.KS_OK
        binfo = native.ks_server_wait(srv, idb, 60_000.0)
        native.ks_server_destroy(srv)
    assert binfo["done"] and binfo["status"] == native.KS_OK
    assert rel_blocks(cov, cov_ref) < 1e-10
    assert rel(ra["u_out"].cpu().numpy(), ua_ref) < 1e-10
    assert rel(rb["u_out"].cpu().numpy(), ub_ref) < 1e-10


def generated(ctx, k, n, m, seed):
    import torch
    dev = "cuda"
    F, H, K = (torch.empty((n, n), dtype=torch.float64, device=dev) for _ in range(3))
    G = torch.empty((m, n), dtype=torch.float64, device=dev)
    C = torch.empty((m, m), dtype=torch.float64, device=dev)
    o = torch.empty((k, m), dtype=torch.float64, device=dev)
    native.ks_generate(ctx, k, n, m, seed, 0.99, F, H, K, G, C, o)
    return F, H, K, G, C, o


def test_generator_statistics():
    import torch
    with Smoother(device=0, precision="fp64") as sm:
        F, H, K, G, C, o = generated(sm.ctx, 200_000, 24, 24, seed=9)
    F, K, C = F.cpu().numpy(), K.cpu().numpy(), C.cpu().numpy()
    assert np.allclose(F @ F.T, 0.99 ** 2 * np.eye(24), atol=1e-12)       # scaled orthogonal
    assert np.array_equal(H.cpu().numpy(), np.eye(24))
    assert np.allclose(K, K.T) and np.all(np.linalg.eigvalsh(K) > 0)
    assert np.all(np.linalg.eigvalsh(C) > 0)
    ov = o.cpu().numpy().ravel()
    assert abs(ov.mean()) < 0.005 and abs(ov.var() - 1.0) < 0.01       # N(0, 1)
    g = G.cpu().numpy().ravel()
    assert abs(g.var() * 24 - 1.0) < 0.3                                 # variance 1/n


@pytest.mark.parametrize("precision", ["fp64", "fp32_refine"])
def test_synthetic_requests_match_ks_smooth(precision):
    import torch
    specs = [(1000, 6, 6, 11), (333, 24, 24, 12), (2049, 4, 2, 13)]
    with Smoother(device=0, precision=precision) as sm:
        srv = native.ks_server_create(sm.ctx)
        ids = [native.ks_server_submit_synthetic(srv, k, n, m, seed, want_cov=True)
               for k, n, m, seed in specs]
        for rid, (k, n, m, seed) in zip(ids, specs):
            assert native.ks_server_wait(srv, rid)["status"] == native.KS_OK
            u = torch.empty((k, n), dtype=torch.float64, device="cuda")
            cov = torch.empty((k, n, n), dtype=torch.float64, device="cuda")
            native.ks_server_result(srv, rid, u, cov)
            native.ks_server_release(srv, rid)
            F, H, K, G, C, o = generated(sm.ctx, k, n, m, seed)
            arr = {"m": np.full(k, m, np.int32), "F": F.expand(k - 1, n, n).contiguous(),
                   "H": H.expand(k - 1, n, n).contiguous(), "K": K.expand(k - 1, n, n).contiguous(),
                   "c": None, "G": G.expand(k, m, n).contiguous(), "o": o.contiguous(),
                   "C": C.expand(k, m, m).contiguous()}
            u_ref, h = sm.smooth(k, n, arr, keep=True)
            cov_ref = sm.covariances(h, k, n, arr["F"])
            sm.release(h)
            tol = 1e-10 if precision == "fp64" else 1e-6
            assert rel(u.cpu().numpy(), u_ref.cpu().numpy()) < tol
            assert rel_blocks(cov.cpu().numpy(), cov_ref.cpu().numpy()) < (1e-10 if precision == "fp64" else 1e-3)
        native.ks_server_destroy(srv)


def test_per_step_generator_recipe_and_parity():
    """ks_generate_steps (the batched-benchmark inputs): F_i the same scaled orthogonal matrix at
    every step, H_i = I, independent SPD K_i and C_i per step, G ~ N(0, 1/n), o ~ N(0, 1); and
    the smoother on those very bytes matches the oracle."""
    import torch
    from inputs_helpers import as_problem
    k, n, m = 3000, 8, 4
    T = lambda *s: torch.empty(s, dtype=torch.float64, device="cuda")   # noqa: E731
    F, H, K, G, C, o = T(k - 1, n, n), T(k - 1, n, n), T(k - 1, n, n), T(k, m, n), T(k, m, m), T(k, m)
    with Smoother(device=0, precision="fp64") as sm:
        native.ks_generate_steps(sm.ctx, k, n, m, 77, 0.99, F, H, K, G, C, o)
        Fh, Kh, Ch = F.cpu().numpy(), K.cpu().numpy(), C.cpu().numpy()
        assert np.array_equal(Fh, np.broadcast_to(Fh[0], Fh.shape))
        assert np.allclose(Fh[0] @ Fh[0].T, 0.99 ** 2 * np.eye(n), atol=1e-12)
        assert np.array_equal(H.cpu().numpy(), np.broadcast_to(np.eye(n), (k - 1, n, n)))
        assert not np.array_equal(Kh[0], Kh[1]) and not np.array_equal(Ch[0], Ch[1])
        assert np.allclose(Kh, np.swapaxes(Kh, 1, 2)) and np.all(np.linalg.eigvalsh(Kh) > 0)
        assert np.all(np.linalg.eigvalsh(Ch) > 0)
        assert abs(G.var().item() * n - 1.0) < 0.05 and abs(o.var().item() - 1.0) < 0.05
        p = as_problem(k, n, m, F, H, K, G, C, o)
        arr = {nm: getattr(p, nm) for nm in ("m", "F", "H", "c", "K", "G", "o", "C")}
        u, h = sm.smooth(k, n, {x: (torch.from_numpy(v).cuda() if v is not None and x != "m" else v)
                                for x, v in arr.items()}, keep=True)
        cov = sm.covariances(h, k, n, F)
        sm.release(h)
    ref = oracle.smooth(p)
    assert rel(u.cpu().numpy(), ref["u"]) < 1e-10
    assert rel_blocks(cov.cpu().numpy(), ref["cov"]) < 1e-10

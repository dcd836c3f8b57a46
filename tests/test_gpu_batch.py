"""The batched form (ks_smooth_batch) against the oracle and against one-problem calls.

Each problem of a mixed batch -- different lengths, state dimensions on both kernel paths,
ragged observation counts, with and without covariances -- must give the oracle's states and
covariances (1e-10 relative in FP64, 1e-6 for FP32 + refinement states) and the same result
as when it is smoothed alone (same tolerance; the batched and one-problem launches may use
different kernels for the top levels).  A second batch of the same shape replays the captured
graph and must reproduce the first bitwise.
"""
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


def mixed_problems():
    rng = np.random.default_rng(2024)
    probs = []
    spec = [(1, 1), (2, 3), (17, 4), (100, 6), (257, 8), (1000, 4), (33, 12), (129, 16),
            (64, 6), (3, 2), (500, 3), (2049, 5), (31, 16), (9, 1)]
    for i, (k, n) in enumerate(spec):
        if i % 5 == 3:   # ragged, some steps with more rows than n -> column-owner path
            m = rng.integers(0, n + 3, size=k).astype(np.int32)
            m[0] = n
            m[-1] = n
        elif i % 5 == 4:
            m = np.where(rng.uniform(size=k) < 0.3, 0, n).astype(np.int32)
            m[0] = n
        else:
            m = n
        probs.append((inputs.random_problem(k, n, m, seed=500 + i, with_c=(i % 2 == 0)), i % 3 != 1))
    return probs


def as_batch(problems, device="cuda"):
    import torch
    out, arrays = [], []
    for p, want_cov in problems:
        arr = problem_arrays(p, device)
        if device is None:
            u = np.zeros((p.k, p.n))
            cov = np.zeros((p.k, p.n, p.n)) if want_cov else None
        else:
            u = torch.zeros((p.k, p.n), dtype=torch.float64, device=device)
            cov = torch.zeros((p.k, p.n, p.n), dtype=torch.float64, device=device) if want_cov else None
        d = dict(arr, k=p.k, n=p.n, u_out=u, cov_out=cov)
        d["m"] = np.ascontiguousarray(p.m, dtype=np.int32)
        out.append(d)
        arrays.append(arr)
    return out


def to_np(x):
    return None if x is None else (x if isinstance(x, np.ndarray) else x.cpu().numpy())


@pytest.fixture(scope="module")
def sm64():
    s = Smoother(device=0, precision="fp64")
    yield s
    s.close()


def test_batch_fp64_matches_oracle_alone_and_replay(sm64):
    problems = mixed_problems()
    batch = as_batch(problems)
    native.ks_smooth_batch(sm64.ctx, batch)          # first batch of this shape: eager (+ tuning)
    first = [(to_np(b["u_out"]).copy(), to_np(b["cov_out"])) for b in batch]
    for (p, want_cov), (u, cov) in zip(problems, first):
        ref = oracle.smooth(p, covariances=want_cov)
        assert rel(u, ref["u"]) < 1e-10, (p.name, p.k, p.n)
        if want_cov:
            assert rel_blocks(cov, ref["cov"]) < 1e-10, (p.name, p.k, p.n)
        arr = problem_arrays(p, "cuda")
        ua, h = sm64.smooth(p.k, p.n, arr, keep=want_cov)
        assert rel(u, ua.cpu().numpy()) < 1e-10
        if want_cov:
            ca = sm64.covariances(h, p.k, p.n, arr["F"] if arr["F"] is not None else arr["G"])
            sm64.release(h)
            assert rel_blocks(cov, ca.cpu().numpy()) < 1e-10
    # Same shape again: served by the captured graph.
    for b in batch:
        b["u_out"].zero_()
        if b["cov_out"] is not None:
            b["cov_out"].zero_()
    native.ks_smooth_batch(sm64.ctx, batch)
    for b, (u, cov) in zip(batch, first):
        assert np.array_equal(to_np(b["u_out"]), u)
        if cov is not None:
            assert np.array_equal(to_np(b["cov_out"]), cov)


def test_batch_host_pointers(sm64):
    problems = mixed_problems()[:6]
    batch = as_batch(problems, device=None)
    native.ks_smooth_batch(sm64.ctx, batch)
    for (p, want_cov), b in zip(problems, batch):
        ref = oracle.smooth(p, covariances=want_cov)
        assert rel(b["u_out"], ref["u"]) < 1e-10
        if want_cov:
            assert rel_blocks(b["cov_out"], ref["cov"]) < 1e-10


def test_batch_fp32_refine():
    problems = [(inputs.random_problem(k, n, m, seed=900 + k, f_scale=0.99), True)
                for k, n, m in [(100, 4, 2), (3000, 8, 8), (777, 16, 8), (2000, 6, 6), (64, 32, 32)]]
    with Smoother(device=0, precision="fp32_refine") as sm:
        batch = as_batch(problems)
        native.ks_smooth_batch(sm.ctx, batch)
        for (p, _), b in zip(problems, batch):
            ref = oracle.smooth(p)
            assert rel(to_np(b["u_out"]), ref["u"]) < 1e-6
            assert rel_blocks(to_np(b["cov_out"]), ref["cov"]) < 1e-5


def test_batch_reports_failing_problem(sm64):
    good = inputs.random_problem(50, 3, 3, seed=1)
    bad = inputs.random_problem(40, 3, 3, seed=2)
    bad.K = bad.K.copy()
    bad.K[7] = -np.eye(3)
    batch = as_batch([(good, False), (bad, False)])
    st, sts, infos = native.ks_smooth_batch(sm64.ctx, batch, check=False)
    assert st == native.KS_ERR_NOT_SPD
    assert sts == [native.KS_OK, native.KS_ERR_NOT_SPD] and infos[1] == 7
    assert rel(to_np(batch[0]["u_out"]), oracle.smooth(good, covariances=False)["u"]) < 1e-10


FAMILY = 64   # tuned value in the tune cache = family * FAMILY + blocks per SM


def _batch_with_cache(problems, path):
    o = native.ks_default_options()
    o.precision = native.KS_FP64
    cache = str(path).encode()
    o.tune_cache = cache
    ctx = native.ks_create(o)
    try:
        batch = as_batch(problems)
        native.ks_smooth_batch(ctx, batch)
        return [(to_np(b["u_out"]).copy(), to_np(b["cov_out"])) for b in batch]
    finally:
        native.ks_destroy(ctx)


def _register_column_problems():
    return [(inputs.random_problem(k, n, n, seed=700 + n, with_c=True, f_scale=0.99), True)
            for k, n in [(257, 12), (129, 16), (96, 32)]]


def test_batch_tuner_picks_grid_and_level_kernel(tmp_path):
    """The first batch of a new group tunes its level launch over the persistent grid and, for
    state dimensions with a register-column level kernel, over the kernel family; the choice
    is written to the tune cache as family * 64 + blocks per SM."""
    problems = _register_column_problems()
    path = tmp_path / "tune.txt"
    out = _batch_with_cache(problems, path)
    for (p, _), (u, cov) in zip(problems, out):
        ref = oracle.smooth(p, covariances=True)
        assert rel(u, ref["u"]) < 1e-10 and rel_blocks(cov, ref["cov"]) < 1e-10
    tuned = dict(line.split() for line in path.read_text().splitlines())
    for n in (12, 16, 32):
        v = int(tuned[f"f64:n{n}:g:m{n}"])
        assert v // FAMILY in (0, 1) and v % FAMILY in (1, 2, 4, 8, 16, 32), (n, v)


@pytest.mark.parametrize("family", [0, 1], ids=["register_column", "column_owner"])
def test_batch_level_kernel_family_from_cache(family, tmp_path):
    """Either level kernel family, forced through the tune cache, matches the oracle."""
    problems = _register_column_problems()
    path = tmp_path / "tune.txt"
    path.write_text("".join(f"f64:n{n}:g:m{n} {family * FAMILY + 8}\n" for n in (12, 16, 32)))
    out = _batch_with_cache(problems, path)
    for (p, _), (u, cov) in zip(problems, out):
        ref = oracle.smooth(p, covariances=True)
        assert rel(u, ref["u"]) < 1e-10, (family, p.n)
        assert rel_blocks(cov, ref["cov"]) < 1e-10, (family, p.n)

"""Pins of the oracle's variable-dimension smoother (per-step state dimensions n_i, evolution
equations with l_i rows and rectangular H_i; Section 2) -- no GPU.

* Dense least squares of the ragged stacked whitened system and the explicit inverse of
  (UA)^T (UA) on tiny problems: dimension increases (l_i < n_{i+1}), decreases and
  over-determined evolution rows (l_i > n_{i+1}), ragged and missing observations.
* The uniform special case (every n_i = l_i = n) equals the fixed-dimension oracle, which has
  its own pins.
* Planted mistakes in copies of the variable-dimension routine are caught by the dense pins.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from dense_ref import dense_lstsq_var
from paper_2502_11686_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "ks_oracle.c")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


CASES = [(k, ns, rect, mm) for k in (1, 2, 3, 5, 8, 11) for ns in ((2, 3), (1, 4), (3, 5, 2))
         for rect in (False, True) for mm in ("n", "ragged", "gaps")]


@pytest.mark.parametrize("k,ns,rect,mm", CASES)
def test_dense_lstsq_ragged_dimensions(k, ns, rect, mm):
    p = inputs.var_problem(k, ns, seed=k * 31 + len(ns) + 7 * rect, rect=rect, m_mode=mm)
    try:
        ref = dense_lstsq_var(p)
    except np.linalg.LinAlgError:
        pytest.skip("rank-deficient draw")
    A_rank_ok = np.all(np.isfinite(ref["cov"]))
    got = oracle.smooth_var(p, covariances=True)
    assert A_rank_ok
    assert rel(got["u"], ref["u"]) < 1e-10
    assert rel(got["cov"], ref["cov"]) < 1e-10
    assert abs(got["resid2"] - ref["resid2"]) <= 1e-10 * max(1.0, ref["resid2"])


@pytest.mark.parametrize("k,n", [(1, 3), (6, 2), (17, 4)])
def test_uniform_case_equals_fixed_dimension_oracle(k, n):
    p = inputs.random_problem(k, n, n, seed=k + n, with_c=True)
    vp = inputs.VarProblem(k=k, nd=np.full(k, n, np.int32), l=np.full(max(k - 1, 0), n, np.int32),
                           m=p.m, F=p.F.reshape(-1), H=p.H.reshape(-1), c=p.c.reshape(-1),
                           K=p.K.reshape(-1), G=p.G, o=p.o, C=p.C)
    a = oracle.smooth(p)
    b = oracle.smooth_var(vp)
    assert rel(b["u"], a["u"].reshape(-1)) < 1e-13
    assert rel(b["cov"], a["cov"].reshape(-1)) < 1e-13


def test_underdetermined_state_is_singular():
    """u_2 appears in no equation (evolution 1 has no rows and u_2 no observation), so the
    least-squares problem has no unique solution and the oracle reports a singular R."""
    p = inputs.VarProblem(k=3, nd=np.array([3, 3, 3], np.int32), l=np.array([1, 0], np.int32),
                          m=np.array([3, 3, 0], np.int32), F=np.ones(3), H=np.ones(3), c=None,
                          K=np.ones(1), G=np.ones(18), o=np.ones(6),
                          C=np.concatenate([np.eye(3).reshape(-1)] * 2))
    with pytest.raises(oracle.OracleError) as ei:
        oracle.smooth_var(p)
    assert ei.value.code == 3


VAR_MUTANTS = {
    "wrong F offset": ("fo += (int64_t)li * ni; ho += (int64_t)li * nj;",
                       "fo += (int64_t)li * nj; ho += (int64_t)li * nj;"),
    "H of the wrong block column": ("tmp[r * w + ni + q] = H[ho + (int64_t)r * nj + q];",
                                    "tmp[r * w + ni + q] = H[ho + (int64_t)q * li + r];"),
    "dropped coupling in back substitution": (
        "s -= Roff[ro[i] + (int64_t)r * nd[i + 1] + q] * u[uo[i + 1] + q];",
        "s -= 0.0 * Roff[ro[i] + (int64_t)r * nd[i + 1] + q] * u[uo[i + 1] + q];"),
    "transposed T in SelInv": ("for (int p = 0; p < nb; p++) s += Sx[r * nb + p] * T[q * nb + p];",
                               "for (int p = 0; p < nb; p++) s += Sx[r * nb + p] * T[p * nb + q];"),
    "observation offset of the wrong width": ("go += mi; gv += (int64_t)mi * nj;",
                                              "go += mi; gv += (int64_t)mi * ni;"),
}


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    c = tmp_path / f"v{abs(hash(name))}.c"
    so = tmp_path / f"v{abs(hash(name))}.so"
    c.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"])
    return oracle.load_library(str(so))


def _pins_pass(lib):
    for seed, ns, rect in ((3, (2, 3), True), (4, (3, 5, 2), True), (5, (2, 4), False)):
        p = inputs.var_problem(9, ns, seed=seed, rect=rect, m_mode="ragged")
        ref = dense_lstsq_var(p)
        try:
            got = oracle.smooth_var(p, lib=lib)
        except oracle.OracleError:
            return False
        for key in ("u", "cov"):
            if not np.all(np.isfinite(got[key])) or rel(got[key], ref[key]) > 1e-9:
                return False
    return True


def test_unmutated_var_copy_passes(tmp_path):
    assert _pins_pass(_compile(tmp_path, "identity", "#include <math.h>", "#include <math.h>"))


@pytest.mark.parametrize("name", sorted(VAR_MUTANTS))
def test_var_mutant_is_caught(tmp_path, name):
    old, new = VAR_MUTANTS[name]
    assert not _pins_pass(_compile(tmp_path, name, old, new))

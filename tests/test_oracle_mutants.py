"""Planted mistakes: each copy of the oracle source below carries one plausible error (a
dropped term, a wrong sign, a transposed operand, a wrong index).  The pins of
``test_oracle_pins.py`` must reject every copy; the mistakes live only in temporary copies
compiled on the CPU."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from dense_ref import dense_lstsq
from paper_2502_11686_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "ks_oracle.c")

MUTANTS = {
    "sign of F in the evolution rows": ("tmp[r * cols + cc] = -F[", "tmp[r * cols + cc] = F["),
    "transposed whitening factor": ("V[i * d + j] = Ci[j * d + i];", "V[i * d + j] = Ci[i * d + j];"),
    "dropped Householder rhs update": ("A[j * cols + c] -= s;", "A[j * cols + c] -= 0.0 * s;"),
    "wrong sign of the Householder tau": ("double tau = (beta - alpha) / beta;",
                                          "double tau = (alpha - beta) / beta;"),
    "dropped coupling in back substitution": (
        "s -= Roff[(size_t)i * n * n + r * n + cc] * u[(size_t)(i + 1) * n + cc];",
        "s -= 0.0 * Roff[(size_t)i * n * n + r * n + cc] * u[(size_t)(i + 1) * n + cc];"),
    "dropped update term in SelInv": ("Scur[r * n + cc] -= s;", "Scur[r * n + cc] -= 0.0 * s;"),
    "transposed T in SelInv": ("s += Sx[r * n + p] * T[cc * n + p];",
                               "s += Sx[r * n + p] * T[p * n + cc];"),
    "wrong packed observation offset": ("goff += mi; coff += (int64_t)mi * mi;",
                                        "goff += mi; coff += (int64_t)mi;"),
    "residual of dropped rows not accumulated": (
        "*res += carry[r * (n + 1) + n] * carry[r * (n + 1) + n];", "(void)res;"),
}


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new)
    c = tmp_path / f"{abs(hash(name))}.c"
    so = tmp_path / f"{abs(hash(name))}.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(c), "-lm"])
    return oracle.load_library(str(so))


def _pins_pass(lib):
    """A compact subset of the pins: dense least squares on ragged and uniform tiny problems."""
    cases = [inputs.random_problem(7, 3, 3, seed=1, with_c=True),
             inputs.random_problem(9, 2, np.array([2, 0, 3, 4, 1, 2, 5, 2, 2], np.int32), seed=2,
                                   with_c=True)]
    for p in cases:
        ref = dense_lstsq(p)
        try:
            got = oracle.smooth(p, covariances=True, lib=lib)
        except oracle.OracleError:
            return False
        for key in ("u", "cov"):
            if not np.all(np.isfinite(got[key])):
                return False
            if np.linalg.norm(got[key] - ref[key]) > 1e-9 * np.linalg.norm(ref[key]):
                return False
        if abs(got["resid2"] - ref["resid2"]) > 1e-9 * max(1.0, ref["resid2"]):
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_compile(tmp_path, "identity", "#include <math.h>", "#include <math.h>"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_compile(tmp_path, name, old, new))

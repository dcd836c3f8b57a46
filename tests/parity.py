"""Error measures of the parity tests (CUDA path vs the CPU oracle) and their bounds.

* States: the relative 2-norm error over the concatenated vector, and the largest per-state
  error ||u_i - u*_i|| / max(||u*_i||, 0.1 rms_j ||u*_j||) (the floor keeps a state that is
  near zero by chance -- a scalar state, say -- from dividing by ~0; one wrong state still
  stands out by orders of magnitude).  Both are asserted.
* Covariance blocks (and lag-one blocks): the largest per-block relative Frobenius error.

FP64 bounds: 1e-10 for states (both measures) and every covariance block.  FP32 + refinement:
states 1e-6 (global) and 1e-5 per state (one refinement step leaves an absolute error of a few
1e-8 in every state, so a small state reads ~1e-6 relative);
FP32 covariances carry about cond x 6e-8 and are bounded per workload at about ten times the
error measured on GB300.

With KS_PARITY_LOG set to a file name, every check appends one JSON line (test, measure, value,
bound) to it, which is how the measured errors quoted next to the bounds were collected.
"""
from __future__ import annotations

import json
import os

import numpy as np

TOL64 = 1e-10
TOL32_STATES = 1e-6
TOL32_MAX_STATE = 1e-5


def rel_states(u, ref) -> float:
    return float(np.linalg.norm(u - ref) / max(np.linalg.norm(ref), 1e-300))


def max_state_rel(u, ref) -> float:
    u = np.asarray(u).reshape(len(ref), -1)
    ref = np.asarray(ref).reshape(len(ref), -1)
    num = np.linalg.norm(u - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    floor = 0.1 * float(np.sqrt(np.mean(den ** 2)))
    return float(np.max(num / np.maximum(den, max(floor, 1e-300))))


def rel_blocks(c, ref) -> float:
    if len(ref) == 0:
        return 0.0
    num = np.linalg.norm((c - ref).reshape(len(ref), -1), axis=1)
    den = np.linalg.norm(ref.reshape(len(ref), -1), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def _log(measure, value, bound):
    path = os.environ.get("KS_PARITY_LOG")
    if not path:
        return
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    with open(path, "a") as fh:
        fh.write(json.dumps({"test": test, "measure": measure, "value": value,
                             "bound": bound}) + "\n")


def check_states(u, ref, tol, what=""):
    """Both state measures; tol is the global bound, and the per-state bound is tol too in
    FP64 and TOL32_MAX_STATE for the FP32 + refinement bound."""
    tol_s = TOL32_MAX_STATE if tol == TOL32_STATES else tol
    g, s = rel_states(u, ref), max_state_rel(u, ref)
    _log("states" + what, g, tol)
    _log("max_state" + what, s, tol_s)
    assert g < tol, ("states", what, g, tol)
    assert s < tol_s, ("max per-state", what, s, tol_s)


def check_blocks(c, ref, tol, what="cov"):
    e = rel_blocks(c, ref)
    _log(what, e, tol)
    assert e < tol, (what, e, tol)

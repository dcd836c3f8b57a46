"""GB300-native odd-even Kalman smoother (Gargir & Toledo, IPDPS 2025).

The compute path is libks.so (hand-written sm_103a CUDA kernels behind the C ABI of
``include/ks.h``).  ``native`` binds that ABI with the same names; :class:`Smoother` below only
moves arrays to / from the library (torch tensors for device memory, numpy for host data).
Importing this package does not load the library; the first call does, and fails loudly if it
is not built.
"""
from __future__ import annotations

from . import native
from .native import (KS_FP32_REFINE, KS_FP64, KsError, ks_covariances, ks_create,  # noqa: F401
                     ks_default_options, ks_destroy, ks_last_error, ks_max_m, ks_max_n,
                     ks_profile_read, ks_release, ks_residual, ks_smooth, ks_sync)

PRECISIONS = {"fp64": KS_FP64, "fp32_refine": KS_FP32_REFINE}


def problem_arrays(prob, device=None):
    """The arrays of an ``inputs.Problem`` as a dict, moved to ``device`` (torch) if given."""
    names = ("m", "F", "H", "c", "K", "G", "o", "C")
    out = {}
    for nm in names:
        a = getattr(prob, nm)
        if a is None or nm == "m" or device is None:
            out[nm] = a
        else:
            import torch
            out[nm] = torch.from_numpy(a).to(device)
    return out


class Smoother:
    """One ks_ctx: ``smooth`` returns the smoothed states (and optionally a handle for
    ``covariances``).  Device tensors in -> device tensors out; numpy in -> numpy out."""

    def __init__(self, device: int = 0, precision: str = "fp64", stream=None, sync: bool = True,
                 mem_budget: int = 0, profile: bool = False):
        o = ks_default_options()
        o.profile = 1 if profile else 0
        o.device = device
        o.precision = PRECISIONS[precision]
        o.stream = stream
        o.sync = 1 if sync else 0
        o.mem_budget = mem_budget
        self.device = device
        self.precision = precision
        self.ctx = ks_create(o)

    def close(self):
        if self.ctx is not None:
            ks_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def max_n(self) -> int:
        return ks_max_n(self.ctx)

    def _like(self, ref, shape):
        import numpy as np
        if hasattr(ref, "data_ptr"):
            import torch
            return torch.empty(shape, dtype=torch.float64, device=ref.device)
        return np.empty(shape, dtype=np.float64)

    def smooth(self, k, n, arrays: dict, keep: bool = False, out=None, reuse=None):
        """Smoothed states [k, n]; returns (u, handle) with handle None unless keep.
        ``reuse``: a handle whose memory the next factorization may take over."""
        import numpy as np
        m = np.ascontiguousarray(arrays["m"], dtype=np.int32)
        ref = arrays["F"] if arrays.get("F") is not None else arrays["G"]
        u = out if out is not None else self._like(ref, (k, n))
        _, h, _ = ks_smooth(self.ctx, k, n, m, arrays.get("F"), arrays.get("H"), arrays.get("c"),
                            arrays.get("K"), arrays.get("G"), arrays.get("o"), arrays.get("C"),
                            u, keep=keep, reuse=reuse)
        return u, h

    def covariances(self, h, k, n, like, cross: bool = False):
        cov = self._like(like, (k, n, n))
        crs = self._like(like, (max(k - 1, 1), n, n)) if cross else None
        ks_covariances(self.ctx, h, cov, crs)
        return (cov, crs[: k - 1]) if cross else cov

    def smooth_var(self, prob, device="cuda", covariances: bool = False):
        """A variable-dimension problem (``inputs.VarProblem``): packed states (and packed
        covariance blocks), as device tensors (device given) or numpy arrays (device None)."""
        import numpy as np
        arr = {nm: getattr(prob, nm) for nm in ("F", "H", "c", "K", "G", "o", "C")}
        tot_u = int(np.asarray(prob.nd, dtype=np.int64).sum())
        tot_s = int((np.asarray(prob.nd, dtype=np.int64) ** 2).sum())
        if device is not None:
            import torch
            arr = {nm: (torch.from_numpy(np.ascontiguousarray(a)).to(device) if a is not None
                        and a.size else None) for nm, a in arr.items()}
            u = torch.empty(tot_u, dtype=torch.float64, device=device)
            cov = torch.empty(max(tot_s, 1), dtype=torch.float64, device=device)
        else:
            arr = {nm: (np.ascontiguousarray(a) if a is not None and a.size else None)
                   for nm, a in arr.items()}
            u = np.empty(tot_u)
            cov = np.empty(max(tot_s, 1))
        _, h, _ = native.ks_smooth_var(self.ctx, prob.k, prob.nd, prob.l, prob.m, arr["F"],
                                       arr["H"], arr["c"], arr["K"], arr["G"], arr["o"],
                                       arr["C"], u, keep=covariances)
        if not covariances:
            return u
        native.ks_covariances_var(self.ctx, h, cov)
        ks_release(self.ctx, h)
        return u, cov

    def residual(self, h) -> float:
        return ks_residual(self.ctx, h)

    def release(self, h):
        ks_release(self.ctx, h)

    def profile(self, reset: bool = False) -> dict:
        return ks_profile_read(self.ctx, reset)

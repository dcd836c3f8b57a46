"""Seeded synthetic smoothing problems (host, FP64, numpy).

This module only draws inputs; it holds none of the smoother's arithmetic, so the CUDA path and
the CPU oracle can both consume the very same bytes.  Layout of a :class:`Problem`
(row-major, step-major):

* ``F, H, K``: ``[k-1, n, n]`` -- evolution equation i links state i to state i+1,
  ``H_i u_{i+1} = F_i u_i + c_i + eps_i`` with ``cov(eps_i) = K_i``;
* ``c``: ``[k-1, n]`` or ``None`` (all zero);
* ``m``: int32 ``[k]`` observation counts (0 allowed);
* ``G``: packed, observation i occupies ``m_i * n`` values (``o_i = G_i u_i + delta_i``);
* ``o``: packed ``sum(m_i)`` values;
* ``C``: packed, observation i occupies ``m_i * m_i`` values (``cov(delta_i) = C_i``).

Recipes (the paper's own benchmark problems are synthetic, Section 5: orthonormal F, H = I,
random observations):

* :func:`cv_problem` -- 2-D constant velocity, n=4, m=2, G ~ N(0,1), K=0.01 I, C=0.25 I,
  trajectory and observations simulated from the seed.
* :func:`random_problem` -- F = scale * (random orthogonal), one draw per problem stored for
  every step; H = I; G_i ~ N(0, 1/n) (variance 1/n) drawn per step; K_i, C_i = L L^T per step
  with L lower triangular, diagonal U[0.5, 1.5], off-diagonal N(0, 0.1^2) (std 0.1); c = 0;
  o ~ N(0, 1).
* :func:`scalar_random_walk` -- n = m = 1, F = H = G = 1, K = q, C = r.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    k: int
    n: int
    m: np.ndarray
    F: np.ndarray
    H: np.ndarray
    c: np.ndarray | None
    K: np.ndarray
    G: np.ndarray
    o: np.ndarray
    C: np.ndarray
    truth: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def steps(self) -> int:
        return self.k

    def input_bytes(self) -> int:
        arrs = [self.m, self.F, self.H, self.K, self.G, self.o, self.C]
        if self.c is not None:
            arrs.append(self.c)
        return int(sum(a.nbytes for a in arrs))

    def obs_offsets(self):
        """Packed offsets (G/o offset in rows, C offset in values) of every observation."""
        m = self.m.astype(np.int64)
        go = np.zeros(self.k + 1, dtype=np.int64)
        co = np.zeros(self.k + 1, dtype=np.int64)
        np.cumsum(m, out=go[1:])
        np.cumsum(m * m, out=co[1:])
        return go, co


def _spd_factor(rng, count, d, off_std=0.1):
    """Lower-triangular L with diagonal U[0.5,1.5] and off-diagonal N(0, off_std^2)."""
    L = np.tril(rng.normal(0.0, off_std, size=(count, d, d)), -1)
    idx = np.arange(d)
    L[:, idx, idx] = rng.uniform(0.5, 1.5, size=(count, d))
    return L


def random_spd(rng, count, d, off_std=0.1):
    L = _spd_factor(rng, count, d, off_std)
    return np.matmul(L, np.swapaxes(L, 1, 2))


def random_orthogonal(rng, n):
    q, r = np.linalg.qr(rng.normal(size=(n, n)))
    return q * np.sign(np.diag(r))[None, :]


def cv_problem(k: int = 1000, seed: int = 0, dt: float = 0.1, m: int = 2) -> Problem:
    """2-D constant-velocity model: u = (position, velocity), F = [[I, dt I], [0, I]]."""
    rng = np.random.default_rng(seed)
    n = 4
    I2 = np.eye(2)
    F1 = np.block([[I2, dt * I2], [np.zeros((2, 2)), I2]])
    Kc, Cc = 0.01, 0.25
    truth = np.zeros((k, n))
    truth[0] = rng.normal(size=n)
    for i in range(1, k):
        truth[i] = F1 @ truth[i - 1] + rng.normal(0.0, np.sqrt(Kc), size=n)
    G = rng.normal(size=(k, m, n))
    o = np.einsum("kij,kj->ki", G, truth) + rng.normal(0.0, np.sqrt(Cc), size=(k, m))
    return Problem(
        k=k, n=n, m=np.full(k, m, dtype=np.int32),
        F=np.ascontiguousarray(np.broadcast_to(F1, (k - 1, n, n))),
        H=np.ascontiguousarray(np.broadcast_to(np.eye(n), (k - 1, n, n))),
        c=None,
        K=np.ascontiguousarray(np.broadcast_to(Kc * np.eye(n), (k - 1, n, n))),
        G=G.reshape(-1), o=o.reshape(-1),
        C=np.ascontiguousarray(np.broadcast_to(Cc * np.eye(m), (k, m, m))).reshape(-1),
        truth=truth, name=f"cv k={k} n=4 m={m}")


def random_problem(k: int, n: int, m=None, seed: int = 0, f_scale: float = 0.99,
                   with_c: bool = False, g_var=None) -> Problem:
    """Random orthogonal dynamics (scaled), H = I, G_i ~ N(0, 1/n), SPD K_i and C_i per step.

    ``m`` is an int (uniform) or an int array of length k (0 allowed).
    """
    rng = np.random.default_rng(seed)
    m_arr = np.full(k, n if m is None else m, dtype=np.int32) if np.isscalar(m) or m is None \
        else np.asarray(m, dtype=np.int32)
    assert m_arr.shape == (k,)
    F1 = f_scale * random_orthogonal(rng, n)
    F = np.ascontiguousarray(np.broadcast_to(F1, (max(k - 1, 0), n, n)))
    H = np.ascontiguousarray(np.broadcast_to(np.eye(n), (max(k - 1, 0), n, n)))
    K = random_spd(rng, max(k - 1, 0), n)
    gstd = np.sqrt(1.0 / n if g_var is None else g_var)
    tot = int(m_arr.sum())
    G = rng.normal(0.0, gstd, size=tot * n)
    o = rng.normal(size=tot)
    if np.all(m_arr == m_arr[0]):
        mm = int(m_arr[0])
        C = random_spd(rng, k, mm).reshape(-1) if mm > 0 else np.zeros(0)
    else:
        C = np.concatenate([random_spd(rng, 1, int(mi)).reshape(-1) if mi > 0 else np.zeros(0)
                            for mi in m_arr]) if tot else np.zeros(0)
    c = rng.normal(size=(k - 1, n)) if with_c else None
    return Problem(k=k, n=n, m=m_arr, F=F, H=H, c=c, K=K, G=G, o=o, C=C,
                   name=f"random k={k} n={n} m={m if np.isscalar(m) or m is None else 'var'}")


def consistent_problem(k: int, n: int, m, seed: int = 0, f_scale: float = 0.99,
                       with_c: bool = True) -> Problem:
    """Noise-free data: o_i = G_i u_i and u_{i+1} = H^{-1}(F_i u_i + c_i) exactly (H = I), so
    the minimiser is the generating trajectory and the minimal objective is 0."""
    p = random_problem(k, n, m, seed=seed, f_scale=f_scale, with_c=with_c)
    rng = np.random.default_rng(seed + 7919)
    u = np.zeros((k, n))
    u[0] = rng.normal(size=n)
    for i in range(1, k):
        u[i] = p.F[i - 1] @ u[i - 1] + (p.c[i - 1] if p.c is not None else 0.0)
    go, _ = p.obs_offsets()
    o = np.zeros_like(p.o)
    for i in range(k):
        mi = int(p.m[i])
        if mi:
            o[go[i]:go[i] + mi] = p.G[go[i] * n:(go[i] + mi) * n].reshape(mi, n) @ u[i]
    p.o = o
    p.truth = u
    p.name = f"consistent k={k} n={n}"
    return p


def scalar_random_walk(k: int, q: float, r: float, seed: int = 0) -> Problem:
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.normal(0.0, np.sqrt(q), size=k))
    o = x + rng.normal(0.0, np.sqrt(r), size=k)
    return Problem(k=k, n=1, m=np.ones(k, dtype=np.int32),
                   F=np.ones((k - 1, 1, 1)), H=np.ones((k - 1, 1, 1)), c=None,
                   K=np.full((k - 1, 1, 1), q), G=np.ones(k), o=o, C=np.full(k, r),
                   truth=x, name=f"random walk q={q} r={r}")


def uneven_batch(nprob: int = 512, seed0: int = 0, k_lo: int = 100, k_hi: int = 20000,
                 ns=(4, 8, 16, 32)):
    """Independent problems, problem i drawn from seed seed0+i: k log-uniform in [k_lo, k_hi],
    n uniform over ``ns``, m = n/2 or n (equally likely)."""
    probs = []
    for i in range(nprob):
        k, n, m = uneven_shape(seed0 + i, k_lo, k_hi, ns)
        probs.append(random_problem(k, n, m, seed=seed0 + i, f_scale=0.99))
    return probs


def uneven_shape(seed: int, k_lo: int = 100, k_hi: int = 20000, ns=(4, 8, 16, 32)):
    """(k, n, m) of the uneven-batch problem drawn from ``seed``."""
    rng = np.random.default_rng(seed)
    k = int(round(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi)))))
    n = int(rng.choice(ns))
    m = n if rng.uniform() < 0.5 else n // 2
    return k, n, m


@dataclass
class VarProblem:
    """A problem whose state dimension varies from step to step (Section 2: u_i has n_i
    entries; evolution equation i has l_i rows, H_i is l_i x n_{i+1} and F_i is l_i x n_i).

    Packed row-major FP64 arrays in step order: F (l_i * n_i per equation), H (l_i * n_{i+1}),
    c (l_i, or None), K (l_i * l_i), G (m_i * n_i per observation), o (m_i), C (m_i * m_i).
    ``nd`` int32 [k] state dimensions, ``l`` int32 [k-1] evolution rows, ``m`` int32 [k]."""
    k: int
    nd: np.ndarray
    l: np.ndarray
    m: np.ndarray
    F: np.ndarray
    H: np.ndarray
    c: np.ndarray | None
    K: np.ndarray
    G: np.ndarray
    o: np.ndarray
    C: np.ndarray
    name: str = ""

    def u_offsets(self):
        off = np.zeros(self.k + 1, dtype=np.int64)
        np.cumsum(self.nd.astype(np.int64), out=off[1:])
        return off

    def cov_offsets(self):
        off = np.zeros(self.k + 1, dtype=np.int64)
        np.cumsum(self.nd.astype(np.int64) ** 2, out=off[1:])
        return off

    def split_states(self, u):
        off = self.u_offsets()
        return [u[off[i]:off[i + 1]] for i in range(self.k)]

    def split_cov(self, cov):
        off = self.cov_offsets()
        return [cov[off[i]:off[i + 1]].reshape(self.nd[i], self.nd[i]) for i in range(self.k)]


def var_problem(k: int, ns=(3, 4, 6), seed: int = 0, rect: bool = True, m_mode: str = "n",
                with_c: bool = True) -> VarProblem:
    """Random problem with state dimension n_i drawn from ``ns`` per step.

    l_i = n_{i+1} (square H_i) unless ``rect``, in which case l_i is drawn from
    [max(1, n_{i+1} - 1), n_{i+1} + 1]: a dimension change handled by a rectangular H_i.
    H_i = the l_i x n_{i+1} identity pattern plus N(0, 0.1^2) noise; F_i ~ N(0, 0.9^2 / n_i);
    K_i, C_i = L L^T as in :func:`random_problem`; G_i ~ N(0, 1/n_i); o ~ N(0, 1).
    ``m_mode``: "n" (m_i = n_i), "ragged" (m_i in {n_i - 1, n_i, n_i + 1}, m_0 = n_0), or
    "gaps" (m_i = n_i, but one step in five has no observation; m_0 = n_0)."""
    rng = np.random.default_rng(seed)
    nd = rng.choice(np.asarray(ns), size=k).astype(np.int32)
    if rect:
        l = np.array([rng.integers(max(1, nd[i + 1] - 1), nd[i + 1] + 2) for i in range(k - 1)],
                     dtype=np.int32)
    else:
        l = nd[1:].copy()
    if m_mode == "n":
        m = nd.copy()
    elif m_mode == "ragged":
        m = np.array([rng.integers(max(0, d - 1), d + 2) for d in nd], dtype=np.int32)
        m[0] = nd[0]
    else:
        m = nd.copy()
        m[1:][rng.uniform(size=k - 1) < 0.2] = 0
    F, H, c, K, G, o, C = [], [], [], [], [], [], []
    for i in range(k - 1):
        li, ni, nj = int(l[i]), int(nd[i]), int(nd[i + 1])
        F.append(rng.normal(0.0, 0.9 / np.sqrt(ni), size=(li, ni)).reshape(-1))
        H.append((np.eye(li, nj) + rng.normal(0.0, 0.1, size=(li, nj))).reshape(-1))
        K.append(random_spd(rng, 1, li).reshape(-1))
        if with_c:
            c.append(rng.normal(size=li))
    for i in range(k):
        mi, ni = int(m[i]), int(nd[i])
        if mi:
            G.append(rng.normal(0.0, np.sqrt(1.0 / ni), size=mi * ni))
            o.append(rng.normal(size=mi))
            C.append(random_spd(rng, 1, mi).reshape(-1))

    def cat(parts):
        return np.concatenate(parts) if parts else np.zeros(0)

    return VarProblem(k=k, nd=nd, l=l, m=m, F=cat(F), H=cat(H), c=cat(c) if with_c else None,
                      K=cat(K), G=cat(G), o=cat(o), C=cat(C),
                      name=f"var k={k} ns={tuple(ns)} rect={rect} m={m_mode}")


@dataclass
class PendulumProblem:
    """Noisy observations of a simulated pendulum (the nonlinear-smoothing workload).

    State u = (theta, w); the evolution is one symplectic Euler step, w' = w - g sin(theta) dt,
    theta' = theta + w' dt, plus noise with covariance K = q [[dt^3/3, dt^2/2], [dt^2/2, dt]];
    the observation sin(theta) plus noise with variance r.  ``K`` [k-1, 2, 2] and ``C`` [k, 1, 1] are stored per step,
    ``o`` [k, 1]; ``u0`` is an initial guess built from the observations alone (theta =
    arcsin of the clipped observation, w = its centred difference quotient)."""
    k: int
    dt: float
    gravity: float
    K: np.ndarray
    C: np.ndarray
    o: np.ndarray
    truth: np.ndarray
    u0: np.ndarray


def pendulum_problem(k: int, seed: int = 0, dt: float = 0.01, q: float = 0.01, r: float = 0.01,
                     gravity: float = 9.81, theta0: float = 1.2) -> PendulumProblem:
    rng = np.random.default_rng(seed)
    Q = q * np.array([[dt ** 3 / 3, dt ** 2 / 2], [dt ** 2 / 2, dt]])
    Lq = np.linalg.cholesky(Q)
    x = np.zeros((k, 2))
    x[0] = (theta0, 0.0)
    for i in range(1, k):
        th, w = x[i - 1]
        w1 = w - gravity * np.sin(th) * dt
        x[i] = (th + w1 * dt, w1)
        x[i] += Lq @ rng.normal(size=2)
    o = np.sin(x[:, :1]) + np.sqrt(r) * rng.normal(size=(k, 1))
    th = np.arcsin(np.clip(o[:, 0], -1.0, 1.0))
    w = np.gradient(th, dt)
    u0 = np.stack([th, w], axis=1)
    return PendulumProblem(k=k, dt=dt, gravity=gravity,
                           K=np.ascontiguousarray(np.broadcast_to(Q, (k - 1, 2, 2))),
                           C=np.full((k, 1, 1), r), o=o, truth=x, u0=u0)

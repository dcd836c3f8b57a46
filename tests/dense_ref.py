"""Independent numpy references used to pin the oracle (tests only).

Everything here is written from the definitions in Section 2 of the paper (the generalized
least-squares form of the smoother) with library primitives (Cholesky, triangular solve,
lstsq, inverse); none of it is shared with ``oracle/`` or with the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def dense_system(p):
    """Whitened dense U A and U b for a (tiny) problem.

    Block rows in time order: observation 0, evolution 0, observation 1, ...; U is the block
    diagonal of L^{-1} with cov = L L^T (a different whitening factor from the oracle's)."""
    k, n = p.k, p.n
    go, co = p.obs_offsets()
    rows_A, rows_b = [], []
    for i in range(k):
        mi = int(p.m[i])
        if mi:
            Gi = p.G[go[i] * n:(go[i] + mi) * n].reshape(mi, n)
            oi = p.o[go[i]:go[i] + mi]
            Ci = p.C[co[i]:co[i] + mi * mi].reshape(mi, mi)
            L = np.linalg.cholesky(Ci)
            blk = np.zeros((mi, k * n))
            blk[:, i * n:(i + 1) * n] = sla.solve_triangular(L, Gi, lower=True)
            rows_A.append(blk)
            rows_b.append(sla.solve_triangular(L, oi, lower=True))
        if i + 1 < k:
            L = np.linalg.cholesky(p.K[i])
            blk = np.zeros((n, k * n))
            blk[:, i * n:(i + 1) * n] = -sla.solve_triangular(L, p.F[i], lower=True)
            blk[:, (i + 1) * n:(i + 2) * n] = sla.solve_triangular(L, p.H[i], lower=True)
            rows_A.append(blk)
            ci = p.c[i] if p.c is not None else np.zeros(n)
            rows_b.append(sla.solve_triangular(L, ci, lower=True))
    return np.vstack(rows_A), np.concatenate(rows_b)


def dense_lstsq(p):
    """Smoothed states by dense least squares, covariances from the explicit inverse of
    (UA)^T (UA) (Section 4: cov(u_hat) = (R^T R)^{-1} = ((UA)^T UA)^{-1})."""
    A, b = dense_system(p)
    x, *_ = np.linalg.lstsq(A, b, rcond=None)
    k, n = p.k, p.n
    Sinv = np.linalg.inv(A.T @ A)
    cov = np.stack([Sinv[i * n:(i + 1) * n, i * n:(i + 1) * n] for i in range(k)])
    cross = np.stack([Sinv[i * n:(i + 1) * n, (i + 1) * n:(i + 2) * n] for i in range(k - 1)]) \
        if k > 1 else np.zeros((0, n, n))
    r = A @ x - b
    return {"u": x.reshape(k, n), "cov": cov, "cross": cross, "resid2": float(r @ r)}


def normal_equations(p):
    """Brute-force normal equations (UA)^T (UA) x = (UA)^T U b by a dense Cholesky solve."""
    A, b = dense_system(p)
    M = A.T @ A
    x = sla.cho_solve(sla.cho_factor(M), A.T @ b)
    return x.reshape(p.k, p.n)


def objective(p, u):
    """sum ||L_K^{-1}(H u_{i+1} - F u_i - c)||^2 + ||L_C^{-1}(o - G u)||^2, vectorised."""
    k, n = p.k, p.n
    tot = 0.0
    if k > 1:
        ci = p.c if p.c is not None else np.zeros((k - 1, n))
        e = np.einsum("kij,kj->ki", p.H, u[1:]) - np.einsum("kij,kj->ki", p.F, u[:-1]) - ci
        L = np.linalg.cholesky(p.K)
        w = np.linalg.solve(L, e[..., None])[..., 0]
        tot += float(np.sum(w * w))
    tot += float(np.sum(_obs_whitened_residual(p, u) ** 2))
    return tot


def _obs_whitened_residual(p, u):
    k, n = p.k, p.n
    go, co = p.obs_offsets()
    out = []
    if np.all(p.m == p.m[0]):
        mi = int(p.m[0])
        if mi == 0:
            return np.zeros(0)
        G = p.G.reshape(k, mi, n)
        C = p.C.reshape(k, mi, mi)
        r = p.o.reshape(k, mi) - np.einsum("kij,kj->ki", G, u)
        L = np.linalg.cholesky(C)
        return np.linalg.solve(L, r[..., None])[..., 0].reshape(-1)
    for i in range(k):
        mi = int(p.m[i])
        if mi:
            Gi = p.G[go[i] * n:(go[i] + mi) * n].reshape(mi, n)
            Ci = p.C[co[i]:co[i] + mi * mi].reshape(mi, mi)
            L = np.linalg.cholesky(Ci)
            out.append(sla.solve_triangular(L, p.o[go[i]:go[i] + mi] - Gi @ u[i], lower=True))
    return np.concatenate(out) if out else np.zeros(0)


def gradient(p, u):
    """Gradient of half the objective, (UA)^T U (A u - b), per state, vectorised (uniform m).

    Zero at the minimiser: this pins the states at any size."""
    k, n = p.k, p.n
    g = np.zeros((k, n))
    if k > 1:
        ci = p.c if p.c is not None else np.zeros((k - 1, n))
        e = np.einsum("kij,kj->ki", p.H, u[1:]) - np.einsum("kij,kj->ki", p.F, u[:-1]) - ci
        q = np.linalg.solve(p.K, e[..., None])[..., 0]          # K^{-1} e
        g[1:] += np.einsum("kji,kj->ki", p.H, q)
        g[:-1] -= np.einsum("kji,kj->ki", p.F, q)
    mi = int(p.m[0])
    assert np.all(p.m == mi)
    if mi:
        G = p.G.reshape(k, mi, n)
        C = p.C.reshape(k, mi, mi)
        r = np.einsum("kij,kj->ki", G, u) - p.o.reshape(k, mi)
        q = np.linalg.solve(C, r[..., None])[..., 0]
        g += np.einsum("kji,kj->ki", G, q)
    return g


def rts_smoother(p):
    """Conventional Kalman filter + RTS smoother (Section 2.2), H = I, every m_i >= n.

    The unknown initial expectation is handled by starting from the least-squares estimate of
    u_0 from observation 0 alone, which equals the diffuse formulation."""
    k, n = p.k, p.n
    go, co = p.obs_offsets()

    def obs(i):
        mi = int(p.m[i])
        return (p.G[go[i] * n:(go[i] + mi) * n].reshape(mi, n), p.o[go[i]:go[i] + mi],
                p.C[co[i]:co[i] + mi * mi].reshape(mi, mi))

    G0, o0, C0 = obs(0)
    Ci = np.linalg.inv(C0)
    P = np.linalg.inv(G0.T @ Ci @ G0)
    x = P @ G0.T @ Ci @ o0
    xf, Pf, xp, Pp = [x], [P], [None], [None]
    for i in range(1, k):
        Fm, Q = p.F[i - 1], p.K[i - 1]
        ci = p.c[i - 1] if p.c is not None else 0.0
        xpred = Fm @ xf[-1] + ci
        Ppred = Fm @ Pf[-1] @ Fm.T + Q
        Gi, oi, Cm = obs(i)
        S = Gi @ Ppred @ Gi.T + Cm
        Kg = Ppred @ Gi.T @ np.linalg.inv(S)
        xf.append(xpred + Kg @ (oi - Gi @ xpred))
        Pf.append((np.eye(n) - Kg @ Gi) @ Ppred)
        xp.append(xpred)
        Pp.append(Ppred)
    xs, Ps = [None] * k, [None] * k
    xs[-1], Ps[-1] = xf[-1], Pf[-1]
    for i in range(k - 2, -1, -1):
        J = Pf[i] @ p.F[i].T @ np.linalg.inv(Pp[i + 1])
        xs[i] = xf[i] + J @ (xs[i + 1] - xp[i + 1])
        Ps[i] = Pf[i] + J @ (Ps[i + 1] - Pp[i + 1]) @ J.T
    return np.array(xs), np.array(Ps)


def dense_system_var(p):
    """Whitened dense U A and U b of a problem with per-step state dimensions (``VarProblem``):
    block column i has n_i columns; evolution equation i has l_i rows,
    L_K^{-1} (H_i u_{i+1} - F_i u_i) = L_K^{-1} c_i with K_i = L_K L_K^T (Section 2)."""
    k = p.k
    uoff = p.u_offsets()
    N = int(uoff[-1])
    rows_A, rows_b = [], []
    fo = ho = eo = ko = 0
    go = gv = co = 0
    for i in range(k):
        ni, mi = int(p.nd[i]), int(p.m[i])
        if mi:
            Gi = p.G[gv:gv + mi * ni].reshape(mi, ni)
            oi = p.o[go:go + mi]
            Ci = p.C[co:co + mi * mi].reshape(mi, mi)
            L = np.linalg.cholesky(Ci)
            blk = np.zeros((mi, N))
            blk[:, uoff[i]:uoff[i + 1]] = sla.solve_triangular(L, Gi, lower=True)
            rows_A.append(blk)
            rows_b.append(sla.solve_triangular(L, oi, lower=True))
            go += mi
            gv += mi * ni
            co += mi * mi
        if i + 1 < k:
            li, nj = int(p.l[i]), int(p.nd[i + 1])
            if li:
                Fi = p.F[fo:fo + li * ni].reshape(li, ni)
                Hi = p.H[ho:ho + li * nj].reshape(li, nj)
                Ki = p.K[ko:ko + li * li].reshape(li, li)
                ci = p.c[eo:eo + li] if p.c is not None else np.zeros(li)
                L = np.linalg.cholesky(Ki)
                blk = np.zeros((li, N))
                blk[:, uoff[i]:uoff[i + 1]] = -sla.solve_triangular(L, Fi, lower=True)
                blk[:, uoff[i + 1]:uoff[i + 2]] = sla.solve_triangular(L, Hi, lower=True)
                rows_A.append(blk)
                rows_b.append(sla.solve_triangular(L, ci, lower=True))
            fo += li * ni
            ho += li * nj
            eo += li
            ko += li * li
    return np.vstack(rows_A), np.concatenate(rows_b)


def dense_lstsq_var(p):
    """States (packed) by dense least squares, covariance blocks (packed n_i x n_i) from the
    explicit inverse of (UA)^T UA, and the minimal objective."""
    A, b = dense_system_var(p)
    x, *_ = np.linalg.lstsq(A, b, rcond=None)
    Sinv = np.linalg.inv(A.T @ A)
    uoff = p.u_offsets()
    cov = np.concatenate([Sinv[uoff[i]:uoff[i + 1], uoff[i]:uoff[i + 1]].reshape(-1)
                          for i in range(p.k)])
    r = A @ x - b
    return {"u": x, "cov": cov, "resid2": float(r @ r)}

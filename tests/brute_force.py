"""Brute-force CONCORD minimiser for tiny p, independent of coordinate descent.

The objective (Eq. 1 of arXiv 2106.09382 divided by n, penalty on the S scale)

    f(Omega) = -sum_i log w_ii + 1/2 tr(Omega S Omega) + lam sum_{i<j} |w_ij|

is convex.  On a fixed sign pattern sigma_ij in {-1, 0, +1} of the
off-diagonal entries the penalty is linear, so the restricted problem is
smooth and strictly convex (S positive definite); it is solved here by damped
Newton with analytic derivatives.  The global minimiser is the restricted
solution whose signs agree with its pattern and which satisfies the full
subgradient conditions.  Enumerating all 3^(p(p-1)/2) patterns is feasible
for p <= 4.
"""
from __future__ import annotations

import itertools

import numpy as np


def _assemble(p, iu, ju, active, x):
    Om = np.zeros((p, p))
    Om[np.arange(p), np.arange(p)] = x[:p]
    for k, a in enumerate(active):
        Om[iu[a], ju[a]] = Om[ju[a], iu[a]] = x[p + k]
    return Om


def _restricted_newton(S, lam, iu, ju, active, signs, iters=200):
    p = S.shape[0]
    nv = p + len(active)
    # directions: E_i = e_i e_i^T (diagonal), E_ij = e_i e_j^T + e_j e_i^T
    dirs = []
    for i in range(p):
        E = np.zeros((p, p))
        E[i, i] = 1.0
        dirs.append(E)
    for a in active:
        E = np.zeros((p, p))
        E[iu[a], ju[a]] = E[ju[a], iu[a]] = 1.0
        dirs.append(E)
    lin = np.zeros(nv)
    for k, a in enumerate(active):
        lin[p + k] = lam * signs[a]
    H2 = np.empty((nv, nv))
    for a in range(nv):
        for b in range(nv):
            H2[a, b] = np.trace(dirs[a] @ S @ dirs[b])

    def f(x):
        if np.any(x[:p] <= 0):
            return np.inf
        Om = _assemble(p, iu, ju, active, x)
        return -np.log(x[:p]).sum() + 0.5 * np.trace(Om @ S @ Om) + lin @ x

    x = np.concatenate([1.0 / np.sqrt(np.diag(S)), np.zeros(len(active))])
    for _ in range(iters):
        Om = _assemble(p, iu, ju, active, x)
        M = Om @ S
        g = np.array([np.trace(E @ M) for E in dirs])  # = tr(E S Omega) sym. part
        g[:p] += -1.0 / x[:p]
        g += lin
        H = H2.copy()
        H[np.arange(p), np.arange(p)] += 1.0 / x[:p] ** 2
        step = np.linalg.solve(H, -g)
        t, f0 = 1.0, f(x)
        while f(x + t * step) > f0 + 1e-4 * t * (g @ step) and t > 1e-12:
            t *= 0.5
        x = x + t * step
        if np.abs(g).max() < 1e-14 or np.abs(t * step).max() < 1e-16:
            break
    return _assemble(p, iu, ju, active, x)


def objective(S, Om, lam):
    iu, ju = np.triu_indices(S.shape[0], 1)
    return (-np.log(np.diag(Om)).sum() + 0.5 * np.trace(Om @ S @ Om)
            + lam * np.abs(Om[iu, ju]).sum())


def minimise(S, lam, kkt_slack=1e-9):
    """Global minimiser of f for tiny p by sign-pattern enumeration."""
    S = np.asarray(S, dtype=np.float64)
    p = S.shape[0]
    iu, ju = np.triu_indices(p, 1)
    m = iu.size
    best, best_f = None, np.inf
    for signs in itertools.product((-1, 0, 1), repeat=m):
        active = [a for a in range(m) if signs[a] != 0]
        Om = _restricted_newton(S, lam, iu, ju, active, signs)
        ok = True
        W = Om @ S
        G = W + W.T
        for a in range(m):
            w = Om[iu[a], ju[a]]
            if signs[a] != 0:
                if w * signs[a] < -kkt_slack:
                    ok = False
                    break
            elif abs(G[iu[a], ju[a]]) > lam + kkt_slack:
                ok = False
                break
        if not ok:
            continue
        fv = objective(S, Om, lam)
        if fv < best_f:
            best, best_f = Om, fv
    return best, best_f

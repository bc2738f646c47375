"""Implicit differentiation of the CONCORD estimate: dense FP64 reference.

TEST INFRASTRUCTURE ONLY, like the rest of this package: plain numpy at
small p, imported by the tests and by nothing in the CUDA package.

What is differentiated.  Omega(S, lambda) minimises Eq. 1 in S units,
    f(Omega) = g(Omega) + lambda sum_{i<j} |w_ij|,
    g(Omega) = - sum_i log w_ii + 1/2 tr(Omega S Omega).
The variables are the diagonal entries w_ii and the pairs w_ij = w_ji
(i < j).  With W = Omega S the gradient of g is
    dg/dw_ii = W_ii - 1 / w_ii,      dg/dw_ij = W_ij + W_ji,
so the subgradient conditions of the minimiser (the KKT conditions that the
solver's stopping rule measures) read, on the active set A (the diagonal and
the pairs with w_ij != 0),
    F(Omega_A; S, lambda) = grad_A g + lambda sign(w_ij) = 0,
with every inactive pair held at zero.  Away from the threshold (every
inactive pair has |W_ij + W_ji| < lambda strictly) A and the signs are
locally constant, F is smooth, and the implicit-function theorem gives
    d Omega_A = - H^{-1} dF,      H = d F / d Omega_A,
H the Hessian of g on A: in the direction V (symmetric, supported on A)
    (H V)_ij = (V S + S V)_ij            (pairs),
    (H V)_ii = (V S)_ii + v_ii / w_ii^2  (diagonal).
H is symmetric positive semi-definite (g is convex, strictly so on the
diagonal).

Adjoint.  For a loss L(Omega) with gradient gL = dL/dOmega in the
full-matrix convention (every entry an independent variable), the gradient
on A is b_ii = gL_ii, b_ij = gL_ij + gL_ji.  Solve H a = b and put the
solution into the symmetric matrix Ahat (Ahat_ii = a_ii, Ahat_ij = Ahat_ji =
a_ij, zero off A).  Then
    dL/dlambda = - sum_{i<j in A} a_ij sign(w_ij),
    dL/dS      = - Omega Ahat             (full-matrix convention for S),
and, through S = Z^T Z / n with Z = X after the data preparation of Section
2.1 (columns centred, optionally scaled to unit 1/n variance),
    dL/dZ = Z (G + G^T) / n,   G = dL/dS,
followed by the preparation's own chain rule (see grad_X).

Parity pins (tests): H against second differences of the oracle's Eq. 1
objective at lambda = 0; dL/dlambda, dL/dS and dL/dX against central
differences of the oracle's solver; the diagonal regime lambda >= lambda_max
against its closed form (w_ii = s_ii^{-1/2}).
"""
import numpy as np


def active_set(Om):
    """Off-diagonal pairs (i < j) with w_ij != 0, as an (m, 2) int array in
    row-major order."""
    iu, ju = np.nonzero(np.triu(Om, 1))
    return np.stack([iu, ju], axis=1)


def _unit(p, pairs, c):
    """The symmetric direction of variable c (c < p: w_cc; else pair c - p)."""
    V = np.zeros((p, p))
    if c < p:
        V[c, c] = 1.0
    else:
        i, j = pairs[c - p]
        V[i, j] = V[j, i] = 1.0
    return V


def hvp(Om, S, V):
    """H V for a symmetric direction V supported on the active set of Om,
    returned as the symmetric matrix with (H V)_ii on the diagonal and
    (H V)_ij at both (i, j) and (j, i); zero off the active set."""
    p = Om.shape[0]
    VS = V @ S
    out = VS + VS.T
    out[np.diag_indices(p)] = np.diag(VS) + np.diag(V) / np.diag(Om) ** 2
    mask = (Om != 0)
    return np.where(mask, out, 0.0)


def hessian(Om, S):
    """H as a dense |A| x |A| matrix; variables ordered as the p diagonal
    entries, then the pairs of active_set(Om)."""
    p = Om.shape[0]
    pairs = active_set(Om)
    nA = p + len(pairs)
    H = np.empty((nA, nA))
    for c in range(nA):
        Y = hvp(Om, S, _unit(p, pairs, c))
        H[:p, c] = np.diag(Y)
        H[p:, c] = Y[pairs[:, 0], pairs[:, 1]]
    return H


def rhs(Om, gL):
    """b: the loss gradient on the active set (pairs carry gL_ij + gL_ji)."""
    pairs = active_set(Om)
    return np.concatenate([np.diag(gL), gL[pairs[:, 0], pairs[:, 1]] + gL[pairs[:, 1], pairs[:, 0]]])


def adjoint(Om, S, lam, gL):
    """dL/dlambda, dL/dS and the adjoint matrix Ahat for the loss gradient
    gL (p x p, full-matrix convention); H is solved directly."""
    p = Om.shape[0]
    pairs = active_set(Om)
    H = hessian(Om, S)
    b = rhs(Om, gL)
    a = np.linalg.solve(H, b)
    Ahat = np.diag(a[:p])
    Ahat[pairs[:, 0], pairs[:, 1]] = a[p:]
    Ahat[pairs[:, 1], pairs[:, 0]] = a[p:]
    sg = np.sign(Om[pairs[:, 0], pairs[:, 1]])
    return {"dlambda": -float(np.dot(a[p:], sg)), "dS": -Om @ Ahat, "Ahat": Ahat,
            "H": H, "b": b, "a": a}


def grad_Z(Z, dS):
    """dL/dZ for S = Z^T Z / n, given G = dL/dS (full-matrix convention)."""
    n = Z.shape[0]
    return Z @ (dS + dS.T) / n


def grad_X(X, prep, dZ):
    """Chain rule of the data preparation Z = (X - mean) * inv_scale:
    prep 0: Z = X; prep 1: columns centred; prep 2: centred and divided by the
    population standard deviation.  mean and the scale depend on X."""
    n = X.shape[0]
    if prep == 0:
        return dZ.copy()
    mu = X.mean(axis=0)
    Xc = X - mu
    if prep == 1:
        return dZ - dZ.mean(axis=0)
    sd = np.sqrt((Xc * Xc).sum(axis=0) / n)
    Z = Xc / sd
    return (dZ - dZ.mean(axis=0) - Z * (dZ * Z).mean(axis=0)) / sd


def heldout_loss(Om, S_val):
    """Held-out negative CONCORD pseudo-log-likelihood: the smooth part of
    Eq. 1 (S units) evaluated with the validation Gram S_val."""
    return float(-np.sum(np.log(np.diag(Om))) + 0.5 * np.trace(Om @ S_val @ Om))


def heldout_grad(Om, S_val):
    """Full-matrix gradient of heldout_loss at a symmetric Omega."""
    return -np.diag(1.0 / np.diag(Om)) + 0.5 * (S_val @ Om + Om @ S_val)


def hypergrad_descent(S, S_val, lam0, steps=20, lr=0.5, tol=1e-10, max_sweeps=20000):
    """Gradient descent on log lambda for the held-out loss: every step solves
    Eq. 1 at lambda (warm-started from the previous step), takes
    dL/dlambda from the adjoint and moves log lambda by -lr * lambda * dL/dlambda.
    Returns one (lambda, loss, dL/dlambda) row per step."""
    from . import solve
    log_lam = float(np.log(lam0))
    Om0 = None
    rows = []
    for _ in range(steps):
        lam = float(np.exp(log_lam))
        Om, _info = solve(S, lam, tol=tol, max_sweeps=max_sweeps, Om0=Om0)
        d = adjoint(Om, S, lam, heldout_grad(Om, S_val))["dlambda"]
        rows.append((lam, heldout_loss(Om, S_val), d))
        log_lam -= lr * lam * d
        Om0 = Om
    return np.array(rows)

"""Pins of the implicit-differentiation reference (oracle/adjoint.py).

The reference is checked against things other than itself: second
differences of the oracle's Eq. 1 objective (the Hessian), central
differences of the oracle's coordinate-descent solver (dL/dlambda, dL/dS,
dL/dX), and the closed form of the diagonal regime.  The FD checks run at
p = 20, n = 40 in FP64 on a block-diagonal precision matrix, with lambda
chosen so that the active set has a margin on both sides of the threshold
(the implicit-function theorem needs strict complementarity).
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2106_09382_gb300 import synth


def _problem(p=20, n=40, n_val=30, frac=0.46, seed=17):
    Om0 = synth.block_diag(p, 2, edge_prob=0.3, seed=seed)
    X = synth.sample(Om0, n, seed)
    Xv = synth.sample(Om0, n_val, seed + 50)
    S = O.gram(O.standardize(X))
    Sv = O.gram(O.standardize(Xv))
    lam = frac * O.lambda_max(S)
    Om, info = O.solve(S, lam, tol=1e-14, max_sweeps=200000)
    return X, Xv, S, Sv, lam, Om


def _margins(S, Om, lam):
    """(smallest |w_ij| on the active set, smallest lambda - |G_ij| off it)."""
    G = Om @ S
    G = G + G.T
    iu, ju = np.triu_indices(S.shape[0], 1)
    act = Om[iu, ju] != 0
    return np.abs(Om[iu, ju][act]).min(), (lam - np.abs(G[iu, ju][~act])).min()


def _solve_at(S, lam, Om0):
    Om, _ = O.solve(S, lam, tol=1e-14, max_sweeps=200000, Om0=Om0)
    return Om


def test_problem_is_strictly_complementary():
    X, Xv, S, Sv, lam, Om = _problem()
    a_min, gap = _margins(S, Om, lam)
    assert len(A.active_set(Om)) >= 5
    assert a_min > 1e-2 and gap > 1e-2


def test_hessian_matches_second_differences_of_objective():
    """H_cd = d^2 g / dw_c dw_d with g the oracle's Eq. 1 objective at
    lambda = 0, by central second differences."""
    X, Xv, S, Sv, lam, Om = _problem()
    p = S.shape[0]
    pairs = A.active_set(Om)
    H = A.hessian(Om, S)
    nA = H.shape[0]
    h = 1e-3
    E = [A._unit(p, pairs, c) for c in range(nA)]
    g = lambda M: O.objective(S, M, 0.0)
    Hfd = np.empty_like(H)
    for c in range(nA):
        for d in range(c, nA):
            v = (g(Om + h * E[c] + h * E[d]) - g(Om + h * E[c] - h * E[d])
                 - g(Om - h * E[c] + h * E[d]) + g(Om - h * E[c] - h * E[d])) / (4 * h * h)
            Hfd[c, d] = Hfd[d, c] = v
    assert np.abs(H - H.T).max() == 0.0
    assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() > 0


def test_hvp_matches_oracle_kkt_gradient_difference():
    """H V equals the directional derivative of the stationarity residual
    W + W^T (pairs) / W_ii - 1/w_ii (diagonal), by central differences."""
    X, Xv, S, Sv, lam, Om = _problem()
    p = S.shape[0]
    rng = np.random.default_rng(0)
    V = rng.standard_normal((p, p))
    V = np.where(Om != 0, V + V.T, 0.0)

    def F(M):
        Wm = M @ S
        out = Wm + Wm.T
        out[np.diag_indices(p)] = np.diag(Wm) - 1.0 / np.diag(M)
        return np.where(Om != 0, out, 0.0)

    h = 1e-5
    fd = (F(Om + h * V) - F(Om - h * V)) / (2 * h)
    assert np.abs(A.hvp(Om, S, V) - fd).max() <= 1e-7 * np.abs(fd).max()


def test_dlambda_matches_central_difference_of_solver():
    X, Xv, S, Sv, lam, Om = _problem()
    d = A.adjoint(Om, S, lam, A.heldout_grad(Om, Sv))["dlambda"]
    h = 1e-6 * lam
    Lp = A.heldout_loss(_solve_at(S, lam + h, Om), Sv)
    Lm = A.heldout_loss(_solve_at(S, lam - h, Om), Sv)
    fd = (Lp - Lm) / (2 * h)
    assert abs(d) > 1e-3
    assert abs(d - fd) <= 1e-5 * abs(d) + 1e-7


def test_dS_matches_central_difference_of_solver():
    """A symmetric perturbation of s_ab (both triangles) changes L by
    G_ab + G_ba in the full-matrix convention; a diagonal one by G_aa."""
    X, Xv, S, Sv, lam, Om = _problem()
    G = A.adjoint(Om, S, lam, A.heldout_grad(Om, Sv))["dS"]
    p = S.shape[0]
    rng = np.random.default_rng(1)
    cases = [(a, a) for a in rng.choice(p, 4, replace=False)]
    pairs = A.active_set(Om)
    cases += [tuple(pairs[k]) for k in rng.choice(len(pairs), 4, replace=False)]
    cases += [(0, p - 1), (2, 15)]  # across the two blocks: inactive pairs
    h = 1e-6
    for a, b in cases:
        E = np.zeros((p, p))
        E[a, b] = E[b, a] = 1.0
        Lp = A.heldout_loss(_solve_at(S + h * E, lam, Om), Sv)
        Lm = A.heldout_loss(_solve_at(S - h * E, lam, Om), Sv)
        fd = (Lp - Lm) / (2 * h)
        an = G[a, a] if a == b else G[a, b] + G[b, a]
        assert abs(an - fd) <= 1e-5 * np.abs(G).max(), (a, b, an, fd)


@pytest.mark.parametrize("prep", [0, 1, 2])
def test_dX_matches_central_difference_through_gram(prep):
    """dL/dX through S = Z^T Z / n and the data preparation."""
    X, Xv, S, Sv, lam, Om = _problem()
    n, p = X.shape

    def prepare(Xm):
        if prep == 0:
            return Xm.copy()
        return O.standardize(Xm, scale=(prep == 2))

    Z = prepare(X)
    S0 = O.gram(Z)
    lam0 = 0.46 * O.lambda_max(S0)
    Om0, _ = O.solve(S0, lam0, tol=1e-14, max_sweeps=200000)
    assert min(_margins(S0, Om0, lam0)) > 1e-3
    res = A.adjoint(Om0, S0, lam0, A.heldout_grad(Om0, Sv))
    dX = A.grad_X(X, prep, A.grad_Z(Z, res["dS"]))
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(6):
        r, c = int(rng.integers(n)), int(rng.integers(p))
        E = np.zeros_like(X)
        E[r, c] = h
        Lp = A.heldout_loss(_solve_at(O.gram(prepare(X + E)), lam0, Om0), Sv)
        Lm = A.heldout_loss(_solve_at(O.gram(prepare(X - E)), lam0, Om0), Sv)
        fd = (Lp - Lm) / (2 * h)
        assert abs(dX[r, c] - fd) <= 1e-5 * np.abs(dX).max(), (r, c, dX[r, c], fd)
    if prep:
        # the preparation removes the column means from the gradient
        assert np.abs(dX.sum(axis=0)).max() <= 1e-10 * np.abs(dX).max() * n


def test_diagonal_regime_closed_form():
    """At lambda >= lambda_max, Omega = diag(s_ii^{-1/2}) for every nearby
    lambda, so dL/dlambda = 0 and dL/ds_ii = gL_ii * (-1/2) s_ii^{-3/2}."""
    X, Xv, S, Sv, lam, Om = _problem()
    lam = 1.5 * O.lambda_max(S)
    Omd = _solve_at(S, lam, None)
    assert np.count_nonzero(Omd - np.diag(np.diag(Omd))) == 0
    gL = A.heldout_grad(Omd, Sv)
    res = A.adjoint(Omd, S, lam, gL)
    assert res["dlambda"] == 0.0
    s = np.diag(S)
    assert np.allclose(np.diag(res["dS"]), -0.5 * np.diag(gL) * s ** -1.5, rtol=1e-13, atol=0)
    assert np.count_nonzero(res["dS"] - np.diag(np.diag(res["dS"]))) == 0


def test_heldout_loss_is_the_oracle_objective_at_lambda_zero():
    X, Xv, S, Sv, lam, Om = _problem()
    assert abs(A.heldout_loss(Om, Sv) - O.objective(Sv, Om, 0.0)) <= 1e-12 * abs(A.heldout_loss(Om, Sv))


def test_hypergradient_descent_lowers_heldout_loss():
    X, Xv, S, Sv, lam, Om = _problem()
    rows = A.hypergrad_descent(S, Sv, 0.6 * O.lambda_max(S), steps=8, lr=0.5, tol=1e-11)
    assert rows[-1, 1] < rows[0, 1]
    # the step is a descent step on log lambda: lambda moves against dL/dlambda
    for k in range(len(rows) - 1):
        assert np.sign(rows[k + 1, 0] - rows[k, 0]) == -np.sign(rows[k, 2]) or rows[k, 2] == 0


def _fd_errors(S, Sv, lam, Om):
    """Largest deviation of the reference dL/dlambda and dL/dS from central
    differences of the solver (relative to the gradient's size)."""
    res = A.adjoint(Om, S, lam, A.heldout_grad(Om, Sv))
    h = 1e-6 * lam
    fd = (A.heldout_loss(_solve_at(S, lam + h, Om), Sv)
          - A.heldout_loss(_solve_at(S, lam - h, Om), Sv)) / (2 * h)
    err = abs(res["dlambda"] - fd) / abs(fd)
    p = S.shape[0]
    G = res["dS"]
    for a, b in [(1, 1), tuple(A.active_set(Om)[0])]:
        E = np.zeros((p, p))
        E[a, b] = E[b, a] = 1.0
        fdS = (A.heldout_loss(_solve_at(S + 1e-6 * E, lam, Om), Sv)
               - A.heldout_loss(_solve_at(S - 1e-6 * E, lam, Om), Sv)) / 2e-6
        an = G[a, a] if a == b else G[a, b] + G[b, a]
        err = max(err, abs(an - fdS) / np.abs(G).max())
    return err


def _drop_diag_term(Om, S, V):
    VS = V @ S
    out = VS + VS.T
    out[np.diag_indices(S.shape[0])] = np.diag(VS)
    return np.where(Om != 0, out, 0.0)


def _half_rhs(Om, gL):
    pairs = A.active_set(Om)
    return np.concatenate([np.diag(gL), gL[pairs[:, 0], pairs[:, 1]]])


@pytest.mark.parametrize("mutant", ["hvp_without_diagonal_term", "rhs_one_triangle", "dS_sign"])
def test_planted_mistakes_fail_the_fd_pins(monkeypatch, mutant):
    """A plausible mistake in the reference is caught by the FD pins."""
    X, Xv, S, Sv, lam, Om = _problem()
    assert _fd_errors(S, Sv, lam, Om) <= 1e-5
    if mutant == "hvp_without_diagonal_term":
        monkeypatch.setattr(A, "hvp", _drop_diag_term)
    elif mutant == "rhs_one_triangle":
        monkeypatch.setattr(A, "rhs", _half_rhs)
    else:
        real = A.adjoint
        monkeypatch.setattr(A, "adjoint", lambda *a: {**real(*a), "dS": -real(*a)["dS"]})
    assert _fd_errors(S, Sv, lam, Om) > 1e-2

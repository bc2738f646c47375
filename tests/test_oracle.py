"""Pins of the CPU oracle against what arXiv 2106.09382 and the mathematics fix.

None of these re-types the oracle's own formulas: each checks a result the
oracle computes against something independent of it (a table printed in the
paper, a closed form, a brute-force minimiser, a different formula for the
same quantity, an invariant of the method).
"""
import os

import numpy as np
import pytest

import oracle as O
from brute_force import minimise, objective as bf_objective

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _data_S(n, p, seed, mix=0.6):
    """A well-conditioned S = Z^T Z / n from correlated Gaussian data."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    for j in range(1, p):
        X[:, j] += mix * X[:, j - 1]
    return O.gram(O.standardize(X))


# --------------------------------------------------------------------------
# Schedule (Section 3.2, Algorithm 1; Table 1; Theorem 1)
# --------------------------------------------------------------------------

def test_schedule_matches_table1():
    """Table 1 (K_6, minimal colouring) in the paper's colour order."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_k6_colours.txt"))
            if ln.strip() and not ln.startswith("#")]
    want = [sorted(tuple(sorted((int(e[0]), int(e[1])))) for e in row) for row in rows]
    got = O.schedule(6) + 1
    have = [sorted(tuple(sorted(map(int, pr))) for pr in colour) for colour in got]
    assert have == want


def _check_colouring(p, pairs):
    pe = p + (p % 2)
    assert pairs.shape == (pe - 1, pe // 2, 2)
    real = pairs[:, :, 0] >= 0
    # the discarded pair of a colour is the one that held the extra vertex
    assert np.all((~real).sum(axis=1) == (p % 2))
    assert np.all((pairs[:, :, 1] >= 0) == real)
    i, j = pairs[:, :, 0], pairs[:, :, 1]
    assert np.all(i[real] != j[real]) and np.all((i[real] < p) & (j[real] < p))
    # each colour is a matching: a vertex appears at most once per colour
    occ = np.zeros((pe - 1, p), dtype=np.int64)
    k = np.broadcast_to(np.arange(pe - 1)[:, None], i.shape)
    np.add.at(occ, (k[real], i[real]), 1)
    np.add.at(occ, (k[real], j[real]), 1)
    assert occ.max() == 1, "a colour is not a matching"
    # every edge of K_p exactly once
    lo, hi = np.minimum(i[real], j[real]), np.maximum(i[real], j[real])
    codes = lo.astype(np.int64) * p + hi
    assert codes.size == p * (p - 1) // 2
    assert np.unique(codes).size == codes.size
    # odd p: every vertex sits out exactly once per sweep
    byes = (occ == 0).sum(axis=0)
    assert np.all(byes == (p % 2))


@pytest.mark.parametrize("p", list(range(2, 41)) + [99, 100, 255, 256, 999, 1000])
def test_schedule_is_minimal_edge_colouring(p):
    """Theorem 1: p-1 colours (even p) or p colours (odd p), each a matching,
    every edge exactly once."""
    _check_colouring(p, O.schedule(p))


@pytest.mark.slow
@pytest.mark.parametrize("p", [4999, 5000])
def test_schedule_bench_sizes(p):
    _check_colouring(p, O.schedule(p))


def test_schedule_rejects_tiny_p():
    with pytest.raises(ValueError):
        O.schedule(1)


# --------------------------------------------------------------------------
# Data preparation and Gram (Section 2.1; Algorithm 1 line T <- X^T X)
# --------------------------------------------------------------------------

def test_standardize_properties():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((37, 9)) * rng.uniform(0.1, 5, 9) + rng.uniform(-3, 3, 9)
    Z = O.standardize(X)
    assert np.abs(Z.mean(axis=0)).max() < 1e-14
    assert np.abs((Z ** 2).mean(axis=0) - 1.0).max() < 1e-13
    C = O.standardize(X, scale=False)
    assert np.abs(C.mean(axis=0)).max() < 1e-13
    assert np.allclose(C, X - X.mean(axis=0), atol=1e-13)
    bad = X.copy()
    bad[:, 3] = 2.5
    with pytest.raises(ValueError):
        O.standardize(bad)


def test_gram_known_values():
    # orthogonal +-1 columns (Hadamard) -> S = I exactly
    H = np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]], float)
    assert np.array_equal(O.gram(H), np.eye(4))
    # a hand-computed 3 x 2 case
    Z = np.array([[1.0, 2.0], [3.0, -1.0], [0.5, 4.0]])
    want = np.array([[1 + 9 + 0.25, 2 - 3 + 2], [2 - 3 + 2, 4 + 1 + 16]]) / 3.0
    assert np.allclose(O.gram(Z), want, rtol=0, atol=1e-15)


def test_gram_against_blas_and_symmetry():
    rng = np.random.default_rng(1)
    Z = O.standardize(rng.standard_normal((50, 23)))
    S = O.gram(Z)
    assert np.array_equal(S, S.T)
    assert np.allclose(S, Z.T @ Z / 50, atol=1e-14)
    assert np.allclose(np.diag(S), 1.0, atol=1e-14)
    assert np.linalg.eigvalsh(S).min() > 0


# --------------------------------------------------------------------------
# Soft-threshold and single coordinate updates (Eq. 2, Eq. 3)
# --------------------------------------------------------------------------

def test_soft_threshold_values():
    assert O.soft(1.5, 0.5) == 1.0
    assert O.soft(-1.5, 0.5) == -1.0
    assert O.soft(0.5, 0.5) == 0.0      # tie -> 0
    assert O.soft(-0.3, 0.5) == 0.0
    assert O.soft(0.0, 0.0) == 0.0
    assert O.soft(2.0, 0.0) == 2.0


def _numpy_objective(S, Om, lam):
    return bf_objective(S, Om, lam)


@pytest.mark.parametrize("lam", [0.0, 0.05, 0.3, 2.0])
def test_offdiag_update_is_exact_coordinate_minimiser(lam):
    """Eq. 3 gives the exact minimiser of Eq. 1 along omega_ij = omega_ji:
    checked against a dense 1-D scan of the objective evaluated in numpy."""
    S = _data_S(30, 6, 2)
    rng = np.random.default_rng(5)
    Om = np.eye(6) * 1.3
    for (a, b) in [(0, 2), (1, 4), (3, 5)]:
        Om[a, b] = Om[b, a] = rng.uniform(-0.3, 0.3)
    for (i, j) in [(0, 1), (2, 5), (4, 3)]:
        base = Om.copy()
        O.offdiag_update(S, Om, lam, i, j)
        w = Om[i, j]
        assert Om[j, i] == w
        grid = w + np.linspace(-0.05, 0.05, 2001)
        vals = []
        for g in grid:
            T = base.copy()
            T[i, j] = T[j, i] = g
            vals.append(_numpy_objective(S, T, lam))
        assert abs(grid[int(np.argmin(vals))] - w) <= 0.05 / 1000 + 1e-15
        f_new = _numpy_objective(S, Om, lam)
        for eps in (1e-4, -1e-4):
            T = Om.copy()
            T[i, j] = T[j, i] = w + eps
            assert _numpy_objective(S, T, lam) >= f_new - 1e-14


def test_diag_update_is_stationary():
    """Eq. 2 gives the positive root of s_ii w^2 + c w - 1 = 0, i.e. the
    stationarity omega_ii (Omega S)_ii = 1, checked with a numpy product."""
    S = _data_S(30, 7, 3)
    rng = np.random.default_rng(7)
    Om = np.eye(7)
    for (a, b) in [(0, 1), (2, 6), (3, 4), (1, 5)]:
        Om[a, b] = Om[b, a] = rng.uniform(-0.4, 0.4)
    for i in range(7):
        O.diag_update(S, Om, i)
        assert Om[i, i] > 0
        assert abs(Om[i, i] * (Om @ S)[i, i] - 1.0) < 1e-13


# --------------------------------------------------------------------------
# Closed forms and special cases of the minimiser
# --------------------------------------------------------------------------

def _p2_closed_form(r, lam):
    """Minimiser of Eq. 1 for S = [[1, r], [r, 1]]: omega_11 = omega_22 = a,
    omega_12 = c.  If |r| <= lam / 2 then a = 1, c = 0; otherwise
    (1 - r^2) a^2 + (lam/2)|r| a - 1 = 0 and c = -r a + (lam/2) sign(r)."""
    if abs(r) <= lam / 2:
        return 1.0, 0.0
    k = 1.0 - r * r
    b = lam * abs(r) / 2
    a = (-b + np.sqrt(b * b + 4 * k)) / (2 * k)
    return a, -r * a + (lam / 2) * np.sign(r)


@pytest.mark.parametrize("r,lam", [(0.6, 0.3), (-0.6, 0.3), (0.9, 0.1), (0.2, 0.5),
                                   (-0.95, 0.0), (0.3, 0.6), (0.5, 0.05)])
def test_p2_closed_form(r, lam):
    S = np.array([[1.0, r], [r, 1.0]])
    Om, info = O.solve(S, lam, tol=1e-14, max_sweeps=100000)
    a, c = _p2_closed_form(r, lam)
    assert info["converged"]
    assert abs(Om[0, 0] - a) < 1e-12 and abs(Om[1, 1] - a) < 1e-12
    assert abs(Om[0, 1] - c) < 1e-12 and Om[0, 1] == Om[1, 0]


def test_p2_printed_value():
    """r = 0.6, lam = 0.3: a = 1.181663477..., c = -0.558998086..."""
    Om, _ = O.solve(np.array([[1.0, 0.6], [0.6, 1.0]]), 0.3, tol=1e-14, max_sweeps=100000)
    assert abs(Om[0, 0] - 1.181663477) < 1e-9
    assert abs(Om[0, 1] + 0.558998086) < 1e-9


def test_p3_block_reduces_to_p2():
    r, lam = 0.7, 0.2
    S = np.array([[1.0, r, 0.0], [r, 1.0, 0.0], [0.0, 0.0, 2.5]])
    Om, info = O.solve(S, lam, tol=1e-14, max_sweeps=100000)
    a, c = _p2_closed_form(r, lam)
    assert abs(Om[0, 0] - a) < 1e-12 and abs(Om[0, 1] - c) < 1e-12
    assert abs(Om[2, 2] - 2.5 ** -0.5) < 1e-14
    assert Om[0, 2] == 0 and Om[1, 2] == 0


@pytest.mark.parametrize("lam", [0.0, 0.1, 1.0])
def test_diagonal_S(lam):
    d = np.array([0.5, 1.0, 2.0, 4.0, 9.0])
    Om, info = O.solve(np.diag(d), lam, tol=1e-15, max_sweeps=10)
    assert np.allclose(Om, np.diag(d ** -0.5), rtol=0, atol=1e-15)


def test_lambda_max_threshold():
    """At lam >= lam_max the minimiser is diagonal; just below it exactly the
    argmax pair becomes nonzero."""
    S = _data_S(40, 8, 11)
    lmax = O.lambda_max(S)
    Om, _ = O.solve(S, lmax * 1.0000001, tol=1e-13, max_sweeps=1000)
    assert np.count_nonzero(Om - np.diag(np.diag(Om))) == 0
    Om, _ = O.solve(S, lmax * 0.999, tol=1e-13, max_sweeps=1000)
    off = np.abs(Om - np.diag(np.diag(Om)))
    M = np.abs(S) * (1 / np.sqrt(np.diag(S)))[:, None]
    M = M + M.T
    np.fill_diagonal(M, 0)
    i, j = np.unravel_index(np.argmax(M), M.shape)
    nz = np.argwhere(off > 0)
    assert {tuple(x) for x in nz} == {(i, j), (j, i)}


# --------------------------------------------------------------------------
# Objective and KKT: two formulas for one quantity; KKT vs objective slopes
# --------------------------------------------------------------------------

def test_objective_from_S_equals_objective_from_data():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((25, 6))
    Z = O.standardize(X)
    S = O.gram(Z)
    Om = np.eye(6) * 1.1
    Om[0, 3] = Om[3, 0] = -0.2
    Om[1, 2] = Om[2, 1] = 0.35
    for lam in (0.0, 0.25):
        a = O.objective(S, Om, lam)
        b = O.objective_data(Z, Om, lam)
        c = _numpy_objective(S, Om, lam)
        assert abs(a - b) < 1e-12 and abs(a - c) < 1e-12


def test_kkt_matches_objective_slopes():
    """The KKT residual equals the largest directional-derivative violation of
    the objective, measured by finite differences of the numpy objective."""
    S = _data_S(30, 5, 8)
    lam = 0.15
    Om = np.eye(5) * 1.2
    Om[0, 1] = Om[1, 0] = -0.3
    Om[2, 4] = Om[4, 2] = 0.1
    h = 1e-6
    worst = 0.0
    for i in range(5):
        T1, T2 = Om.copy(), Om.copy()
        T1[i, i] += h
        T2[i, i] -= h
        d = (_numpy_objective(S, T1, lam) - _numpy_objective(S, T2, lam)) / (2 * h)
        worst = max(worst, abs(d))
        for j in range(i + 1, 5):
            Tp, Tm = Om.copy(), Om.copy()
            Tp[i, j] = Tp[j, i] = Om[i, j] + h
            Tm[i, j] = Tm[j, i] = Om[i, j] - h
            f0 = _numpy_objective(S, Om, lam)
            fp, fm = _numpy_objective(S, Tp, lam), _numpy_objective(S, Tm, lam)
            if Om[i, j] != 0:
                worst = max(worst, abs((fp - fm) / (2 * h)))
            else:
                right, left = (fp - f0) / h, (f0 - fm) / h
                worst = max(worst, max(0.0, -right, left))
    assert abs(O.kkt(S, Om, lam) - worst) < 1e-5


# --------------------------------------------------------------------------
# Lemma 1 / Lemma 2 / Theorem 2: order inside a colour does not matter;
# every colour step and the diagonal step decrease the objective
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p", [11, 12])
def test_order_within_colour_is_irrelevant(p):
    S = _data_S(3 * p, p, 21 + p)
    pairs = O.schedule(p)
    rng = np.random.default_rng(p)
    shuffled = np.stack([c[rng.permutation(len(c))] for c in pairs])
    flipped = shuffled[:, :, ::-1].copy()
    A, B, C = np.eye(p), np.eye(p), np.eye(p)
    for _ in range(3):
        O.sweep(S, A, 0.05, pairs)
        O.sweep(S, B, 0.05, shuffled)
        O.sweep(S, C, 0.05, flipped)
    assert np.array_equal(A, B) and np.array_equal(A, C)   # bit-exact
    # sensitivity: moving one pair across colours changes the trajectory
    moved = pairs.copy()
    moved[[0, 1], 0] = moved[[1, 0], 0]
    if p % 2 == 0:
        D = np.eye(p)
        for _ in range(3):
            O.sweep(S, D, 0.05, moved)
        assert not np.array_equal(A, D)


@pytest.mark.parametrize("p,lam", [(12, 0.05), (13, 0.2), (12, 0.0)])
def test_monotone_descent_every_step(p, lam):
    S = _data_S(4 * p, p, 31 + p)
    pairs = O.schedule(p)
    Om = np.eye(p)
    prev = O.objective(S, Om, lam)
    for sweep in range(4):
        for k in range(pairs.shape[0]):
            O.colour_steps(S, Om, lam, pairs, k, k + 1)
            f = O.objective(S, Om, lam)
            assert f <= prev + 1e-12 * abs(prev)
            prev = f
        O.diag_step(S, Om)
        f = O.objective(S, Om, lam)
        assert f <= prev + 1e-12 * abs(prev)
        prev = f
    assert np.array_equal(Om, Om.T)


# --------------------------------------------------------------------------
# The converged result is the global minimiser (Theorem 2), by brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("p,lam,seed", [(3, 0.2, 1), (3, 0.05, 2), (4, 0.2, 3),
                                        (4, 0.1, 4)])
def test_solution_matches_brute_force(p, lam, seed):
    S = _data_S(10 * p, p, seed, mix=0.8)
    Ob, fb = minimise(S, lam)
    Om, info = O.solve(S, lam, tol=1e-13, max_sweeps=100000)
    assert info["converged"] and info["kkt"] <= 1e-13
    assert abs(info["objective"] - fb) <= 1e-10 * abs(fb)
    assert np.abs(Om - Ob).max() <= 1e-8
    assert O.kkt(S, Ob, lam) < 1e-9


def test_small_workload_converges():
    from paper_2106_09382_gb300 import synth
    w = synth.workload_small()
    Z = O.standardize(w["X"])
    S = O.gram(Z)
    Om, info = O.solve(S, w["lam"], tol=w["tol"], max_sweeps=500, history=True)
    assert info["converged"] and info["kkt"] <= w["tol"]
    assert np.array_equal(Om, Om.T)
    obj = info["history"][:, 2]
    assert np.all(np.diff(obj) <= 1e-12 * abs(obj[0]))
    assert np.all(np.diag(Om) > 0)

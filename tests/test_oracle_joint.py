"""Pins of the joint two-population CONCORD oracle (the extension that closes
Section 6: the joint objective with lasso weight lambda1 and fusion weight
lambda2, minimised by block coordinate descent over (omega1_ij, omega2_ij)
in Algorithm 1's colour order).

Each pin is independent of the oracle's own closed forms:
  * the two block minimisers against nested one-dimensional numerical
    minimisation of the block problems;
  * lambda2 = 0: the joint sweeps are two independent Algorithm 1 runs,
    bit for bit (the single-population oracle is pinned in test_oracle.py);
  * lambda2 large: both estimates fuse to the single-population estimate on
    the average Gram (the joint objective restricted to Omega1 = Omega2 is
    twice the single objective on (S1 + S2) / 2);
  * identical populations: both estimates equal the single estimate for
    every lambda2;
  * descent: every block update lowers the joint objective;
  * optimality: at convergence no small perturbation lowers the objective,
    and the closed-form KKT residual agrees with a brute-force search over
    the fusion subgradient.
Planted mistakes (builds with ORACLE_MUTANT = 11..14) must fail a pin.
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle as O
from paper_2106_09382_gb300 import synth


def _S_pair(p=12, n=60, seed=3, n_shared=3, n_own=3):
    Om1, Om2 = synth.joint_ar1(p, n_shared=n_shared, n_own=n_own, seed=seed)
    S1 = O.gram(O.standardize(synth.sample(Om1, n, seed)))
    S2 = O.gram(O.standardize(synth.sample(Om2, n, seed + 11)))
    return S1, S2


# ---- block problems ---------------------------------------------------------

def _q(c1, g1, c2, g2, l1, l2):
    return lambda x, y: (0.5 * c1 * x * x + g1 * x + 0.5 * c2 * y * y + g2 * y
                         + l1 * (abs(x) + abs(y)) + l2 * abs(x - y))


def _nested_min(f, lo=None, hi=None):
    """argmin of a convex f(x, y) by nested 1-D minimisation (Brent, or
    bounded when lo/hi are given)."""
    kw = dict(method="bounded", bounds=(lo, hi), options={"xatol": 1e-13}) if lo is not None \
        else dict(method="brent", tol=1e-13)

    def inner(x):
        return minimize_scalar(lambda y: f(x, y), **kw)

    rx = minimize_scalar(lambda x: inner(x).fun, **kw)
    return rx.x, inner(rx.x).x


def _pair_cases(n=60, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        c1, c2 = rng.uniform(0.5, 3.0, 2)
        g1, g2 = rng.standard_normal(2)
        l1, l2 = rng.uniform(0.0, 0.6, 2)
        if k % 6 == 1:
            l2 = 0.0
        if k % 6 == 2:
            l1 = 0.0
        if k % 6 == 3:
            l2 = 5.0
        if k % 6 == 4:
            g2 = g1 + rng.normal(0, 0.05)  # near-fused
        out.append((c1, g1, c2, g2, l1, l2))
    return out


def check_pair(o, cases=None):
    worst = 0.0
    for args in cases or _pair_cases():
        x, y = o.joint_pair(*args)
        q = _q(*args)
        bx, by = _nested_min(q)
        if q(x, y) > q(bx, by) + 1e-12 * (1 + abs(q(bx, by))):
            return np.inf
        worst = max(worst, abs(x - bx), abs(y - by))
    return worst


def test_pair_minimiser_matches_nested_minimisation():
    assert check_pair(O.default()) <= 1e-5


def _h(s1, b1, s2, b2, l2):
    return lambda u, v: (-np.log(u) - np.log(v) + 0.5 * s1 * u * u + b1 * u
                         + 0.5 * s2 * v * v + b2 * v + l2 * abs(u - v))


def _diag_cases(n=40, seed=1):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        s1, s2 = rng.uniform(0.5, 2.0, 2)
        b1, b2 = rng.normal(0, 0.6, 2)
        l2 = [0.0, 0.05, 0.3, 2.0][k % 4]
        out.append((s1, b1, s2, b2, l2))
    return out


def check_diag(o):
    worst = 0.0
    for args in _diag_cases():
        d1, d2 = o.joint_diag(*args)
        h = _h(*args)
        bu, bv = _nested_min(h, 1e-6, 50.0)
        if not (d1 > 0 and d2 > 0) or h(d1, d2) > h(bu, bv) + 1e-12 * (1 + abs(h(bu, bv))):
            return np.inf
        worst = max(worst, abs(d1 - bu), abs(d2 - bv))
    return worst


def test_diag_minimiser_matches_nested_minimisation():
    assert check_diag(O.default()) <= 1e-4


def test_three_cases_are_exclusive_on_a_grid():
    """Exactly one of (x > y, x < y, x = y) comes out, and each is reached."""
    seen = set()
    for g2 in np.linspace(-2, 2, 41):
        x, y = O.joint_pair(1.5, 0.4, 2.0, g2, 0.1, 0.3)
        seen.add(int(np.sign(x - y)))
    assert seen == {-1, 0, 1}


# ---- sweeps and solves -------------------------------------------------------

def check_lambda2_zero(o, sweeps=6):
    S1, S2 = _S_pair()
    A1, A2, info = o.joint_solve(S1, S2, 0.15, 0.0, tol=1e-300, max_sweeps=sweeps)
    B1, i1 = o.solve(S1, 0.15, tol=1e-300, max_sweeps=sweeps)
    B2, i2 = o.solve(S2, 0.15, tol=1e-300, max_sweeps=sweeps)
    return (info["sweeps"] == sweeps and np.array_equal(A1, B1) and np.array_equal(A2, B2)
            and info["kkt"] == max(i1["kkt"], i2["kkt"]))


def test_lambda2_zero_is_two_independent_single_solves_bit_for_bit():
    assert check_lambda2_zero(O.default())


def check_fused_limit(o):
    S1, S2 = _S_pair()
    A1, A2, info = o.joint_solve(S1, S2, 0.15, 1e3, tol=1e-12, max_sweeps=5000)
    Sbar = 0.5 * (S1 + S2)
    B, ib = O.solve(Sbar, 0.15, tol=1e-12, max_sweeps=5000)
    return (info["converged"] and np.array_equal(A1, A2)
            and np.abs(A1 - B).max() <= 1e-9
            and abs(info["objective"] - 2 * ib["objective"]) <= 1e-10 * abs(info["objective"]))


def test_large_lambda2_fuses_to_the_average_gram_estimate():
    assert check_fused_limit(O.default())


@pytest.mark.parametrize("l2", [0.0, 0.02, 0.5])
def test_identical_populations_give_the_single_estimate(l2):
    S1, _ = _S_pair()
    A1, A2, info = O.joint_solve(S1, S1.copy(), 0.15, l2, tol=1e-12, max_sweeps=5000)
    B, ib = O.solve(S1, 0.15, tol=1e-12, max_sweeps=5000)
    assert info["converged"]
    assert np.array_equal(A1, A2)
    assert np.abs(A1 - B).max() <= 1e-9


def test_every_block_update_lowers_the_objective():
    S1, S2 = _S_pair()
    p = S1.shape[0]
    l1, l2 = 0.12, 0.04
    # a start away from the optimum: a few sweeps at another lambda
    A1, A2, _ = O.joint_solve(S1, S2, 0.3, 0.0, tol=1e-300, max_sweeps=2)
    A1, A2 = A1.copy(), A2.copy()
    f = O.joint_objective(S1, S2, A1, A2, l1, l2)
    pairs = O.schedule(p)
    for k in range(pairs.shape[0]):
        for i, j in pairs[k]:
            if i < 0:
                continue
            O.default().joint_offdiag_update(S1, S2, A1, A2, l1, l2, int(i), int(j))
            g = O.joint_objective(S1, S2, A1, A2, l1, l2)
            assert g <= f + 1e-13 * abs(f)
            f = g
    for i in range(p):
        O.default().joint_diag_update(S1, S2, A1, A2, l2, i)
        g = O.joint_objective(S1, S2, A1, A2, l1, l2)
        assert g <= f + 1e-13 * abs(f)
        f = g


def _sym_dirs(p, rng, count):
    out = []
    for _ in range(count):
        D = rng.standard_normal((p, p))
        out.append(D + D.T)
    return out


def check_local_optimality(o, l1=0.12, l2=0.04):
    """No perturbation of the converged point lowers the joint objective
    (convexity makes local optimality global)."""
    S1, S2 = _S_pair()
    p = S1.shape[0]
    A1, A2, info = o.joint_solve(S1, S2, l1, l2, tol=1e-11, max_sweeps=20000)
    if not info["converged"]:
        return False
    f0 = o.joint_objective(S1, S2, A1, A2, l1, l2)
    rng = np.random.default_rng(5)
    dirs = [(D, E) for D, E in zip(_sym_dirs(p, rng, 40), _sym_dirs(p, rng, 40))]
    # pure diagonal moves that separate or join the two diagonals
    for i in range(p):
        e = np.zeros((p, p))
        e[i, i] = 1.0
        dirs += [(e, -e), (e, e), (e, 0 * e)]
    for eps in (1e-3, 1e-5):
        for D, E in dirs:
            f = o.joint_objective(S1, S2, A1 + eps * D, A2 + eps * E, l1, l2)
            if f < f0 - 1e-13 * abs(f0):
                return False
    return True


def test_converged_point_is_a_local_and_so_global_minimum():
    assert check_local_optimality(O.default())


def _brute_kkt(S1, S2, A1, A2, l1, l2, grid=4001):
    """The joint KKT residual with the fusion subgradient z searched on a
    grid of [-1, 1] where the two values are equal."""
    W1, W2 = A1 @ S1, A2 @ S2
    p = S1.shape[0]
    zs = np.linspace(-1.0, 1.0, grid)

    def lasso_dist(g, x):
        if x > 0:
            return np.abs(g + l1)
        if x < 0:
            return np.abs(g - l1)
        return np.maximum(np.abs(g) - l1, 0.0)

    worst = 0.0
    for i in range(p):
        for j in range(i, p):
            x, y = A1[i, j], A2[i, j]
            if i == j:
                g1, g2 = W1[i, i] - 1 / x, W2[i, i] - 1 / y
                d1 = lambda g, v: np.abs(g)
            else:
                g1, g2 = W1[i, j] + W1[j, i], W2[i, j] + W2[j, i]
                d1 = lasso_dist
            z = zs if x == y else np.array([np.sign(x - y)])
            r = np.maximum(d1(g1 + l2 * z, x), d1(g2 - l2 * z, y)).min()
            worst = max(worst, float(r))
    return worst


def check_kkt_formula(o):
    S1, S2 = _S_pair()
    ok = True
    for l1, l2, sweeps in [(0.12, 0.04, 3), (0.12, 0.04, 400), (0.2, 0.3, 2), (0.05, 0.0, 3)]:
        A1, A2, info = o.joint_solve(S1, S2, l1, l2, tol=1e-300, max_sweeps=sweeps)
        k = o.joint_kkt(S1, S2, A1, A2, l1, l2)
        b = _brute_kkt(S1, S2, A1, A2, l1, l2)
        # the grid can only miss the optimum by its spacing times l2
        ok &= (k <= b + 1e-12) and (b <= k + 2 * l2 / 4000 + 1e-12)
    return ok


def test_kkt_residual_matches_brute_force_search():
    assert check_kkt_formula(O.default())


def test_solve_converges_and_reports_its_kkt():
    S1, S2 = _S_pair()
    A1, A2, info = O.joint_solve(S1, S2, 0.12, 0.04, tol=1e-9, max_sweeps=20000, history=True)
    assert info["converged"] and info["kkt"] <= 1e-9
    h = info["history"]
    assert np.all(np.diff(h[:, 2]) <= 1e-12 * np.abs(h[:-1, 2]))  # objective never rises
    assert np.array_equal(A1, A1.T) and np.array_equal(A2, A2.T)
    # the fusion is doing something: some entries fused, some not
    iu = np.triu_indices(S1.shape[0], 1)
    act = (A1[iu] != 0) | (A2[iu] != 0)
    assert np.any(act & (A1[iu] == A2[iu])) and np.any(act & (A1[iu] != A2[iu]))


# ---- planted mistakes ---------------------------------------------------------

JOINT_MUTANTS = {
    11: "pair update: wrong sign of lambda2 for the second population",
    12: "fused diagonal root: 4 (s1 + s2) instead of 8 (s1 + s2)",
    13: "objective: fusion penalty skips the diagonal",
    14: "KKT: fused blocks take u = 0 instead of the clamped optimum",
}


def _pins_pass(o):
    return (check_pair(o, _pair_cases(24)) <= 1e-5 and check_diag(o) <= 1e-4
            and check_lambda2_zero(o) and check_fused_limit(o)
            and check_local_optimality(o) and check_kkt_formula(o))


@pytest.mark.parametrize("k", sorted(JOINT_MUTANTS))
def test_planted_mistake_fails_a_pin(k):
    o = O.load_mutant(k)
    assert not _pins_pass(o), JOINT_MUTANTS[k]

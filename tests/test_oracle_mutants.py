"""Planted mistakes in the oracle are caught by its pins.

``concord_oracle.c`` and ``concord_oracle_w.c`` compiled with
``-DORACLE_MUTANT=k`` carry one plausible mistake (a dropped term, a wrong sign or index, a wrong normalisation, a
reversed rotation).  Each must fail at least one of the pin checks below,
which restate, against an arbitrary build, the independent references used in
test_oracle.py: Table 1, the p=2 closed form, the brute-force minimiser, the
data form of Eq. 1, finite-difference slopes of the objective, the
population (1/n) standardization, and (for the maintained-product mode)
agreement with the definition mode.
"""
import os

import numpy as np
import pytest

import oracle as O
from brute_force import minimise, objective as np_objective

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MUTANTS = {
    1: "Eq. 3 first sum keeps the u = j term",
    2: "Eq. 3 second sum reads row j of S instead of row i",
    3: "soft-threshold returns the wrong sign",
    4: "Eq. 3 denominator drops s_jj",
    5: "Eq. 2 sum keeps the j = i term",
    6: "circle-method rotation runs the wrong way",
    7: "KKT residual uses the wrong sign of lambda",
    8: "objective drops the factor 1/2",
    9: "Gram is not divided by n",
    10: "standardization uses 1/(n-1)",
    15: "maintained-product mode: Eq. 3 first sum keeps the u = j term",
    16: "maintained-product mode: a pair change updates row i of W only",
    17: "maintained-product mode: a diagonal change leaves W unchanged",
}


def _S(n, p, seed, mix=0.7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    for j in range(1, p):
        X[:, j] += mix * X[:, j - 1]
    Z = X - X.mean(axis=0)
    Z /= np.sqrt((Z ** 2).mean(axis=0))
    return Z.T @ Z / n


def check_table1(o):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_k6_colours.txt"))
            if ln.strip() and not ln.startswith("#")]
    want = [sorted(tuple(sorted((int(e[0]), int(e[1])))) for e in row) for row in rows]
    got = o.schedule(6) + 1
    return [sorted(tuple(sorted(map(int, pr))) for pr in c) for c in got] == want


def check_p2_closed_form(o):
    for r, lam in [(0.6, 0.3), (-0.8, 0.1)]:
        k = 1 - r * r
        b = lam * abs(r) / 2
        a = (-b + np.sqrt(b * b + 4 * k)) / (2 * k)
        c = -r * a + lam / 2 * np.sign(r)
        Om, info = o.solve(np.array([[1.0, r], [r, 1.0]]), lam, tol=1e-13, max_sweeps=5000)
        if not (abs(Om[0, 0] - a) < 1e-10 and abs(Om[0, 1] - c) < 1e-10):
            return False
    return True


def check_brute_force(o):
    S = _S(30, 3, 1)
    Ob, fb = minimise(S, 0.1)
    Om, info = o.solve(S, 0.1, tol=1e-12, max_sweeps=20000)
    return (np.abs(Om - Ob).max() < 1e-8
            and abs(info["objective"] - fb) < 1e-9 * abs(fb))


def check_objective_forms(o):
    rng = np.random.default_rng(2)
    X = rng.standard_normal((20, 4))
    Z = X - X.mean(axis=0)
    Z /= np.sqrt((Z ** 2).mean(axis=0))
    S = Z.T @ Z / 20
    Om = np.eye(4) * 1.2
    Om[0, 2] = Om[2, 0] = 0.3
    return (abs(o.objective(S, Om, 0.2) - np_objective(S, Om, 0.2)) < 1e-12
            and abs(o.objective_data(Z, Om, 0.2) - np_objective(S, Om, 0.2)) < 1e-12)


def check_kkt_slopes(o):
    S = _S(25, 4, 3)
    lam = 0.2
    Om = np.eye(4) * 1.1
    Om[0, 1] = Om[1, 0] = -0.25
    Om[2, 3] = Om[3, 2] = 0.15
    h = 1e-6
    worst = 0.0
    for i in range(4):
        for j in range(i, 4):
            Tp, Tm = Om.copy(), Om.copy()
            Tp[i, j] += h
            Tm[i, j] -= h
            if i != j:
                Tp[j, i] += h
                Tm[j, i] -= h
            fp, fm, f0 = (np_objective(S, T, lam) for T in (Tp, Tm, Om))
            if i == j or Om[i, j] != 0:
                worst = max(worst, abs((fp - fm) / (2 * h)))
            else:
                worst = max(worst, 0.0, -(fp - f0) / h, (f0 - fm) / h)
    return abs(o.kkt(S, Om, lam) - worst) < 1e-5


def check_gram_and_standardize(o):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((15, 3)) * 3 + 1
    Z = o.standardize(X)
    S = o.gram(Z)
    return (np.abs((Z ** 2).mean(axis=0) - 1).max() < 1e-13
            and np.abs(np.diag(S) - 1).max() < 1e-13)


def check_w_mode(o):
    """The maintained-product mode against the definition mode of the same
    build (the other checks pin the definition mode)."""
    S = _S(60, 31, 5, mix=0.5)
    Om1, i1 = o.solve(S, 0.05, tol=1e-9, max_sweeps=200)
    Om2, i2 = o.solve_w(S, 0.05, tol=1e-9, max_sweeps=200)
    return i1["sweeps"] == i2["sweeps"] and np.abs(Om1 - Om2).max() < 1e-12


CHECKS = [check_table1, check_p2_closed_form, check_brute_force, check_objective_forms,
          check_kkt_slopes, check_gram_and_standardize, check_w_mode]


def test_normal_build_passes_every_check():
    o = O.default()
    for chk in CHECKS:
        assert chk(o), chk.__name__


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_planted_mistake_is_caught(k):
    o = O.load_mutant(k)
    failed = []
    for chk in CHECKS:
        try:
            ok = chk(o)
        except Exception:
            ok = False
        if not ok:
            failed.append(chk.__name__)
    assert failed, "mutant %d (%s) passed every pin" % (k, MUTANTS[k])

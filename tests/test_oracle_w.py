"""The oracle's maintained-product mode (oracle/concord_oracle_w.c), the
timed CPU baseline, against its definition mode (Eq. 3 and Eq. 2 as direct
sums), which the other oracle tests pin to the paper.

The two modes run the same Algorithm 1 in the same colour order; they
differ only in how the sums of Eq. 3 / Eq. 2 are formed (read off
W = Omega S, which accumulates its row updates, instead of summed directly),
so every iterate agrees to rounding.  A slip in the W form (a missing
correction term, an update of the wrong row, a diagonal step that forgets
its own row) changes the iterates by far more than that.
"""
import numpy as np
import pytest

import oracle as O


def _data(n, p, seed, mix=0.5):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    for j in range(1, p):
        X[:, j] += mix * X[:, j - 1]
    return X * rng.uniform(0.5, 2.0, p) + rng.uniform(-1, 1, p)


@pytest.mark.parametrize("n,p,lam", [(40, 2, 0.1), (20, 3, 0.05), (60, 31, 0.02),
                                     (200, 100, 0.3), (60, 333, 0.15), (300, 517, 0.1)])
def test_w_mode_matches_definition_mode(n, p, lam):
    Z = O.standardize(_data(n, p, n + p))
    S = O.gram(Z)
    Om1, i1 = O.solve(S, lam, tol=1e-9, max_sweeps=60, history=True)
    Om2, i2 = O.solve_w(S, lam, tol=1e-9, max_sweeps=60, history=True)
    assert i1["sweeps"] == i2["sweeps"]
    assert np.abs(Om1 - Om2).max() <= 1e-12 * np.abs(Om1).max()
    h1, h2 = i1["history"], i2["history"]
    np.testing.assert_allclose(h2[:, 0], h1[:, 0], rtol=1e-9, atol=1e-13)  # delta
    np.testing.assert_allclose(h2[:, 1], h1[:, 1], rtol=1e-9, atol=1e-13)  # KKT
    np.testing.assert_allclose(h2[:, 2], h1[:, 2], rtol=1e-13)            # objective
    assert i1["first_delta_sweep"] == i2["first_delta_sweep"]
    assert i1["nonzero_changes"] == i2["nonzero_changes"]
    assert np.array_equal(Om2, Om2.T)


def test_w_mode_larger_p_few_sweeps():
    """p = 1000 (the definition mode at a few seconds per sweep): two sweeps."""
    Z = O.standardize(_data(400, 1000, 7))
    S = O.gram_w(Z)
    Om1, i1 = O.solve(S, 0.12, tol=1e-12, max_sweeps=2, history=True)
    Om2, i2 = O.solve_w(S, 0.12, tol=1e-12, max_sweeps=2, history=True)
    assert np.abs(Om1 - Om2).max() <= 1e-12 * np.abs(Om1).max()
    np.testing.assert_allclose(i2["history"][:, 2], i1["history"][:, 2], rtol=1e-13)


def test_w_mode_does_not_depend_on_the_thread_count():
    Z = O.standardize(_data(120, 257, 3))
    S = O.gram_w(Z, threads=1)
    assert np.array_equal(S, O.gram_w(Z))
    Om1, i1 = O.solve_w(S, 0.1, tol=1e-8, max_sweeps=100, threads=1, history=True)
    Om2, i2 = O.solve_w(S, 0.1, tol=1e-8, max_sweeps=100, threads=0, history=True)
    assert i1["threads"] == 1 and i2["threads"] == O.threads(0)
    assert np.array_equal(Om1, Om2)
    assert np.array_equal(i1["history"], i2["history"])


def test_w_mode_gram_is_the_oracle_gram():
    for n, p in [(5, 2), (61, 333), (37, 517)]:
        Z = O.standardize(_data(n, p, n * p))
        assert np.array_equal(O.gram_w(Z), O.gram(Z))


def test_w_mode_warm_start_and_arguments():
    Z = O.standardize(_data(80, 40, 11))
    S = O.gram(Z)
    Om0, _ = O.solve(S, 0.2, tol=1e-3, max_sweeps=3)
    Om1, i1 = O.solve(S, 0.2, tol=1e-9, max_sweeps=100, Om0=Om0)
    Om2, i2 = O.solve_w(S, 0.2, tol=1e-9, max_sweeps=100, Om0=Om0)
    assert i1["sweeps"] == i2["sweeps"]
    assert np.abs(Om1 - Om2).max() <= 1e-12
    with pytest.raises(ValueError):
        O.solve_w(S, -1.0)
    S_bad = S.copy()
    S_bad[3, 3] = 0.0
    with pytest.raises(ValueError):
        O.solve_w(S_bad, 0.1)

"""Warm-started lambda path and stability selection (concord_path,
concord_stability) against sequential solves and the FP64 oracle.

Tolerances: a path step is the same computation as a warm-started
concord_run at that lambda, so Omega must agree bit for bit; against the
oracle (n > p: unique minimiser) max|dOmega| <= 1e-6 max|Omega| and the
objective within 1e-7 relative, as for single solves.  Stability frequencies
are fractions of subsamples whose Omega has w_ij != 0: equal to the oracle's
except for pairs whose |G_ij| sits within 1e-6 of lambda in some subsample.
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_09382_gb300 import concord as C
from paper_2106_09382_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _data(p=60):
    """The first p columns of the small seeded workload (n = 200 > p)."""
    return synth.workload_small()["X"][:, :p]


def _lambdas(S, k=6, lo=0.1):
    off = np.abs(S - np.diag(np.diag(S)))
    lmax = 2.0 * off.max()  # standardized S: s_ii = 1
    return lmax * np.logspace(0.0, np.log10(lo), k)


def test_path_equals_sequential_warm_starts():
    X = _data()
    S = O.gram(O.standardize(X))
    lams = _lambdas(S)
    p = S.shape[0]
    with C.State(p, C.FP64) as a, C.State(p, C.FP64) as b:
        a.set_S(dev(S))
        b.set_S(dev(S))
        out = torch.empty((len(lams), p, p), dtype=torch.float64, device="cuda")
        res = a.path(lams, tol=1e-7, max_sweeps=300, omega_out=out)
        for k, lam in enumerate(lams):
            r = b.run(lam, tol=1e-7, max_sweeps=300)
            assert np.array_equal(host(out[k]), host(b.get_omega())), k
            assert res[k].lam == lam and res[k].sweeps == r.sweeps
            assert abs(res[k].objective - r.objective) <= 1e-12 * abs(r.objective)


def test_path_matches_oracle_at_each_lambda():
    X = _data()
    S = O.gram(O.standardize(X))
    lams = _lambdas(S)
    p = S.shape[0]
    with C.State(p, C.FP64) as st:
        st.set_S(dev(S))
        out = torch.empty((len(lams), p, p), dtype=torch.float64, device="cuda")
        res = st.path(lams, tol=1e-9, max_sweeps=500, omega_out=out)
    for k, lam in enumerate(lams):
        Om_or, info = O.solve(S, lam, tol=1e-10, max_sweeps=2000)
        G = host(out[k])
        assert res[k].status == C.OK and res[k].kkt <= 1e-9
        scale = np.abs(Om_or).max()
        assert np.abs(G - Om_or).max() <= 1e-6 * scale, k
        assert abs(res[k].objective - info["objective"]) <= 1e-7 * abs(info["objective"])
    # the first lambda is lambda_max: Omega is diagonal
    G0 = host(out[0])
    assert np.count_nonzero(G0 - np.diag(np.diag(G0))) == 0


def test_mixed_path_tracks_fp64_path():
    X = _data()
    S = O.gram(O.standardize(X))
    lams = _lambdas(S)
    p = S.shape[0]
    with C.State(p, C.FP64) as a, C.State(p, C.MIXED) as b:
        a.set_S(dev(S))
        b.set_S(dev(S, torch.float32))
        ra = a.path(lams, tol=1e-6, max_sweeps=500)
        rb = b.path(lams, tol=1e-5, max_sweeps=500)
    for x, y in zip(ra, rb):
        assert y.kkt <= 1e-5
        assert abs(x.objective - y.objective) <= 1e-5 * abs(x.objective)


def test_stability_frequencies_match_oracle():
    rng = np.random.default_rng(11)
    w = synth.workload_small()
    X = w["X"][:, :30]
    n, p = X.shape
    subsets = [np.sort(rng.choice(n, size=int(m), replace=False)) for m in (60, 75, 90, 110, 140)]
    S_full = O.gram(O.standardize(X))
    lams = _lambdas(S_full, k=3, lo=0.3)
    with C.State(p, C.FP64, n_cap=n) as st:
        freq = host(st.stability(dev(X), subsets, lams, tol=1e-10, max_sweeps=1000))
    expect = np.zeros((len(lams), p, p))
    near = np.zeros((len(lams), p, p), dtype=bool)
    for rows in subsets:
        S = O.gram(O.standardize(X[rows]))
        for k, lam in enumerate(lams):
            Om, _ = O.solve(S, lam, tol=1e-11, max_sweeps=5000)
            expect[k] += (Om != 0)
            Wm = Om @ S
            near[k] |= np.abs(np.abs(Wm + Wm.T) - lam) <= 1e-6
    expect /= len(subsets)
    diff = np.abs(freq - expect) > 1e-6
    assert not (diff & ~near).any()
    assert np.allclose(np.diagonal(freq, axis1=1, axis2=2), 1.0)


def test_path_with_dense_handover():
    """At p = 600 the candidate lists (65536 pairs) cannot hold a low lambda's
    candidates on correlated data: that path step runs on the dense kernel
    and the path continues; every step equals a sequential solve."""
    rng = np.random.default_rng(5)
    p, n = 600, 800
    X = rng.standard_normal((n, p)) @ (np.eye(p) + np.triu(rng.uniform(-0.3, 0.3, (p, p)) / np.sqrt(p), 1))
    S = O.gram(O.standardize(X))
    lmax = 2.0 * np.abs(S - np.diag(np.diag(S))).max()
    lams = lmax * np.array([0.5, 0.1, 0.01])
    with C.State(p, C.FP64) as a, C.State(p, C.FP64) as b:
        a.set_S(dev(S))
        b.set_S(dev(S))
        out = torch.empty((len(lams), p, p), dtype=torch.float64, device="cuda")
        ra = a.path(lams, tol=1e-6, max_sweeps=400, omega_out=out)
        for k, lam in enumerate(lams):
            rb = b.run(lam, tol=1e-6, max_sweeps=400)
            assert np.array_equal(host(out[k]), host(b.get_omega())), k
            assert ra[k].sweeps == rb.sweeps and ra[k].dense_sweeps == rb.dense_sweeps
    assert ra[-1].dense_sweeps > 0


def test_stability_workers_do_not_change_frequencies():
    rng = np.random.default_rng(12)
    w = synth.workload_small()
    X = w["X"][:, :40]
    n, p = X.shape
    subsets = [np.sort(rng.choice(n, size=int(m), replace=False)) for m in (60, 80, 100, 120, 150, 170)]
    S_full = O.gram(O.standardize(X))
    lams = _lambdas(S_full, k=4, lo=0.2)
    with C.State(p, C.FP64, n_cap=n) as st:
        f1 = host(st.stability(dev(X), subsets, lams, tol=1e-8, max_sweeps=1000, workers=1))
        f4 = host(st.stability(dev(X), subsets, lams, tol=1e-8, max_sweeps=1000, workers=4))
    assert np.array_equal(f1, f4)

"""Batched independent problems (concord_batch_* through the C ABI): many
CONCORD problems of uneven p and n in one persistent launch, each walking a
warm-started lambda path.

* FP64 batch against the oracle, problem by problem: the oracle solves each
  lambda from the previous lambda's Omega (Algorithm 1 in the same colour
  order, the same KKT stopping rule); the GPU forms Eq. 3 from a maintained W,
  the oracle from the direct sums, so the sweeps agree and Omega agrees to
  rounding (1e-9 of max |Omega|).
* The iterates of a problem do not depend on the batch around it, nor on the
  layout (rows per warp): each row receives the same updates in the same
  order.  Mixed-precision problems are compared bit for bit with a single
  state's path (same FP32 FMA chains).
* Support counts of the batched stability selection equal those of the
  one-state-per-subsample form (whole numbers added atomically).
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_09382_gb300 import concord as C
from paper_2106_09382_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def data(n, p, seed, mix=0.5):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    for j in range(1, p):
        X[:, j] += mix * X[:, j - 1]
    return X * rng.uniform(0.5, 2.0, p) + rng.uniform(-1, 1, p)


SIZES = [(60, 31), (200, 100), (40, 2), (90, 57), (30, 3), (150, 64)]  # (n, p): uneven


def oracle_path(S, lams, tol, max_sweeps):
    Om, out = None, []
    for lam in lams:
        Om, info = O.solve(S, lam, tol=tol, max_sweeps=max_sweeps, Om0=Om)
        out.append((Om.copy(), info))
    return out


def test_fp64_batch_matches_oracle_paths():
    Ss = [O.gram(O.standardize(data(n, p, 7 * p + n))) for n, p in SIZES]
    lams = np.array([0.4, 0.25, 0.12])
    with C.Batch([p for _, p in SIZES], C.FP64) as bt:
        for b, S in enumerate(Ss):
            bt.set_S(b, dev(S))
        res = bt.path(lams, tol=1e-9, max_sweeps=500)
        G = [host(bt.get_omega(b)) for b in range(len(SIZES))]
        info = bt.info()
    assert info["waves"] >= 1 and info["ctas"] >= len(SIZES)
    for b, S in enumerate(Ss):
        ref = oracle_path(S, lams, 1e-9, 500)
        for k in range(len(lams)):
            r, (_, oi) = res[b][k], ref[k]
            assert r.status == C.OK and r.kkt <= 1e-9
            assert abs(r.sweeps - oi["sweeps"]) <= 1, (b, k, r.sweeps, oi["sweeps"])
            assert abs(r.objective - oi["objective"]) <= 1e-10 * abs(oi["objective"])
        Om_ref = ref[-1][0]
        assert np.abs(G[b] - Om_ref).max() <= 1e-9 * np.abs(Om_ref).max(), b
        assert np.array_equal(G[b], G[b].T)


@pytest.mark.parametrize("rows", [32, 8, 2])
def test_mixed_batch_is_bitwise_a_single_state_path(rows):
    """Each problem of a mixed batch ends on the same Omega, bit for bit, as a
    single state walking the same path on the dense grid kernel, whatever the
    layout and the other problems of the batch."""
    Ss = [O.gram(O.standardize(data(n, p, 3 * p + n))) for n, p in SIZES]
    lams = np.array([0.3, 0.15])
    with C.Batch([p for _, p in SIZES], C.MIXED) as bt:
        bt.set_rows_per_warp(rows)
        for b, S in enumerate(Ss):
            bt.set_S(b, dev(S, torch.float32))
        res = bt.path(lams, tol=1e-5, max_sweeps=300)
        G = [host(bt.get_omega(b, torch.float32)) for b in range(len(SIZES))]
    for b, S in enumerate(Ss):
        p = S.shape[0]
        with C.State(p, C.MIXED) as st:
            st.set_S(dev(S, torch.float32))
            ref = st.path(lams, tol=1e-5, max_sweeps=300)  # FP32 sweeps, no polish
            want = host(st.get_omega(torch.float32))
        for k in range(len(lams)):
            assert ref[k].sweeps == res[b][k].sweeps, (b, k, ref[k].sweeps, res[b][k].sweeps)
            assert res[b][k].status == C.OK
        assert np.array_equal(G[b], want), b


def test_batch_gram_from_data_rows_and_uneven_n():
    """S of each problem from a row subset of X (uneven n): the batch's
    tensor-core Gram of the gathered rows equals the state's Gram of the same
    rows (same kernels), and the FP64 batch's Gram equals the oracle's."""
    X = data(300, 80, 5)
    rng = np.random.default_rng(1)
    sets = [np.sort(rng.choice(300, m, replace=False)).astype(np.int32) for m in (60, 140, 250)]
    for prec in (C.FP64, C.MIXED):
        with C.Batch([80, 80, 80], prec, n_cap=300) as bt:
            Xd = dev(X)
            for b, rows in enumerate(sets):
                bt.gram(b, Xd, torch.as_tensor(rows, device="cuda"))
            lam = 0.2
            res = bt.path([lam], tol=1e-7 if prec == C.FP64 else 1e-5, max_sweeps=2000)
            for b, rows in enumerate(sets):
                S = O.gram(O.standardize(X[rows]))
                G = host(bt.get_omega(b))
                Om, info = O.solve(S, lam, tol=1e-9, max_sweeps=5000)
                tol_rel = 1e-5 if prec == C.FP64 else 5e-4
                assert res[b][0].status == C.OK
                assert np.abs(G - Om).max() <= tol_rel * np.abs(Om).max(), (prec, b)


def test_batched_stability_equals_per_subsample_states():
    w = synth.workload_small()
    X = dev(w["X"])
    n, p = w["X"].shape
    subs = synth.subsamples(n, 6, 80, 180, seed=3)
    with C.State(p, C.MIXED, n_cap=n) as st:
        st.set_S(C.concord_gram(X, C.PREP_STANDARDIZE, C.GRAM_TF32X3))
        lams = st.lambda_max() * np.logspace(0, -1.0, 5)
        f1 = host(st.stability(X, subs, lams, tol=1e-5, max_sweeps=400, workers=1))
        f0 = host(st.stability(X, subs, lams, tol=1e-5, max_sweeps=400, workers=0))
    assert np.array_equal(f0, f1)
    assert f0.max() <= 1.0 and f0.min() >= 0.0 and f0[-1].sum() > f0[0].sum()


def test_batch_arguments():
    with pytest.raises(C.ConcordError):
        C.Batch([5, 1], C.MIXED)
    with C.Batch([5, 7], C.MIXED) as bt:
        with pytest.raises(C.ConcordError):
            bt.path([0.1])  # no S yet
        with pytest.raises(C.ConcordError):
            bt.set_rows_per_warp(3)
        bt.set_S(0, dev(np.eye(5), torch.float32))
        with pytest.raises(C.ConcordError):
            bt.set_S(1, dev(np.ones((7, 7)) + np.diag(np.arange(7.0)) - np.tri(7), torch.float32))


def test_mixed_batch_polishes_stalled_lambdas():
    """A tolerance below what FP32 sweeps reach makes every lambda stall in
    FP32; each is polished in FP64 (W rebuilt from Omega and the FP64 S) and
    converges.  With S given in FP64 the polished path ends on the oracle's
    path end (both at KKT <= 1e-8), and the batch agrees bit for bit with a
    single state's path, which polishes the same way."""
    sizes = [(200, 100), (90, 57), (150, 64)]
    Ss = [O.gram(O.standardize(data(n, p, 11 * p + n))) for n, p in sizes]
    lams = np.array([0.3, 0.2, 0.1])
    tol = 1e-8
    with C.Batch([p for _, p in sizes], C.MIXED) as bt:
        for b, S in enumerate(Ss):
            bt.set_S(b, dev(S))
        res = bt.path(lams, tol=tol, max_sweeps=2000)
        G = [host(bt.get_omega(b)) for b in range(len(sizes))]
    for b, S in enumerate(Ss):
        for k in range(len(lams)):
            r = res[b][k]
            assert r.status == C.OK and r.kkt <= tol, (b, k, r.as_dict())
            assert 0 < r.sweeps_fp32 < r.sweeps
        ref = oracle_path(S, lams, tol, 5000)[-1][0]
        assert np.abs(G[b] - ref).max() <= 1e-6 * np.abs(ref).max(), b
        with C.State(S.shape[0], C.MIXED) as st:
            st.set_S(dev(S))
            rs = st.path(lams, tol=tol, max_sweeps=2000)
            want = host(st.get_omega())
        assert [x.sweeps for x in rs] == [x.sweeps for x in res[b]], b
        assert np.array_equal(G[b], want), b


def test_mixed_batch_without_polish_reports_the_stall():
    S = O.gram(O.standardize(data(200, 100, 4)))
    with C.Batch([100], C.MIXED) as bt:
        bt.set_polish(False)
        bt.set_S(0, dev(S))
        res = bt.path([0.3, 0.2], tol=1e-9, max_sweeps=2000)
    assert all(r.status == C.NOT_CONVERGED and r.sweeps < 2000 for r in res[0])

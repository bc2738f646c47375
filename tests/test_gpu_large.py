"""The large sparse solve at full size: p = 20000, n = 5000, power-law
precision (average degree 4), FP32 data, lambda = 0.15, KKT <= 1e-5.

The oracle cannot solve this size in a test, so the checks are the ones that
hold at any size, plus outputs the oracle computes one by one:
  * sampled rows of the tensor-core Gram against the oracle's Gram rows
    (error bound 128 * 2^-24 + 2^-20 of the 3xTF32 products, as at small
    sizes, plus the FP32 rounding of the output, 2^-24);
  * the KKT residual of the returned Omega recomputed independently (sparse
    Omega times the FP64 copy of the same S, in torch) <= 1e-5, with the
    library's own figure agreeing;
  * symmetry, a positive diagonal, and the mixed solve against the FP64 GPU
    solve from the FP64 Gram: objective within 1e-5 relative, Omega within
    1e-3 of its largest entry (the two Grams differ by ~1e-6 and the two
    solves stop at KKT 1e-5 each).
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_09382_gb300 import concord as C
from paper_2106_09382_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _kkt(Om, S, lam):
    """Subgradient conditions of Eq. 1 (S units) from a sparse Omega."""
    W = torch.sparse.mm(Om.to_sparse(), S)
    G = W + W.t()
    d = torch.diagonal(W) - 1.0 / torch.diagonal(Om)
    act = Om != 0
    off = torch.where(act, (G + lam * torch.sign(Om)).abs(), (G.abs() - lam).clamp_min(0))
    off.fill_diagonal_(0)
    return max(d.abs().max().item(), off.max().item())


def _colours_of(v, p):
    """Colour (0-based) of every pair (v, u) under the circle method (u = v:
    -1): in the round-robin table of colour k vertex w >= 2 (1-based) sits at
    circle position (w - 2 + k) mod m, m = pe - 1; vertex 1 faces position
    m - 1 and positions c, c' face each other when c + c' = m - 2.  Checked
    against the oracle's schedule on the CPU (tests/test_capi_cpu.py)."""
    pe = p + p % 2
    m = pe - 1
    inv2 = (m + 1) // 2
    V, U = v + 1, np.arange(p) + 1
    if V == 1:
        k = (m + 1 - U) % m
    else:
        k = np.where(U == 1, (m + 1 - V) % m, ((m + 2 - V - U) % m) * inv2 % m)
    k = k.astype(np.int64)
    k[v] = -1
    return k


@pytest.fixture(scope="module")
def large():
    return synth.workload_large()


def test_large_sparse_solve(large):
    w = large
    X, p, n, lam, tol = w["X"], w["p"], w["n"], w["lam"], w["tol"]
    S32 = C.concord_gram(X, C.PREP_STANDARDIZE, C.GRAM_TF32X3)
    rows = [0, 1, 777, 12345, p - 1]
    Zh = O.standardize(X.double().cpu().numpy())
    S_rows = O.gram_rows(Zh, rows)
    err = np.abs(S32[rows].double().cpu().numpy() - S_rows).max()
    assert err <= 128 * 2.0 ** -24 + 2.0 ** -20 + 2.0 ** -24, err
    del Zh
    with C.State(p, C.MIXED) as st:
        st.set_S(S32)
        r = st.run(lam, tol=tol, max_sweeps=500)
        assert r.status == C.OK and r.kkt <= tol
        Om = st.get_omega()
    assert torch.equal(Om, Om.t()) and (torch.diagonal(Om) > 0).all()
    kkt = _kkt(Om, S32.double(), lam)
    assert kkt <= tol and abs(kkt - r.kkt) <= 1e-9
    edges = int((torch.triu(Om, 1) != 0).sum())
    assert edges > 0
    # FP64 solve from the FP64 Gram
    S64 = C.concord_gram(X, C.PREP_STANDARDIZE, C.GRAM_FP64)
    with C.State(p, C.FP64) as st:
        st.set_S(S64)
        r64 = st.run(lam, tol=tol, max_sweeps=500)
        assert r64.status == C.OK
        Om64 = st.get_omega()
    assert abs(r.objective - r64.objective) <= 1e-5 * abs(r64.objective)
    assert (Om - Om64).abs().max().item() <= 1e-3 * Om64.abs().max().item()


def test_large_sampled_sweep_entries_against_oracle(large):
    """Sampled outputs of one FP64 sweep at p = 20000, recomputed one by one
    by the oracle: each sampled off-diagonal entry of sweep t+1 from Eq. 3
    with the state the colour order implies (entries of earlier colours from
    Omega^(t+1), later ones from Omega^(t)), each sampled diagonal from Eq. 2
    with the final off-diagonals.  The S rows are the oracle's standardization
    multiplied out (numpy); the GPU state holds the FP64 Gram of the same
    data (within 1e-13 of it), so the entries agree to 1e-9."""
    w = large
    X, p, n, lam = w["X"], w["p"], w["n"], w["lam"]
    S64 = C.concord_gram(X, C.PREP_STANDARDIZE, C.GRAM_FP64)
    rng = np.random.default_rng(20000)
    rows = np.sort(rng.choice(p, 8, replace=False))
    with C.State(p, C.FP64) as st:
        st.set_S(S64)
        st.sweep(lam, 3)
        G3 = st.get_omega()
        st.sweep(lam, 1)
        G4 = st.get_omega()
        cols = {}
        for i in rows:
            nz = torch.nonzero(G4[i]).flatten().cpu().numpy()
            js = rng.choice(np.delete(np.arange(p), i), 5, replace=False)
            cols[int(i)] = np.unique(np.concatenate([js, nz[nz != i][:5]]))
        need = np.unique(np.concatenate([rows] + list(cols.values())))
        R3 = G3[torch.as_tensor(need, device=G3.device)].cpu().numpy()
        R4 = G4[torch.as_tensor(need, device=G4.device)].cpu().numpy()
        del G3, G4
    pos = {int(v): k for k, v in enumerate(need)}
    Z = O.standardize(X.double().cpu().numpy())
    S_need = Z[:, need].T @ Z / n
    del Z
    checked = 0
    for i in rows:
        a = pos[int(i)]
        col_i = _colours_of(int(i), p)
        for j in cols[int(i)]:
            b = pos[int(j)]
            k = col_i[j]
            col_j = _colours_of(int(j), p)  # column j of Omega is row j (symmetric)
            ri = np.where(col_i < k, R4[a], R3[a])
            ri[i] = R3[a, i]
            cj = np.where(col_j < k, R4[b], R3[b])
            cj[j] = R3[b, j]
            want = O.eq3(ri, cj, S_need[a], S_need[b], int(i), int(j), lam)
            assert abs(R4[a, j] - want) <= 1e-9 * max(1.0, abs(want)), (i, j, R4[a, j], want)
            checked += 1
        d_want = O.eq2(R4[a], S_need[a], int(i))
        assert abs(R4[a, i] - d_want) <= 1e-9 * d_want
    assert checked >= 8 * 5

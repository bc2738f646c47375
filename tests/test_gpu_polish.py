"""Sparse FP64 polish of mixed solves (csrc/polish.cu) against the screened
FP64 polish from a rebuilt W = Omega S, and against the oracle.

The two polishes run the same FP64 sweeps (Section 3.2, Algorithm 1) from
the same promoted iterate; they differ only in the order of the FP64 sums
that form each W entry (the screened kernel maintains W row by row, the
sparse polish sums Eq. 3 and Eq. 2 directly over the nonzeros of Omega), so
the results agree to FP64 rounding: max|dOmega| <= 1e-12 max|Omega| after a
few sweeps (each sweep contracts perturbations; 1e-12 leaves three orders of
magnitude above the ~1e-15 relative rounding of the sums), the same sweep
counts, statuses and supports.  A polish whose first sweep would break the
lazy bound commits nothing and hands over to the screened polish: then the
two runs are identical bit for bit.
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


def _solve(X, p, n, lam, tol, sparse, switch_tol=0.0, warm=None, gram=C.GRAM_TF32X3):
    """Mixed solve from device data (standardize, Gram, FP32 sweeps, polish);
    with switch_tol the sweeps start after a zero-sweep solve (the Gram and
    the refinement data in place) and switch to FP64 at that KKT level."""
    with C.State(p, C.MIXED, n_cap=n) as st:
        st.set_gram_mode(gram)
        st.set_sparse_polish(sparse)
        if switch_tol > 0:
            st.solve_device(X, lam, tol=tol, max_sweeps=0)
            r = st.run(lam, tol=tol, max_sweeps=300, switch_tol=switch_tol)
        else:
            r = st.solve_device(X, lam, tol=tol, max_sweeps=300)
        out = [r, host(st.get_omega()), host(st.get_W()), st.history()]
        if warm is not None:  # warm start from the polished iterate
            r2 = st.run(warm, tol=tol, max_sweeps=300)
            out += [r2, host(st.get_omega())]
    return out


def _close(A, B, rel=1e-12):
    return np.abs(A - B).max() <= rel * np.abs(B).max()


@pytest.mark.parametrize("p,n,tol,gram", [(333, 400, 1e-5, C.GRAM_TF32X3),
                                          (1000, 600, 1e-5, C.GRAM_FP64),
                                          (1001, 800, 1e-9, C.GRAM_TF32X3),
                                          (2000, 1000, 1e-7, C.GRAM_BF16X3)])
def test_sparse_polish_matches_screened_polish(p, n, tol, gram):
    w = synth.workload_ar1(p=p, n=n, seed=p)
    X = dev(w["X"])
    ra, Ga, Wa, Ha = _solve(X, p, n, w["lam"], tol, True, gram=gram)
    rb, Gb, Wb, Hb = _solve(X, p, n, w["lam"], tol, False, gram=gram)
    assert ra.status == C.OK and rb.status == C.OK
    assert ra.sweeps == rb.sweeps and ra.sweeps_fp32 == rb.sweeps_fp32
    polish = ra.sweeps - ra.sweeps_fp32
    assert polish >= 1
    # the sparse polish ran every polish sweep
    assert ra.sparse_sweeps == polish and rb.sparse_sweeps == 0
    # FP32 phase identical, polish to FP64 rounding
    f = ra.sweeps_fp32
    assert np.array_equal(Ha[:f, [0, 1, 3]], Hb[:f, [0, 1, 3]])
    np.testing.assert_allclose(Ha[:f, 2], Hb[:f, 2], rtol=1e-13)  # summation order
    np.testing.assert_allclose(Ha[f:, 1], Hb[f:, 1], rtol=0, atol=1e-12)
    assert _close(Ga, Gb)
    assert np.array_equal(Ga != 0, Gb != 0)
    assert abs(ra.kkt - rb.kkt) <= 1e-12 and ra.kkt <= tol
    assert abs(ra.objective - rb.objective) <= 1e-13 * abs(rb.objective)
    # W of the sparse-polished state is rebuilt when asked for
    assert _close(Wa, Wb)


def test_sparse_polish_multi_sweep_against_oracle():
    """Several sparse polish sweeps (KKT 1e-9) against the oracle's solve of
    the exact S.  The refined S entries of the mixed path are exact sums of
    the standardized data rounded to FP32: each product carries at most
    2 * 2^-24 of |z_ki z_kj|, and (1/n) sum_k |z_ki z_kj| <= 1 for unit-variance
    columns, so |dS| <= 2^-23 and the KKT residual on the exact S exceeds the
    solver's by at most 2 max_i ||Omega_i||_1 2^-23.  Omega is within 1e-6 of
    its largest entry of the oracle's, the objective within 1e-9 relative
    (the optimum moves to first order, its value to second order)."""
    p, n = 500, 700
    w = synth.workload_ar1(p=p, n=n, seed=5)
    S = O.gram(O.standardize(w["X"]))
    Om_or, info = O.solve(S, w["lam"], tol=1e-11, max_sweeps=500)
    r, G, _, _ = _solve(dev(w["X"]), p, n, w["lam"], 1e-9, True)
    assert r.status == C.OK and r.sparse_sweeps == r.sweeps - r.sweeps_fp32 >= 2
    assert np.abs(G - Om_or).max() <= 1e-6 * np.abs(Om_or).max()
    row1 = np.abs(G).sum(1).max()
    assert O.kkt(S, G, w["lam"]) <= 1e-9 + 2 * row1 * 2.0 ** -23
    f_or = O.objective(S, Om_or, w["lam"])
    assert abs(O.objective(S, G, w["lam"]) - f_or) <= 1e-9 * abs(f_or)


def test_sparse_polish_hands_over_when_the_bound_fails():
    """A mixed solve whose FP32 phase stops after a sweep or two (switch
    tolerance 0.5): the first FP64 sweep changes far more than the bound
    allows, so the sparse polish commits nothing and the screened polish
    from a rebuilt W runs every polish sweep -- the same run bit for bit as
    with the sparse polish off."""
    p, n = 400, 300
    w = synth.workload_ar1(p=p, n=n, seed=3)
    X = dev(w["X"])
    ra, Ga, Wa, Ha = _solve(X, p, n, w["lam"], 1e-6, True, switch_tol=0.5)
    rb, Gb, Wb, Hb = _solve(X, p, n, w["lam"], 1e-6, False, switch_tol=0.5)
    assert ra.status == C.OK and rb.status == C.OK
    assert ra.sweeps_fp32 <= 2 and ra.sweeps - ra.sweeps_fp32 >= 3
    assert ra.sparse_sweeps == 0  # no sparse sweep was committed
    assert ra.sweeps == rb.sweeps
    assert np.array_equal(Ga, Gb) and np.array_equal(Wa, Wb)
    assert np.array_equal(Ha[:, [0, 1, 3]], Hb[:, [0, 1, 3]])
    np.testing.assert_allclose(Ha[:, 2], Hb[:, 2], rtol=1e-13)


def test_warm_start_after_sparse_polish():
    """A second solve warm-started from a sparse-polished iterate (its FP32
    working set is rebuilt from the FP64 copies, W included) follows the
    run warm-started from the screened polish."""
    p, n = 700, 500
    w = synth.workload_ar1(p=p, n=n, seed=7)
    X = dev(w["X"])
    out_a = _solve(X, p, n, w["lam"], 1e-5, True, warm=0.15)
    out_b = _solve(X, p, n, w["lam"], 1e-5, False, warm=0.15)
    ra2, Ga2 = out_a[4], out_a[5]
    rb2, Gb2 = out_b[4], out_b[5]
    assert ra2.status == C.OK and rb2.status == C.OK and ra2.sparse_sweeps >= 1
    # the FP32 working sets of the two states may differ by the FP32 rounding
    # of W entries that agree to FP64 rounding, so the second solves agree to
    # their tolerance rather than bit for bit
    assert abs(ra2.sweeps - rb2.sweeps) <= 1
    assert np.abs(Ga2 - Gb2).max() <= 1e-4 * np.abs(Gb2).max()
    assert ra2.kkt <= 1e-5 and rb2.kkt <= 1e-5

"""Implicit-differentiation adjoint (concord_heldout / concord_adjoint /
concord_adjoint_data / concord_tune_lambda) against the FP64 reference of
oracle/adjoint.py and against central differences of the GPU solver.

Tolerances.  Both sides solve Eq. 1 to a KKT residual of 1e-12 and then
differentiate their own solution; with the same active set the two
solutions differ by about KKT / (smallest eigenvalue of H) ~ 1e-11, and the
adjoint magnifies that by the condition number of H (< 1e3 here), so
gradients must agree to 1e-7 relative (to the largest entry for matrices),
the held-out loss to 1e-10.  The CG solve runs to 1e-12 relative residual.
Central differences (step h = 1e-6 relative, solves to KKT 1e-13) carry an
O(h^2) truncation and a solve error / h ~ 1e-7: 1e-5 relative.
"""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint as A
from paper_2106_09382_gb300 import concord as C
from paper_2106_09382_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _margins(S, Om, lam):
    G = Om @ S
    G = G + G.T
    iu, ju = np.triu_indices(S.shape[0], 1)
    act = Om[iu, ju] != 0
    a_min = np.abs(Om[iu, ju][act]).min() if act.any() else np.inf
    return a_min, (lam - np.abs(G[iu, ju][~act])).min()


def _lam_with_margin(S):
    """The first fraction of lambda_max whose oracle solution has a margin of
    1e-4 on both sides of the threshold (the implicit-function theorem needs
    strict complementarity), and that solution."""
    lmax = O.lambda_max(S)
    for frac in np.linspace(0.5, 0.15, 36):
        lam = float(frac * lmax)
        Om, _ = O.solve(S, lam, tol=1e-12, max_sweeps=200000)
        if len(A.active_set(Om)) >= 3 and min(_margins(S, Om, lam)) > 1e-4:
            return lam, Om
    raise AssertionError("no lambda with a margin")


def _problem(p, n, n_val, blocks, prob, seed):
    """Block-diagonal data, standardized training and validation Grams."""
    Om0 = synth.block_diag(p, blocks, edge_prob=prob, seed=seed)
    X = synth.sample(Om0, n, seed)
    Xv = synth.sample(Om0, n_val, seed + 50)
    S = O.gram(O.standardize(X))
    Sv = O.gram(O.standardize(Xv))
    lam, Om = _lam_with_margin(S)
    return X, Xv, S, Sv, lam, Om


CASES = [(20, 40, 30, 2, 0.3, 17), (100, 200, 100, 5, 0.2, 1), (257, 400, 200, 8, 0.15, 2)]


@pytest.mark.parametrize("p,n,nv,blocks,prob,seed", CASES)
def test_adjoint_matches_reference(p, n, nv, blocks, prob, seed):
    X, Xv, S, Sv, lam, Om_or = _problem(p, n, nv, blocks, prob, seed)
    ref = A.adjoint(Om_or, S, lam, A.heldout_grad(Om_or, Sv))
    with C.State(p, C.FP64) as st:
        st.set_S(dev(S))
        r = st.run(lam, tol=1e-12, max_sweeps=200000)
        assert r.status == C.OK
        G = host(st.get_omega())
        assert np.array_equal(G != 0, Om_or != 0)  # same active set
        loss = st.heldout(dev(Sv))
        dS = torch.empty((p, p), dtype=torch.float64, device="cuda")
        info = st.adjoint(None, tol=1e-12, dS_out=dS)
    assert info.status == C.OK and info.residual <= 1e-11
    assert info.active_pairs == len(A.active_set(Om_or))
    assert abs(loss - A.heldout_loss(Om_or, Sv)) <= 1e-10 * abs(loss)
    assert abs(info.dlambda - ref["dlambda"]) <= 1e-7 * abs(ref["dlambda"])
    assert np.abs(host(dS) - ref["dS"]).max() <= 1e-7 * np.abs(ref["dS"]).max()


def test_dense_gradient_equals_heldout_gradient():
    """The same loss gradient given densely (full-matrix convention) or left
    by concord_heldout gives the same adjoint."""
    X, Xv, S, Sv, lam, _ = _problem(*CASES[1])
    p = S.shape[0]
    with C.State(p, C.FP64) as st:
        st.set_S(dev(S))
        st.run(lam, tol=1e-12, max_sweeps=200000)
        Om = st.get_omega()
        Svd = dev(Sv)
        g = -torch.diag(1.0 / torch.diagonal(Om)) + 0.5 * (Svd @ Om + Om @ Svd)
        st.heldout(Svd)
        d1 = torch.empty((p, p), dtype=torch.float64, device="cuda")
        i1 = st.adjoint(None, tol=1e-13, dS_out=d1)
        d2 = torch.empty_like(d1)
        i2 = st.adjoint(g, tol=1e-13, dS_out=d2)
    assert abs(i1.dlambda - i2.dlambda) <= 1e-10 * abs(i1.dlambda)
    assert (d1 - d2).abs().max().item() <= 1e-10 * d1.abs().max().item()


def _gpu_loss(st, Svd, lam):
    st.run(lam, tol=1e-13, max_sweeps=500000)
    return st.heldout(Svd)


def test_central_differences_p20():
    """The FD check of the differentiable-solve workload: p = 20, n = 40,
    FP64, every derivative against central differences of the GPU solver."""
    X, Xv, S, Sv, lam, _ = _problem(*CASES[0])
    p = S.shape[0]
    Svd = dev(Sv)
    with C.State(p, C.FP64, n_cap=X.shape[0]) as st:
        Xd = dev(X)
        st.solve_device(Xd, lam, tol=1e-13, max_sweeps=500000, prep=C.PREP_STANDARDIZE)
        Om = host(st.get_omega())
        st.heldout(Svd)
        dS = torch.empty((p, p), dtype=torch.float64, device="cuda")
        info = st.adjoint(None, tol=1e-13, dS_out=dS)
        dX = host(st.adjoint_data(Xd, C.PREP_STANDARDIZE))
        G = host(dS)
        S_gpu = host(C.concord_gram(Xd, C.PREP_STANDARDIZE, C.GRAM_FP64))
        # dL/dlambda
        h = 1e-6 * lam
        st.set_S(dev(S_gpu))
        st.set_omega(dev(Om))
        Lp = _gpu_loss(st, Svd, lam + h)
        st.set_omega(dev(Om))
        Lm = _gpu_loss(st, Svd, lam - h)
        fd = (Lp - Lm) / (2 * h)
        assert abs(info.dlambda - fd) <= 1e-5 * abs(fd)
        # dL/dS (symmetric perturbations, diagonal and off-diagonal)
        pairs = A.active_set(Om)
        for a, b in [(0, 0), (7, 7), tuple(pairs[0]), tuple(pairs[-1]), (0, p - 1)]:
            E = np.zeros((p, p))
            E[a, b] = E[b, a] = 1.0
            st.set_S(dev(S_gpu + 1e-6 * E))
            st.set_omega(dev(Om))
            Lp = _gpu_loss(st, Svd, lam)
            st.set_S(dev(S_gpu - 1e-6 * E))
            st.set_omega(dev(Om))
            Lm = _gpu_loss(st, Svd, lam)
            fd = (Lp - Lm) / 2e-6
            an = G[a, a] if a == b else G[a, b] + G[b, a]
            assert abs(an - fd) <= 1e-5 * np.abs(G).max(), (a, b)
        # dL/dX through the Gram and the standardization
        rng = np.random.default_rng(4)
        for _ in range(4):
            r, c = int(rng.integers(X.shape[0])), int(rng.integers(p))
            L = []
            for sgn in (1.0, -1.0):
                Xe = X.copy()
                Xe[r, c] += sgn * 1e-6
                st.solve_device(dev(Xe), lam, tol=1e-13, max_sweeps=500000,
                                prep=C.PREP_STANDARDIZE)
                L.append(st.heldout(Svd))
            fd = (L[0] - L[1]) / 2e-6
            assert abs(dX[r, c] - fd) <= 1e-5 * np.abs(dX).max(), (r, c)


@pytest.mark.parametrize("prep", [C.PREP_NONE, C.PREP_CENTER, C.PREP_STANDARDIZE])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_data_gradient_matches_reference(prep, xdt):
    X, Xv, _, Sv, _, _ = _problem(*CASES[1])
    if xdt == "f32":
        X = X.astype(np.float32).astype(np.float64)  # the FP32 input, exactly
    n, p = X.shape
    Z = X.copy() if prep == C.PREP_NONE else O.standardize(X, scale=(prep == C.PREP_STANDARDIZE))
    S = O.gram(Z)
    lam, Om_or = _lam_with_margin(S)
    ref = A.adjoint(Om_or, S, lam, A.heldout_grad(Om_or, Sv))
    dX_ref = A.grad_X(X, prep, A.grad_Z(Z, ref["dS"]))
    Xd = dev(X, torch.float32 if xdt == "f32" else torch.float64)
    with C.State(p, C.FP64, n_cap=n) as st:
        st.solve_device(Xd, lam, tol=1e-12, max_sweeps=200000, prep=prep)
        assert np.array_equal(host(st.get_omega()) != 0, Om_or != 0)
        st.heldout(dev(Sv))
        st.adjoint(None, tol=1e-12)
        dX = host(st.adjoint_data(Xd, prep, torch.empty((n, p), dtype=torch.float64,
                                                        device="cuda")))
    assert np.abs(dX - dX_ref).max() <= 1e-7 * np.abs(dX_ref).max()


def test_autograd_functions():
    """torch.autograd through the solve: dL/dlambda and dL/dX of a loss
    written in torch equal the library's held-out adjoint; dL/dS likewise."""
    from paper_2106_09382_gb300 import autograd as AG
    X, Xv, S, Sv, lam, _ = _problem(*CASES[1])
    n, p = X.shape
    Svd = dev(Sv)
    with C.State(p, C.FP64, n_cap=n) as st, C.State(p, C.FP64, n_cap=n) as ref:
        Xd = dev(X).requires_grad_(True)
        lt = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
        Om = AG.solve_X(Xd, lt, st, tol=1e-12)
        loss = -torch.log(torch.diagonal(Om)).sum() + 0.5 * torch.trace(Om @ Svd @ Om)
        loss.backward()
        ref.solve_device(dev(X), lam, tol=1e-12, max_sweeps=200000)
        l_ref = ref.heldout(Svd)
        info = ref.adjoint(None, tol=1e-12)
        dX_ref = ref.adjoint_data(dev(X))
        assert abs(loss.item() - l_ref) <= 1e-10 * abs(l_ref)
        assert abs(lt.grad.item() - info.dlambda) <= 1e-8 * abs(info.dlambda)
        assert (Xd.grad - dX_ref).abs().max().item() <= 1e-8 * dX_ref.abs().max().item()
        # from S
        Sd = dev(S).requires_grad_(True)
        lt2 = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
        Om2 = AG.solve_S(Sd, lt2, st, tol=1e-12)
        (-torch.log(torch.diagonal(Om2)).sum() + 0.5 * torch.trace(Om2 @ Svd @ Om2)).backward()
    Om_or, _ = O.solve(S, lam, tol=1e-12, max_sweeps=200000)
    r = A.adjoint(Om_or, S, lam, A.heldout_grad(Om_or, Sv))
    assert np.abs(host(Sd.grad) - r["dS"]).max() <= 1e-7 * np.abs(r["dS"]).max()
    assert abs(lt2.grad.item() - r["dlambda"]) <= 1e-7 * abs(r["dlambda"])


def test_tune_lambda_follows_reference_descent():
    X, Xv, S, Sv, lam, _ = _problem(*CASES[0])
    p = S.shape[0]
    lam0 = 0.6 * O.lambda_max(S)
    ref = A.hypergrad_descent(S, Sv, lam0, steps=8, lr=0.5, tol=1e-12, max_sweeps=500000)
    with C.State(p, C.FP64) as st:
        st.set_S(dev(S))
        rows = st.tune_lambda(dev(Sv), lam0, steps=8, lr=0.5, tol=1e-12, max_sweeps=500000,
                              cg_tol=1e-13)
    assert np.allclose(rows[:, 0], ref[:, 0], rtol=1e-7, atol=0)
    assert np.allclose(rows[:, 1], ref[:, 1], rtol=1e-9, atol=0)
    assert np.allclose(rows[:, 2], ref[:, 2], rtol=1e-6, atol=1e-9)
    assert rows[-1, 1] < rows[0, 1]


def test_diagonal_regime_and_zero_gradient():
    """lambda >= lambda_max: Omega = diag(s_ii^{-1/2}), A has no pairs,
    dL/dlambda = 0 and dL/ds_ii = -1/2 gL_ii s_ii^{-3/2}; a zero loss
    gradient gives a zero adjoint without iterations."""
    X, Xv, S, Sv, lam, _ = _problem(*CASES[1])
    p = S.shape[0]
    with C.State(p, C.FP64) as st:
        st.set_S(dev(S))
        st.run(1.5 * st.lambda_max(), tol=1e-12, max_sweeps=1000)
        Om = host(st.get_omega())
        st.heldout(dev(Sv))
        dS = torch.empty((p, p), dtype=torch.float64, device="cuda")
        info = st.adjoint(None, tol=1e-13, dS_out=dS)
        assert info.active_pairs == 0 and info.dlambda == 0.0
        gL = -np.diag(1.0 / np.diag(Om)) + 0.5 * (Sv @ Om + Om @ Sv)
        d = host(dS)
        assert np.allclose(np.diag(d), -0.5 * np.diag(gL) * np.diag(S) ** -1.5, rtol=1e-12, atol=0)
        assert np.count_nonzero(d - np.diag(np.diag(d))) == 0
        z = st.adjoint(torch.zeros((p, p), dtype=torch.float64, device="cuda"), tol=1e-10)
        assert z.iterations == 0 and z.dlambda == 0.0 and z.status == C.OK


def test_adjoint_argument_errors():
    with C.State(10, C.FP64) as st:
        S = np.eye(10)
        st.set_S(dev(S))
        with pytest.raises(C.ConcordError) as e:
            st.adjoint(None)
        assert e.value.code == C.E_ARG
        with pytest.raises(C.ConcordError) as e:
            st.adjoint_data(dev(np.ones((5, 10))))
        assert e.value.code == C.E_ARG


def test_mixed_state_adjoint_tracks_fp64():
    """A MIXED solve (FP32 sweeps + FP64 polish) gives the FP64 adjoint within
    the solve tolerance's effect."""
    X, Xv, S, Sv, lam, _ = _problem(*CASES[2])
    p = S.shape[0]
    out = []
    for prec in (C.FP64, C.MIXED):
        with C.State(p, prec) as st:
            st.set_S(dev(S, torch.float32 if prec == C.MIXED else torch.float64))
            st.run(lam, tol=1e-9, max_sweeps=100000)
            st.heldout(dev(Sv))
            out.append(st.adjoint(None, tol=1e-12).dlambda)
    assert abs(out[0] - out[1]) <= 1e-4 * abs(out[0])


def test_config_size_workload():
    """The differentiable-solve workload at full size (p = 2000, 20 blocks,
    n = 1000 train / 500 held-out): CG converges, and dL/dlambda agrees with
    a central difference of the GPU solver."""
    w = synth.workload_adjoint()
    p = w["p"]
    Xd = dev(w["X"])
    Svd = C.concord_gram(dev(w["X_val"]), C.PREP_STANDARDIZE, C.GRAM_FP64)
    with C.State(p, C.FP64) as st:
        st.set_S(C.concord_gram(Xd, C.PREP_STANDARDIZE, C.GRAM_FP64))
        lam = 0.3 * st.lambda_max()
        st.run(lam, tol=1e-11, max_sweeps=100000)
        Om = st.get_omega()
        st.heldout(Svd)
        info = st.adjoint(None, tol=1e-11)
        assert info.status == C.OK and info.residual <= 1e-10
        assert info.active_pairs > 0
        dX = st.adjoint_data(Xd)
        assert torch.isfinite(dX).all()
        h = 1e-6 * lam
        L = []
        for lm in (lam + h, lam - h):
            st.set_omega(Om)
            st.run(lm, tol=1e-12, max_sweeps=100000)
            L.append(st.heldout(Svd))
        fd = (L[0] - L[1]) / (2 * h)
        assert abs(info.dlambda - fd) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("p", [2, 3, 5])
def test_adjoint_minimal_sizes(p):
    """The smallest problems (one pair, a ragged 3 x 3, a 5 x 5), with the
    pair(s) active, against the dense reference."""
    rng = np.random.default_rng(40 + p)
    A0 = np.eye(p) + 0.6 * np.triu(rng.uniform(0.5, 1.0, (p, p)), 1)
    X = rng.standard_normal((60, p)) @ A0
    Xv = rng.standard_normal((40, p)) @ A0
    S = O.gram(O.standardize(X))
    Sv = O.gram(O.standardize(Xv))
    lam = 0.2 * O.lambda_max(S)
    Om_or, _ = O.solve(S, lam, tol=1e-13, max_sweeps=100000)
    assert len(A.active_set(Om_or)) >= 1
    ref = A.adjoint(Om_or, S, lam, A.heldout_grad(Om_or, Sv))
    with C.State(p, C.FP64) as st:
        st.set_S(dev(S))
        st.run(lam, tol=1e-13, max_sweeps=100000)
        assert np.array_equal(host(st.get_omega()) != 0, Om_or != 0)
        loss = st.heldout(dev(Sv))
        dS = torch.empty((p, p), dtype=torch.float64, device="cuda")
        info = st.adjoint(None, tol=1e-13, dS_out=dS)
        rowptr, col, val = st.get_omega_csr()
    assert abs(loss - A.heldout_loss(Om_or, Sv)) <= 1e-10 * abs(loss)
    assert abs(info.dlambda - ref["dlambda"]) <= 1e-7 * max(abs(ref["dlambda"]), 1e-12)
    assert np.abs(host(dS) - ref["dS"]).max() <= 1e-7 * np.abs(ref["dS"]).max()
    assert rowptr[-1] == np.count_nonzero(Om_or)

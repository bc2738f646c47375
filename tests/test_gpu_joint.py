"""Joint two-population CONCORD on the GPU (concord_joint_* through the C
ABI) against the FP64 CPU oracle (oracle.joint_*) on the same seeded inputs.

Tolerances:
  * FP64 sweeps, sweep by sweep: max|dOmega| <= 1e-10 max|Omega| -- the GPU
    forms each block's gradients from the maintained W = Omega S, the oracle
    from the direct sums of Eq. 3 / Eq. 2: rounding order only.  The reported
    KKT residual and objective match the oracle's on the GPU's iterate to
    1e-9 (relative to the objective, absolute on the residual).
  * Converged FP64 solve (n > p, so the joint objective is strictly convex
    and the minimiser unique): max|dOmega| <= 1e-6 max|Omega| against the
    oracle's converged solve; the oracle's residual of the GPU result
    <= 1.5 tol.
  * Mixed (FP32 sweeps, FP64 polish): the same bar as the FP64 solve.
  * Omega is bitwise independent of the grid size (every W row receives the
    same updates in the same order whatever CTA applies them).
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


def grams(p, n, seed, n_shared=None, n_own=None):
    small = p < 8  # too few non-band pairs for extra edges
    ns = n_shared if n_shared is not None else (0 if small else max(2, p // 20))
    no = n_own if n_own is not None else (0 if small else max(2, p // 20))
    Om1, Om2 = synth.joint_ar1(p, n_shared=ns, n_own=no, seed=seed)
    S1 = O.gram(O.standardize(synth.sample(Om1, n, seed)))
    S2 = O.gram(O.standardize(synth.sample(Om2, n, seed + 11)))
    return S1, S2


def joint_state(S1, S2, precision=C.FP64, grid=0):
    J = C.Joint(S1.shape[0], precision)
    J.set_S(0, dev(S1))
    J.set_S(1, dev(S2))
    if grid:
        J.set_grid(grid)
    return J


@pytest.mark.parametrize("p,n,sweeps", [(2, 30, 3), (3, 30, 3), (61, 150, 8), (96, 200, 5),
                                        (130, 300, 4)])
def test_fp64_sweeps_match_oracle_sweep_by_sweep(p, n, sweeps):
    S1, S2 = grams(p, n, p)
    l1, l2 = 0.12, 0.04
    J = joint_state(S1, S2)
    A1, A2 = np.eye(p), np.eye(p)
    pairs = O.schedule(p)
    for t in range(sweeps):
        r = J.sweep(l1, l2, 1)
        O.joint_sweep(S1, S2, A1, A2, l1, l2, pairs)
        G1, G2 = host(J.get_omega(0)), host(J.get_omega(1))
        scale = max(np.abs(A1).max(), np.abs(A2).max())
        assert np.abs(G1 - A1).max() <= 1e-10 * scale, t
        assert np.abs(G2 - A2).max() <= 1e-10 * scale, t
        assert np.array_equal(G1, G1.T) and np.array_equal(G2, G2.T)
        k = O.joint_kkt(S1, S2, G1, G2, l1, l2)
        f = O.joint_objective(S1, S2, G1, G2, l1, l2)
        assert abs(r.kkt - k) <= 1e-9, (r.kkt, k)
        assert abs(r.objective - f) <= 1e-9 * abs(f), (r.objective, f)


def test_lambda2_zero_gives_two_independent_algorithm1_runs():
    p, n = 77, 160
    S1, S2 = grams(p, n, 5)
    J = joint_state(S1, S2)
    J.sweep(0.15, 0.0, 4)
    B1, _ = O.solve(S1, 0.15, tol=1e-300, max_sweeps=4)
    B2, _ = O.solve(S2, 0.15, tol=1e-300, max_sweeps=4)
    assert np.abs(host(J.get_omega(0)) - B1).max() <= 1e-10 * np.abs(B1).max()
    assert np.abs(host(J.get_omega(1)) - B2).max() <= 1e-10 * np.abs(B2).max()


def test_large_lambda2_fuses_bitwise_and_matches_the_average_gram():
    p, n = 64, 200
    S1, S2 = grams(p, n, 9)
    J = joint_state(S1, S2)
    r = J.run(0.15, 1e3, tol=1e-9, max_sweeps=2000)
    assert r.status == C.OK
    G1, G2 = host(J.get_omega(0)), host(J.get_omega(1))
    assert np.array_equal(G1, G2)
    B, ib = O.solve(0.5 * (S1 + S2), 0.15, tol=1e-10, max_sweeps=5000)
    assert np.abs(G1 - B).max() <= 1e-6 * np.abs(B).max()


@pytest.mark.parametrize("precision", [C.FP64, C.MIXED])
def test_converged_solve_matches_oracle(precision):
    p, n = 96, 240
    S1, S2 = grams(p, n, 21)
    l1, l2, tol = 0.12, 0.04, 1e-7
    J = joint_state(S1, S2, precision)
    r = J.run(l1, l2, tol=tol, max_sweeps=5000)
    assert r.status == C.OK and r.kkt <= tol
    if precision == C.MIXED:
        assert r.sweeps_fp32 >= 1
    G1, G2 = host(J.get_omega(0)), host(J.get_omega(1))
    A1, A2, info = O.joint_solve(S1, S2, l1, l2, tol=1e-11, max_sweeps=20000)
    assert info["converged"]
    scale = max(np.abs(A1).max(), np.abs(A2).max())
    assert np.abs(G1 - A1).max() <= 1e-5 * scale
    assert np.abs(G2 - A2).max() <= 1e-5 * scale
    assert O.joint_kkt(S1, S2, G1, G2, l1, l2) <= 1.5 * tol
    assert abs(r.objective - info["objective"]) <= 1e-7 * abs(info["objective"])
    h = J.history()
    assert h.shape[0] == r.sweeps


def test_warm_start_continues_the_oracle_iterate():
    p, n = 50, 120
    S1, S2 = grams(p, n, 31)
    l1, l2 = 0.1, 0.05
    A1, A2 = np.eye(p), np.eye(p)
    for _ in range(2):
        O.joint_sweep(S1, S2, A1, A2, l1, l2)
    J = joint_state(S1, S2)
    J.set_omega(0, dev(A1))
    J.set_omega(1, dev(A2))
    J.sweep(l1, l2, 3)
    for _ in range(3):
        O.joint_sweep(S1, S2, A1, A2, l1, l2)
    scale = max(np.abs(A1).max(), np.abs(A2).max())
    assert np.abs(host(J.get_omega(0)) - A1).max() <= 1e-10 * scale
    assert np.abs(host(J.get_omega(1)) - A2).max() <= 1e-10 * scale


def test_identical_populations_equal_the_single_estimate():
    p, n = 40, 100
    S1, _ = grams(p, n, 41)
    J = joint_state(S1, S1)
    r = J.run(0.15, 0.02, tol=1e-9, max_sweeps=2000)
    assert r.status == C.OK
    G1, G2 = host(J.get_omega(0)), host(J.get_omega(1))
    assert np.array_equal(G1, G2)
    B, _ = O.solve(S1, 0.15, tol=1e-11, max_sweeps=5000)
    assert np.abs(G1 - B).max() <= 1e-6 * np.abs(B).max()


@pytest.mark.parametrize("p", [150, 151])
def test_omega_is_bitwise_independent_of_grid_and_synchronisation(p):
    """Row-version dataflow and one grid barrier per colour, on 1, 7 and the
    automatic number of CTAs: every W row receives the same updates in the
    same order, so the iterates agree bit for bit (and with the oracle)."""
    n = 300
    S1, S2 = grams(p, n, 51)
    outs = []
    for variant in (C.JOINT_ROWFLAGS, C.JOINT_BARRIER):
        for grid in (1, 7, 0):
            J = joint_state(S1, S2, grid=grid)
            J.set_variant(variant)
            J.sweep(0.1, 0.03, 4)
            outs.append((host(J.get_omega(0)), host(J.get_omega(1))))
    for G1, G2 in outs[1:]:
        assert np.array_equal(G1, outs[0][0]) and np.array_equal(G2, outs[0][1])
    A1, A2 = np.eye(p), np.eye(p)
    for _ in range(4):
        O.joint_sweep(S1, S2, A1, A2, 0.1, 0.03)
    scale = max(np.abs(A1).max(), np.abs(A2).max())
    assert np.abs(outs[0][0] - A1).max() <= 1e-10 * scale
    assert np.abs(outs[0][1] - A2).max() <= 1e-10 * scale


def test_zero_sweeps_only_evaluate():
    p, n = 20, 60
    S1, S2 = grams(p, n, 61)
    J = joint_state(S1, S2)
    r = J.sweep(0.1, 0.05, 0)
    assert r.sweeps == 0
    I = np.eye(p)
    assert abs(r.kkt - O.joint_kkt(S1, S2, I, I, 0.1, 0.05)) <= 1e-12
    assert abs(r.objective - O.joint_objective(S1, S2, I, I, 0.1, 0.05)) <= 1e-12
    assert np.array_equal(host(J.get_omega(0)), I)


def test_errors_are_reported():
    p = 8
    J = C.Joint(p)
    with pytest.raises(C.ConcordError) as e:
        J.run(0.1, 0.1)
    assert e.value.code == C.E_ARG  # S not set
    S = np.eye(p)
    S[3, 3] = 0.0
    with pytest.raises(C.ConcordError) as e:
        J.set_S(0, dev(S))
    assert e.value.code == C.E_NONPOS_DIAG
    S = np.eye(p)
    S[2, 5] = np.nan
    with pytest.raises(C.ConcordError) as e:
        J.set_S(1, dev(S))
    assert e.value.code == C.E_NONFINITE
    J.set_S(0, dev(np.eye(p)))
    J.set_S(1, dev(np.eye(p)))
    with pytest.raises(C.ConcordError) as e:
        J.run(-0.1, 0.1)
    assert e.value.code == C.E_ARG
    r = J.run(0.1, 0.1, tol=1e-12)
    assert r.status == C.OK and np.array_equal(host(J.get_omega(0)), np.eye(p))


def test_full_size_workload_converges_with_oracle_kkt():
    """The benchmark's joint workload (p = 1000, n = 500 per population),
    mixed precision as timed: the oracle's residual of the GPU result and the
    oracle's objective at it."""
    w = synth.workload_joint()
    S1 = C.concord_gram(dev(w["X1"]), C.PREP_STANDARDIZE, C.GRAM_FP64)
    S2 = C.concord_gram(dev(w["X2"]), C.PREP_STANDARDIZE, C.GRAM_FP64)
    J = C.Joint(w["p"], C.MIXED)
    J.set_S(0, S1)
    J.set_S(1, S2)
    r = J.run(w["lam1"], w["lam2"], tol=w["tol"], max_sweeps=500)
    assert r.status == C.OK
    G1, G2 = host(J.get_omega(0)), host(J.get_omega(1))
    S1h, S2h = host(S1), host(S2)
    assert O.joint_kkt(S1h, S2h, G1, G2, w["lam1"], w["lam2"]) <= 1.5 * w["tol"]
    f = O.joint_objective(S1h, S2h, G1, G2, w["lam1"], w["lam2"])
    assert abs(r.objective - f) <= 1e-9 * abs(f)


@pytest.mark.parametrize("precision", [C.FP64, C.MIXED])
def test_joint_wait_timeout_is_reported_and_context_survives(precision):
    """A row that skips one version publication makes the next reader's
    bounded wait run out: CONCORD_E_TIMEOUT with that row and colour step,
    and the device and the state stay usable.  Two CTAs hold the 31 pairs of
    a colour (p = 61), so every CTA has pairs: the first wait to start, and so
    the first to run out, is the colour-4 read of row 17 (a CTA without pairs
    would wait at the end-of-sweep grid barrier from the start and run out
    first)."""
    S1, S2 = grams(61, 150, 5)
    l1, l2 = 0.15, 0.05
    with joint_state(S1, S2, precision, grid=2) as J:
        J.set_timeout(0.25)
        J.set_fault(17, 3)
        with pytest.raises(C.ConcordError) as e:
            J.sweep(l1, l2, 1)
        assert e.value.code == C.E_TIMEOUT
        assert J.last.timeout_vertex == 17 and J.last.timeout_step == 4
        # the fault was one-shot: the same state solves to the oracle's answer
        J.set_S(0, dev(S1))
        J.set_S(1, dev(S2))
        J.set_timeout(2.0)
        r = J.run(l1, l2, tol=1e-9, max_sweeps=2000)
        assert r.status == C.OK
        G1 = host(J.get_omega(0))
    A1, A2, info = O.joint_solve(S1, S2, l1, l2, tol=1e-11, max_sweeps=20000)
    assert np.abs(G1 - A1).max() <= 1e-6 * np.abs(A1).max()
    torch.cuda.synchronize()


def test_joint_fault_switch_arguments():
    S1, S2 = grams(20, 60, 6)
    with joint_state(S1, S2) as J:
        for row, step in ((20, 0), (3, -1)):
            with pytest.raises(C.ConcordError) as e:
                J.set_fault(row, step)
            assert e.value.code == C.E_ARG
        J.set_fault(-1, 0)  # clears
        J.set_variant(C.JOINT_BARRIER)
        J.set_fault(5, 2)  # ignored by the barrier variant
        r = J.run(0.1, 0.02, tol=1e-8, max_sweeps=500)
        assert r.status == C.OK

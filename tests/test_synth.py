"""The seeded generators: structure of the precision matrices and the
covariance of the samples (CPU)."""
import numpy as np
import pytest

from paper_2106_09382_gb300 import synth


def test_power_law_is_diagonally_dominant_and_sparse():
    ei, ej, v, diag = synth.power_law(500, 2, 0.2, 0.5, 0.5, seed=3)
    assert (ei < ej).all() and len(ei) == 2 * 500 - 3  # clique of 3, then 2 per vertex
    assert (np.abs(v) >= 0.2).all() and (np.abs(v) <= 0.5).all()
    row = np.zeros(500)
    np.add.at(row, ei, np.abs(v))
    np.add.at(row, ej, np.abs(v))
    assert np.allclose(diag - row, 0.5)
    deg = np.bincount(np.concatenate([ei, ej]), minlength=500)
    assert deg.max() > 10 * np.median(deg)  # hubs: a heavy-tailed degree sequence


def test_sparse_sampler_covariance_is_the_inverse():
    torch = pytest.importorskip("torch")
    ei, ej, v, diag = synth.power_law(30, 2, 0.2, 0.5, 0.5, seed=0)
    Om = np.diag(diag)
    Om[ei, ej] = v
    Om[ej, ei] = v
    X = synth.sample_sparse(ei, ej, v, diag, 100000, seed=1, device="cpu").numpy()
    C = X.T @ X / X.shape[0]
    # sampling error ~ 3 / sqrt(n) of the scale
    assert np.abs(C - np.linalg.inv(Om)).max() <= 0.02 * np.abs(np.linalg.inv(Om)).max()
    X2 = synth.sample_sparse(ei, ej, v, diag, 100, seed=1, device="cpu")
    assert torch.equal(X2, synth.sample_sparse(ei, ej, v, diag, 100, seed=1, device="cpu"))


def test_block_diag_structure():
    Om = synth.block_diag(200, 20, 0.1, 0.3, 0.6, 0.5, seed=0)
    off = Om - np.diag(np.diag(Om))
    for b in range(20):
        s = slice(10 * b, 10 * b + 10)
        off[s, s] = 0
    assert np.count_nonzero(off) == 0
    assert np.allclose(np.diag(Om) - np.abs(Om - np.diag(np.diag(Om))).sum(1), 0.5)


def test_joint_ar1_structure():
    """Two related precision matrices: a common AR(1) band, n_shared extra
    edges with equal values in both, n_own edges in each alone; both
    positive definite (each extra edge adds a PSD term)."""
    p, ns, no = 200, 6, 4
    Om1, Om2 = synth.joint_ar1(p, n_shared=ns, n_own=no, seed=5)
    for Om in (Om1, Om2):
        assert np.array_equal(Om, Om.T)
        assert np.linalg.eigvalsh(Om).min() >= 1.0 / 3.0 - 1e-12
        band = np.diag(Om, 1)
        assert np.allclose(band, -0.5 / 0.75)
    iu, ju = np.triu_indices(p, 2)
    e1 = set(zip(iu[Om1[iu, ju] != 0], ju[Om1[iu, ju] != 0]))
    e2 = set(zip(iu[Om2[iu, ju] != 0], ju[Om2[iu, ju] != 0]))
    shared = e1 & e2
    assert len(shared) == ns and len(e1 - e2) == no and len(e2 - e1) == no
    assert all(Om1[a, b] == Om2[a, b] for a, b in shared)
    assert all(0.3 <= abs(Om1[a, b]) <= 0.6 for a, b in e1)
    # each diagonal carries its own extra edges' magnitudes
    base = synth.ar1_extra(p, 0.5, 0, seed=5)
    for Om in (Om1, Om2):
        extra = np.abs(np.triu(Om, 2)) + np.abs(np.triu(Om, 2)).T
        assert np.allclose(np.diag(Om) - np.diag(base), extra.sum(axis=1))


def test_joint_ar1_rejects_impossible_edge_counts():
    with pytest.raises(ValueError):
        synth.joint_ar1(4, n_shared=2, n_own=2)


def test_workload_joint_shapes():
    w = synth.workload_joint(p=60, n=40)
    assert w["X1"].shape == (40, 60) and w["X2"].shape == (40, 60)
    assert not np.array_equal(w["X1"], w["X2"])
    assert w["lam1"] > w["lam2"] > 0

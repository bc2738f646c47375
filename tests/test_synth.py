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

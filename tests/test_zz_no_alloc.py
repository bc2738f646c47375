"""The allocation-free Gram entry point (concord_gram_static) against the
allocating one (concord_gram, FP64 mode), called through the C ABI.

concord_gram_static serves callers that may not allocate device memory while
they run (a framework owning all device memory in its own pool, a latency-
critical loop where cudaMalloc would synchronise the device, deployments that
forbid allocation after start-up).  Its scratch is a fixed device array that
every call shares, so the check runs two calls in a row with different data:
the second must not see the first one's statistics.
"""
import numpy as np
import pytest

import oracle as O
from paper_2106_09382_gb300 import concord as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _data(n, p, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    for j in range(1, p):
        X[:, j] += 0.5 * X[:, j - 1]
    return X * rng.uniform(0.5, 3.0, p) + rng.uniform(-2, 2, p)


def test_static_gram_matches_allocating_gram_two_calls_in_a_row():
    cases = [(300, 700, 1), (123, 517, 2)]  # several tiles with ragged tails
    for n, p, seed in cases:
        X = torch.as_tensor(_data(n, p, seed), device="cuda")
        want = C.concord_gram(X, C.PREP_STANDARDIZE, C.GRAM_FP64)
        got = C.concord_gram_static(X, C.PREP_STANDARDIZE)
        torch.cuda.synchronize()
        assert torch.equal(got, got.T)
        assert float((got - want).abs().max()) <= 1e-13
        # and directly against the oracle's triple-loop Gram (FP64 sums of
        # the same n products in another order)
        S_or = O.gram(O.standardize(X.cpu().numpy()))
        assert np.abs(got.cpu().numpy() - S_or).max() <= 1e-13


def test_static_gram_float32_input_and_centering():
    X = torch.as_tensor(_data(200, 300, 3), device="cuda")
    for prep in (C.PREP_CENTER, C.PREP_STANDARDIZE):
        for x in (X, X.float()):
            want = C.concord_gram(x, prep, C.GRAM_FP64)
            got = C.concord_gram_static(x, prep)
            assert float((got - want).abs().max()) <= 1e-12


def test_static_gram_limits_and_errors():
    X = torch.zeros((4, 16385), dtype=torch.float64, device="cuda")
    with pytest.raises(C.ConcordError) as e:
        C.concord_gram_static(X)
    assert e.value.code == C.E_ARG and "16384" in str(e.value)
    Y = torch.as_tensor(_data(50, 40, 4), device="cuda")
    Y[:, 7] = 2.0
    with pytest.raises(C.ConcordError) as e:
        C.concord_gram_static(Y)
    assert e.value.code == C.E_NONPOS_DIAG
    # the shared status word is cleared by the next call
    Z = torch.as_tensor(_data(50, 40, 5), device="cuda")
    got = C.concord_gram_static(Z)
    want = C.concord_gram(Z, C.PREP_STANDARDIZE, C.GRAM_FP64)
    assert float((got - want).abs().max()) <= 1e-13


def test_static_gram_rejects_a_bad_output_tensor():
    """The binding checks `out` before the library writes p rows into it."""
    X = torch.as_tensor(_data(30, 40, 6), device="cuda")
    for bad in (torch.empty((39, 40), dtype=torch.float64, device="cuda"),
                torch.empty((40, 40), dtype=torch.float32, device="cuda"),
                torch.empty((40, 80), dtype=torch.float64, device="cuda")[:, ::2],
                torch.empty((40, 40), dtype=torch.float64)):
        with pytest.raises(ValueError):
            C.concord_gram_static(X, out=bad)
    wide = torch.zeros((40, 48), dtype=torch.float64, device="cuda")
    got = C.concord_gram_static(X, out=wide[:, :40])
    want = C.concord_gram(X, C.PREP_STANDARDIZE, C.GRAM_FP64)
    assert float((got - want).abs().max()) <= 1e-13
    assert float(wide[:, 40:].abs().max()) == 0.0

"""The C-ABI library builds, loads and exports every symbol include/concord.h
declares; host-only entry points behave as specified (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2106_09382_gb300 import concord as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "concord.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(concord_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_loads():
    lib = C.load()
    assert lib.concord_version().startswith(b"concord-gb300")
    assert lib.concord_result_size() == ctypes.sizeof(C.ConcordResult)


def test_every_declared_symbol_is_exported_and_bound():
    lib = C.load()
    syms = _declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
        assert s in C.SIGNATURES, "binding lacks %s" % s


@pytest.mark.parametrize("p", list(range(2, 30)) + [99, 100, 333, 517, 1000, 4999, 5000])
def test_schedule_matches_oracle_bit_exact(p):
    """The library's closed-form colouring equals Algorithm 1's rotation
    (oracle), slot by slot and in order within each pair."""
    assert np.array_equal(C.concord_schedule(p), O.schedule(p))


def test_schedule_argument_errors():
    lib = C.load()
    buf = (ctypes.c_int32 * 8)()
    nc = ctypes.c_int(0)
    assert lib.concord_schedule(1, buf, ctypes.byref(nc)) == C.E_ARG
    assert lib.concord_schedule(4, None, ctypes.byref(nc)) == C.E_ARG
    assert "p >= 2" in C.last_error()


def test_host_side_argument_errors():
    lib = C.load()
    assert lib.concord_set_timeout(None, 1.0) == C.E_ARG
    assert lib.concord_sweep(None, 0.1, 1, None) == C.E_ARG
    assert lib.concord_destroy(None) == C.OK
    st = ctypes.c_void_p()
    assert lib.concord_create(ctypes.byref(st), 1, C.FP64, 0, -1) == C.E_ARG
    assert lib.concord_create(ctypes.byref(st), 10, 7, 0, -1) == C.E_ARG
    assert lib.concord_gram(None, 0, 10, 10, 10, 2, 0, None, 0, 10, None) == C.E_ARG


def test_no_gpu_means_error_not_fallback():
    """Without a device the library reports CONCORD_E_CUDA; it never computes
    on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = C.load()
    st = ctypes.c_void_p()
    assert lib.concord_create(ctypes.byref(st), 10, C.FP64, 0, -1) == C.E_CUDA
    data = np.eye(4)
    r = C.ConcordResult()
    out = np.zeros((4, 4))
    rc = lib.concord_solve(data.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 0, 4, 2, 0.1,
                           1e-5, 10, C.FP64, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           ctypes.byref(r))
    assert rc == C.E_CUDA
    assert np.all(out == 0)


def test_joint_no_gpu_means_error_not_fallback():
    """The joint estimator's entry points also refuse to run without a device
    and reject bad arguments before touching one."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    lib = C.load()
    jt = ctypes.c_void_p()
    assert lib.concord_joint_create(ctypes.byref(jt), 10, C.FP64, -1) == C.E_CUDA
    assert not jt.value
    assert lib.concord_joint_create(ctypes.byref(jt), 1, C.FP64, -1) == C.E_ARG
    assert lib.concord_joint_create(ctypes.byref(jt), 10, 7, -1) == C.E_ARG
    assert lib.concord_joint_create(None, 10, C.FP64, -1) == C.E_ARG
    r = C.ConcordResult()
    assert lib.concord_joint_run(None, 0.1, 0.1, 1e-5, 10, ctypes.byref(r)) == C.E_ARG
    assert lib.concord_joint_set_variant(None, C.JOINT_ROWFLAGS) == C.E_ARG
    assert lib.concord_joint_destroy(None) == C.OK
    with pytest.raises(C.ConcordError) as e:
        C.Joint(10, device=0)
    assert e.value.code == C.E_CUDA


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 12, 13, 100, 101, 333, 1000, 1001])
def test_consecutive_partners_walk_the_ring(p):
    """Row v's partner at colour c + 1 follows from its partner at colour c:
    v = 0 meets P - c (first sub-diagonal walk); for v >= 1, when neither
    partner is vertex 0, the next one is next(w) = w - 2 cyclically on 1..P
    (second sub-diagonal walk).  The sweep kernel reads S[w][next(w)] from a
    p-vector on this basis."""
    pairs = C.concord_schedule(p)
    pe = p + (p % 2)
    P = pe - 1
    # partner table including the extra vertex of odd p (index p)
    part = np.full((pe, P), -1, dtype=np.int64)
    for c in range(P):
        used = set()
        for a_, b_ in pairs[c]:
            if a_ >= 0:
                part[a_, c], part[b_, c] = b_, a_
                used |= {int(a_), int(b_)}
        missing = [v for v in range(pe) if v not in used]
        if p % 2:
            assert len(missing) == 2  # the bye vertex and the extra vertex
            part[missing[0], c], part[missing[1], c] = missing[1], missing[0]

    def nxt(w):
        return w - 2 if w >= 3 else w - 2 + P

    for v in range(pe):
        for c in range(P - 1):
            w0, w1 = part[v, c], part[v, c + 1]
            if v == 0:
                assert w1 == w0 - 1
            elif w0 != 0 and w1 != 0:
                assert w1 == nxt(w0), (v, c, w0, w1)


def _c_rem(a, b):
    """C's % (truncating), as the kernel's integer arithmetic computes it."""
    r = abs(a) % b
    return r if a >= 0 else -r


def _joint_slot_pair(q, c, P, p):
    """The joint sweep kernel's slot -> pair closed form (slot_pair in
    csrc/joint.cu), restated: returns (i, j, ra, rb)."""
    if q == 0:
        a, b = 0, _c_rem(_c_rem(P - 1 - c, P) + P, P) + 1
    else:
        r = q - 1
        a = _c_rem(_c_rem(r - c, P) + P, P) + 1
        b = _c_rem(_c_rem(P - 2 - r - c, P) + P, P) + 1
    i, j = min(a, b), max(a, b)
    return (i if j < p else -1), j, a, b


@pytest.mark.parametrize("p", list(range(2, 24)) + [99, 100, 999, 1000, 1001])
def test_joint_slot_map_is_algorithm1_and_covers_every_vertex(p):
    """Colour c's slots hold exactly Algorithm 1's pairs of colour c, and
    every real vertex sits in exactly one slot of every colour (byes
    included): the joint kernel's row-version protocol publishes every row
    once per colour on this basis."""
    pe = p + (p % 2)
    P, half = pe - 1, pe // 2
    sched = O.schedule(p)
    for c in range(P):
        seen, got = [], set()
        for q in range(half):
            i, j, a, b = _joint_slot_pair(q, c, P, p)
            assert 0 <= a <= P and 0 <= b <= P and a != b
            seen += [v for v in (a, b) if v < p]
            if i >= 0:
                got.add((i, j))
        assert sorted(seen) == list(range(p))
        assert got == {tuple(sorted(map(int, pr))) for pr in sched[c] if pr[0] >= 0}


def test_pair_colour_closed_form_used_by_the_large_gpu_test():
    """The closed-form colour of a pair that tests/test_gpu_large.py uses to
    order sampled entries at p = 20000 equals the oracle schedule's colour."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "tgl", os.path.join(os.path.dirname(__file__), "test_gpu_large.py"))
    tgl = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(tgl)
    for p in list(range(2, 30)) + [99, 100, 517]:
        s = O.schedule(p)
        col = np.full((p, p), -1)
        for k in range(s.shape[0]):
            ok = s[k, :, 0] >= 0
            col[s[k, ok, 0], s[k, ok, 1]] = k
            col[s[k, ok, 1], s[k, ok, 0]] = k
        for v in range(p):
            assert np.array_equal(tgl._colours_of(v, p), col[v]), (p, v)

"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the 2^24-branch random circuit and the 2^20-address QRAM workload.
The oracle cannot hold these states, so the checks are properties that hold
at any size (exact halving, norm, apply-then-inverse, closed forms) and
sampled outputs of one full-size gate computed one by one from the
definition."""
import math

import numpy as np
import pytest

from oracle import sampled
from paper_2503_15118_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


def test_config2_full_properties(sqs):
    circ = W.config2(seed=2)
    n_main = len(circ["gates"]) - 8
    st = sqs.State(circ["widths"], capacity_hint=1 << 25, eps=1e-14)
    st.run(circ, upto=n_main)
    assert st.nnz() == 2 ** 24
    _, n2 = st.probabilities(0, with_probs=False)
    assert abs(n2 - 1) < 1e-12
    for i, g in enumerate(circ["gates"][n_main:]):
        st.apply(g)
        assert st.nnz() == 2 ** 24 >> (i + 1)  # each cancelling H merges every pair
    _, n2 = st.probabilities(0, with_probs=False)
    assert abs(n2 - 1) < 1e-12
    assert st.peak_nnz() == 2 ** 24
    # Apply the inverse circuit: back to |0...0> with amplitude 1.
    for g in W.inverse_circuit(circ)["gates"]:
        st.apply(g)
    d = st.to_dict()
    assert list(d) == [0] and abs(d[0] - 1) < 1e-10


@pytest.mark.parametrize("merge", [0, 16])
def test_single_gate_full_size_sampled(sqs, merge):
    widths = [16, 16, 16, 16]
    n = 1 << 24
    t = (2, 5)
    lo, hi, amps = W.random_state(widths, n, seed=2024, pair_fraction=0.5, target=t)
    st = sqs.State(widths, capacity_hint=1 << 25, eps=1e-14, merge=merge)
    st.import_(lo, hi, amps)
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    st.h_gate(*t)
    glo, _, ga = st.export()
    bit = 16 * t[0] + t[1]
    # Every pair class yields its two children (no amplitude here is small).
    assert glo.shape[0] == 2 * sampled.pair_class_count(lo, bit)
    assert np.unique(glo).shape[0] == glo.shape[0]
    assert abs(np.sum(np.abs(ga) ** 2) - np.sum(np.abs(amps) ** 2)) < 1e-9
    ref = sampled.SortedState(lo, amps)
    rng = np.random.default_rng(7)
    pick = rng.choice(glo.shape[0], size=20000, replace=False)
    want = sampled.u1q_amplitudes(ref, bit, H, glo[pick])
    assert np.max(np.abs(ga[pick] - want)) < 1e-12


def test_config3_full_closed_form(sqs):
    """2^20 addresses, 50 rounds of load / acc += data / RY and inverse RY on
    4 data bits / unload: every round returns to 2^20 branches, and the final
    state is sum_i 2^-10 |i>|0>|50 d_i mod 2^32>."""
    circ = W.config3(seed=3, addr_bits=20, rounds=50)
    table = circ["tables"][0].astype(np.uint64)
    st = sqs.State(circ["widths"], capacity_hint=1 << 25, eps=1e-14)
    gates = circ["gates"]
    st.run({"widths": circ["widths"], "tables": circ["tables"], "gates": gates[:20]})
    assert st.nnz() == 2 ** 20
    per_round = (len(gates) - 20) // 50
    for r in range(50):
        st.run({"widths": circ["widths"], "tables": circ["tables"],
                "gates": gates[20 + r * per_round: 20 + (r + 1) * per_round]})
        if r in (0, 49):
            assert st.nnz() == 2 ** 20
    assert st.peak_nnz() == 2 ** 24
    lo, hi, a = st.export()
    assert lo.shape[0] == 2 ** 20
    # Every key: addr in bits 0..19, data in bits 20..51, acc in bits 52..83.
    addr = lo & np.uint64(2 ** 20 - 1)
    data = (lo >> np.uint64(20)) & np.uint64(2 ** 32 - 1)
    acc = ((lo >> np.uint64(52)) | (hi << np.uint64(12))) & np.uint64(2 ** 32 - 1)
    assert np.all(hi >> np.uint64(20) == 0)
    assert np.array_equal(np.sort(addr), np.arange(2 ** 20, dtype=np.uint64))
    assert np.all(data == 0)
    assert np.array_equal(acc, (np.uint64(50) * table[addr]) % np.uint64(2 ** 32))
    assert np.max(np.abs(a - 2.0 ** -10)) < 1e-12
    # Sparse marginals of the 32-bit accumulator: value 50 d_i mod 2^32 with
    # probability 2^-20 per address holding it.
    want_v, want_c = np.unique((np.uint64(50) * table) % np.uint64(2 ** 32), return_counts=True)
    v, p, n2 = st.probabilities_sparse(2)
    assert np.array_equal(v, want_v)
    assert np.max(np.abs(p - want_c * 2.0 ** -20)) < 1e-15
    assert abs(n2 - 1.0) < 1e-12
    v, p, _ = st.probabilities_sparse(1)  # the data register is 0 everywhere
    assert list(v) == [0] and abs(p[0] - 1.0) < 1e-12


def _golden_config2():
    import hashlib
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_seed2.npz")
    gold = np.load(path)
    circ = W.config2(seed=2)
    digest = hashlib.sha256(repr(circ["gates"]).encode()).hexdigest()
    assert str(gold["gates_digest"]) == digest, "the config-2 generator changed: rerun the script"
    return circ, gold


def _sorted_export(st):
    lo, hi, a = st.export()
    assert not hi.any()
    order = np.argsort(lo)
    return lo[order], a[order]


@pytest.mark.parametrize("amp32", [False, True])
def test_config2_full_size_against_oracle_golden(sqs, amp32):
    """The benchmark circuit at full size, in bench.py's launch configuration
    (capacity hint 2^25, a side stream), element by element against values
    the CPU oracle wrote (tests/golden/make_config2_golden.py): 2^17 sampled
    branches of the 2^23-branch state right after the first cancelling H (the
    fold that takes the whole 2^24-branch state in), and the whole final
    state.  FP64: keys bit-exact, amplitudes within 1e-12.  FP32 storage:
    the same keys, amplitudes within 2e-6, fidelity >= 1 - 1e-6."""
    import torch
    circ, gold = _golden_config2()
    atol = 2e-6 if amp32 else 1e-12
    stream = torch.cuda.Stream()
    st = sqs.State(circ["widths"], amp32=amp32, capacity_hint=1 << 25,
                   stream=stream.cuda_stream, eps=circ["eps"])
    after = int(gold["after"])
    st.run(circ, upto=after)
    lo, a = _sorted_export(st)
    assert lo.shape[0] == int(gold["mid_n"])
    pos = np.searchsorted(lo, gold["mid_lo"])
    assert np.all(pos < lo.shape[0]) and np.array_equal(lo[pos], gold["mid_lo"])
    assert np.max(np.abs(a[pos] - gold["mid_amp"])) < atol
    for g in circ["gates"][after:]:
        st.apply(g, circ["tables"])
    lo, a = _sorted_export(st)
    assert np.array_equal(lo, gold["final_lo"])
    err = np.max(np.abs(a - gold["final_amp"]))
    assert err < atol, err
    ref = gold["final_amp"]
    fid = abs(np.vdot(ref, a)) ** 2 / (np.vdot(ref, ref).real * np.vdot(a, a).real)
    assert fid >= (1 - 1e-6 if amp32 else 1 - 1e-10)
    assert st.peak_nnz() == int(gold["peak"])
    st.close()

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
    key = (hi.astype(object) << 64) | lo.astype(object)
    addr = np.array([int(k) & (2 ** 20 - 1) for k in key[:4096]])
    data = np.array([(int(k) >> 20) & (2 ** 32 - 1) for k in key[:4096]])
    acc = np.array([(int(k) >> 52) & (2 ** 32 - 1) for k in key[:4096]])
    assert np.all(data == 0)
    assert np.all(acc == (50 * table[addr]) % 2 ** 32)
    assert np.max(np.abs(a - 2.0 ** -10)) < 1e-12

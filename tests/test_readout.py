"""Readout through the C ABI: the sparse marginal probabilities of a
register of any width (sqs_probabilities_sparse) against the oracle's
marginals, and sqs_export's ascending key order."""
import numpy as np
import pytest

import oracle
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


def _check_sparse(g, o, reg, tol):
    v, p, n2 = g.probabilities_sparse(reg)
    ov, op = o.probabilities(reg)
    assert np.array_equal(v, ov)
    assert np.all(v[1:] > v[:-1])
    assert np.max(np.abs(p - op)) <= tol
    assert abs(n2 - o.norm2()) <= tol * 10
    return v, p


@pytest.mark.parametrize("amp32", [False, True])
def test_sparse_marginals_config3_reduced(sqs, amp32):
    """Two-word keys, 32-bit data and accumulator registers (too wide for the
    dense form), mid-round (data loaded) and at the end, FP64 and FP32."""
    circ = W.config3(seed=3, addr_bits=10, rounds=4)
    per_round = (len(circ["gates"]) - 10) // 4
    cut = 10 + per_round + 3  # inside round 2, after the load and the add
    g = sqs.run_circuit(circ, amp32=amp32, upto=cut)
    o = oracle.run_circuit(circ, upto=cut)
    tol = 1e-6 if amp32 else 1e-13
    for reg in range(len(circ["widths"])):
        _check_sparse(g, o, reg, tol)
    g.run({"widths": circ["widths"], "tables": circ["tables"], "gates": circ["gates"][cut:]})
    o2 = oracle.run_circuit(circ)
    for reg in range(len(circ["widths"])):
        _check_sparse(g, o2, reg, tol)


@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 70001])
def test_sparse_marginals_runs_across_tiles(sqs, n):
    """Random states whose register values repeat in long runs (a 3-bit
    register over up to 70001 branches: runs of thousands spanning many
    2048-branch tiles) and in short ones (a 40-bit register); the narrow
    register also against the dense form."""
    widths = [3, 40, 21]
    lo, hi, amps = W.random_state(widths, n, seed=n)
    g = sqs.State(widths, eps=1e-14)
    g.import_(lo, hi, amps)
    o = oracle.OracleState(widths, eps=1e-14)
    o.import_(lo, hi, amps)
    for reg in range(3):
        _check_sparse(g, o, reg, 1e-12)
    v, p, _ = g.probabilities_sparse(0)
    dense, n2 = g.probabilities(0)
    assert np.array_equal(np.nonzero(dense)[0], v.astype(np.int64))
    assert np.max(np.abs(dense[v.astype(np.int64)] - p)) < 1e-14
    assert abs(dense.sum() - n2) < 1e-12
    # Deterministic: a second call gives the same bits.
    v1, p1, _ = g.probabilities_sparse(1)
    v2, p2, _ = g.probabilities_sparse(1)
    assert np.array_equal(v1, v2) and np.array_equal(p1, p2)


def test_sparse_marginals_empty_and_capacity(sqs):
    g = sqs.State([8, 40], eps=1e-14)
    g.h_gate(0, 0)
    g.h_gate(0, 0)  # back to |0>
    v, p, n2 = g.probabilities_sparse(1)
    assert list(v) == [0] and abs(p[0] - 1) < 1e-15
    g.import_(np.zeros(0, np.uint64), np.zeros(0, np.uint64), np.zeros(0, np.complex128))
    v, p, n2 = g.probabilities_sparse(1)
    assert v.shape[0] == 0 and n2 == 0.0


@pytest.mark.parametrize("widths", [[16, 16, 16, 16], [20, 32, 32]])
@pytest.mark.parametrize("amp32", [False, True])
def test_export_ascending(sqs, widths, amp32):
    """sqs_export returns the branches in ascending key order, after merges
    whose output is segmented (storage order is not key order)."""
    circ = W.random_circuit(widths, 60, seed=11, kinds=("x", "cx", "ry", "h", "phase", "add"))
    g = sqs.run_circuit(circ, amp32=amp32)
    lo, hi, a = g.export()
    key = (hi.astype(object) << 64) | lo.astype(object)
    assert all(key[i] < key[i + 1] for i in range(len(key) - 1))
    o = oracle.run_circuit(circ)
    olo, ohi, _ = o.export()
    assert np.array_equal(lo, olo) or amp32
    assert g.nnz() == len(key)

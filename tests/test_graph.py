"""CUDA-graph capture of circuits (sqs_capture_begin / _end, sqs_graph_launch).

A captured circuit replayed from |0...0> must give the state the same calls
give when issued one by one -- bit for bit, since the same kernels run on the
same inputs -- and therefore the oracle's state.  Calls that would wait for
the device inside a capture are refused and leave the state usable; a static
bound that the circuit outgrows is caught on the device and reported at the
next wait, without out-of-bounds writes.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import qlss as Q
from tests.helpers import build_config1, compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


@pytest.fixture(scope="module")
def cfg1():
    return build_config1(seed=1)


def _stream():
    import torch
    return torch.cuda.Stream().cuda_stream


def _state(sqs, widths, **kw):
    """States on a stream of their own: capture needs one."""
    return sqs.State(widths, stream=_stream(), **kw)


def _eager(sqs, circ, **kw):
    st = _state(sqs, circ["widths"], **kw)
    st.run(circ)
    return st


@pytest.mark.parametrize("amp32", [False, True])
def test_replay_equals_eager_config1(sqs, cfg1, amp32):
    eager = _eager(sqs, cfg1, amp32=amp32).to_dict()
    st = _state(sqs, cfg1["widths"], amp32=amp32)
    st.run(cfg1)            # creates the QRAM table outside the capture
    g = st.capture(cfg1, static_bound=8192)
    assert st.nnz() == 1    # nothing ran: the state is |0...0>
    for _ in range(3):
        g.launch()
        got = st.to_dict()
        assert set(got) == set(eager) and all(got[k] == eager[k] for k in got)
    if not amp32:
        o = oracle.run_circuit(cfg1)
        assert compare_states(got, o.to_dict()) >= 1 - 1e-10
    g.close()


def test_replay_batched_walk(sqs):
    cfg = Q.config5(seed=9, n_inst=8, n_min=2, n_max=3, T=10)
    circ = Q.batched_circuit(cfg, 3)
    eager = _eager(sqs, circ).to_dict()
    st = _state(sqs, circ["widths"])
    st.run(circ)            # tables (QRAM and rotation) exist from here on
    peak = st.peak_nnz()
    g = st.capture(circ, static_bound=2 * peak)
    g.launch()
    g.launch()
    got = st.to_dict()
    assert set(got) == set(eager) and all(got[k] == eager[k] for k in got)


def test_capture_refuses_waits_and_stays_usable(sqs, cfg1):
    st = _state(sqs, cfg1["widths"])
    st.run(cfg1)
    st.capture_begin(8192)
    st.h_gate(0, 0)
    with pytest.raises(sqs.SqsError):
        st.nnz()
    with pytest.raises(sqs.SqsError):
        st.capture_end()
    st.reset()
    st.run(cfg1)
    o = oracle.run_circuit(cfg1)
    assert compare_states(st.to_dict(), o.to_dict()) >= 1 - 1e-10


def test_static_bound_overflow_is_reported(sqs):
    widths = [8, 8]
    circ = {"widths": widths, "eps": 1e-14, "tables": [],
            "gates": [("h", 0, b, ()) for b in range(8)] + [("h", 1, b, ()) for b in range(6)]}
    st = _state(sqs, widths)
    g = st.capture(circ, static_bound=64)     # the circuit reaches 2^14 branches
    g.launch()
    with pytest.raises(sqs.SqsError):
        st.nnz()
    st.reset()                                # the sticky error clears with a reset
    st.run(circ)
    assert st.nnz() == 2 ** 14


def test_replay_is_faster_than_eager_for_small_states(sqs, cfg1):
    """Config 1 is launch-bound: replaying the captured circuit beats issuing
    its 209 gates (timing printed; the assertion is loose)."""
    import torch
    st = _state(sqs, cfg1["widths"])
    st.run(cfg1)
    g = st.capture(cfg1, static_bound=8192)
    for _ in range(3):
        g.launch()
        st.reset()
        st.run(cfg1)
    torch.cuda.synchronize()
    reps = 20
    t0 = time.perf_counter()
    for _ in range(reps):
        st.reset()
        st.run(cfg1)
    st.sync()
    t_eager = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        g.launch()
    st.sync()
    t_graph = (time.perf_counter() - t0) / reps
    print(f"\nconfig 1 per circuit: eager {t_eager * 1e3:.3f} ms, graph {t_graph * 1e3:.3f} ms")
    assert t_graph < t_eager


@pytest.mark.parametrize("factor", [2, 32])
def test_replay_with_a_loose_static_bound(sqs, factor):
    """A static bound far above the peak sizes every segment list of the
    replay mostly empty: the partition and in-place passes search it for
    non-empty units in batches and the pair kernel draws only the buckets
    the device count asks for.  The replay stays bit-identical to eager
    issue and equal to the oracle."""
    from paper_2503_15118_gb300 import workloads as W
    circ = W.random_circuit([8, 8, 8], 80, seed=31,
                            kinds=("x", "cx", "ccx", "ry", "phase", "h", "add"))
    eager = _eager(sqs, circ).to_dict()
    st = _state(sqs, circ["widths"])
    st.run(circ)
    peak = st.peak_nnz()
    g = st.capture(circ, static_bound=factor * peak)
    for _ in range(2):
        g.launch()
        got = st.to_dict()
        assert set(got) == set(eager) and all(got[k] == eager[k] for k in got)
    assert st.stats()["steps_hash"] > 0
    o = oracle.run_circuit(circ)
    assert compare_states(got, o.to_dict()) >= 1 - 1e-10
    g.close()

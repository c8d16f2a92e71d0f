"""The autotuner (SQS_AUTOTUNE): while measuring, every step takes the
candidate with the fewest timed samples -- radix digit widths of 6, 8, 10
and 11 bits for every sort, several tile sizes for fused runs -- so running
the same circuit repeatedly walks through all of them.  The state must be
bit-identical to the untuned one on every repetition (stable LSD sorts give
one order whatever the digit width), the measured choices must appear in the
export, and a new state must take them over through import or the cache
file named by SQS_TUNE_CACHE."""
import os

import numpy as np
import pytest

from paper_2503_15118_gb300 import workloads as W
from tests.test_fused_runs import _run_circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


def _exact(st):
    lo, hi, a = st.export()
    return lo.copy(), hi.copy(), a.copy()


def _same(x, y):
    return all(np.array_equal(p, q) for p, q in zip(x, y))


def _merge_circuit(wide, n_gates, seed):
    """A merge-heavy random circuit whose state stays at or below 2^16
    branches: random gates over 16 qubits, or (wide) over 13 qubits plus a
    64-bit register that takes three CNOT copies half way through, so the
    keys need two words and the copied bits keep up to 8x more branches
    apart."""
    base = [5, 5, 3] if wide else [6, 6, 4]
    c = W.random_circuit(base, n_gates, seed=seed, kinds=("x", "cx", "ccx", "ry", "phase", "h", "add"))
    gates = list(c["gates"])
    widths = list(base)
    if wide:
        widths.append(64)
        half = len(gates) // 2
        gates = gates[:half] + [("x", 3, 20 + 3 * i, ((i, i, 1),)) for i in range(3)] + gates[half:]
    return {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}


def _runs(wide, seed):
    """Fused interference runs; about 0.3-3 million branches."""
    return _run_circuit([40, 40, 6] if wide else [12, 12, 6], seed, n_runs=3, run_len=6, ry_reg=True)


@pytest.mark.parametrize("mode", ["sort_merge", "fused_runs"])
@pytest.mark.parametrize("wide", [False, True])
def test_tuning_walks_every_candidate_bit_identically(sqs, mode, wide):
    if mode == "sort_merge":
        circ = _merge_circuit(wide, 120, seed=9)
        base = sqs.MERGE_SORT
    else:
        circ = _runs(wide, 3 + 86 * wide)
        base = sqs.FUSE_ALWAYS
    ref = sqs.run_circuit(circ, merge=base)
    want = _exact(ref)
    assert ref.nnz() > 2048
    ref.close()
    st = sqs.State(circ["widths"], eps=circ["eps"], merge=base | sqs.AUTOTUNE)
    for rep in range(10):  # 4 candidates x 2 samples, then the choice
        st.reset()
        st.run(circ)
        st.sync()
        assert _same(_exact(st), want), rep
    tuned = st.tune_export()
    assert tuned["gpu"]
    chosen = [e for e in tuned["entries"] if e["choice"] >= 0]
    assert chosen, tuned
    site = "sort_bits" if mode == "sort_merge" else "group_slots"
    assert any(e["site"] == site for e in chosen)
    for e in chosen:
        if e["site"] == "sort_bits":
            assert e["choice"] in (6, 8, 10, 11) and sorted(e["cand"]) == [6, 8, 10, 11]
            assert all(m > 0 for m in e["median_ms"])
    # A new state takes the choices over and computes the same state.
    st2 = sqs.State(circ["widths"], eps=circ["eps"], merge=base | sqs.AUTOTUNE)
    st2.tune_import(tuned)
    got = st2.tune_export()
    assert {(e["site"], e["n_log2"], e["extra"], e["choice"]) for e in got["entries"]} >= \
        {(e["site"], e["n_log2"], e["extra"], e["choice"]) for e in chosen}
    st2.run(circ)
    assert _same(_exact(st2), want)
    st.close()
    st2.close()


def test_cache_file_round_trip(sqs, tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SQS_TUNE_CACHE", str(path))
    circ = _merge_circuit(False, 120, seed=9)
    widths = circ["widths"]
    st = sqs.State(widths, eps=circ["eps"], merge=sqs.MERGE_SORT | sqs.AUTOTUNE)
    for _ in range(10):
        st.reset()
        st.run(circ)
        st.sync()
    st.close()  # writes the cache
    assert path.exists()
    import json
    data = json.loads(path.read_text())
    assert any(e["choice"] >= 0 for e in data["entries"])
    st2 = sqs.State(widths, eps=circ["eps"], merge=sqs.MERGE_SORT | sqs.AUTOTUNE)
    loaded = st2.tune_export()  # read when the state was created
    assert {(e["site"], e["n_log2"], e["extra"], e["choice"]) for e in loaded["entries"]} == \
        {(e["site"], e["n_log2"], e["extra"], e["choice"]) for e in data["entries"] if e["choice"] >= 0}
    st2.close()
    # Entries of another GPU are ignored.
    other = dict(data, gpu="another device")
    monkeypatch.delenv("SQS_TUNE_CACHE")
    st3 = sqs.State(widths, eps=circ["eps"], merge=sqs.MERGE_SORT)
    st3.tune_import(other)
    assert st3.tune_export()["entries"] == []
    st3.close()


@pytest.mark.parametrize("bits", [6, 10, 11])
@pytest.mark.parametrize("amp32", [False, True])
@pytest.mark.parametrize("wide", [False, True])
def test_every_digit_width_sorts_identically(sqs, monkeypatch, bits, amp32, wide):
    """Each supported digit width, forced for every sort (SQS_SORT_BITS): the
    sort merge, fused runs and the sorted export give the state of 8-bit
    digits bit for bit."""
    circ = _merge_circuit(wide, 150, seed=13 + bits)
    runs = _runs(wide, 21 + bits)
    want = []
    for c, merge in ((circ, sqs.MERGE_SORT), (runs, sqs.FUSE_ALWAYS)):
        ref = sqs.run_circuit(c, amp32=amp32, merge=merge)
        want.append((_exact(ref), ref.nnz()))
        ref.close()
    monkeypatch.setenv("SQS_SORT_BITS", str(bits))
    for (c, merge), (w, n) in zip(((circ, sqs.MERGE_SORT), (runs, sqs.FUSE_ALWAYS)), want):
        st = sqs.run_circuit(c, amp32=amp32, merge=merge)
        assert st.nnz() == n
        assert _same(_exact(st), w)
        st.close()

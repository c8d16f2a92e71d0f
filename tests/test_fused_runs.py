"""Fused runs of interference steps (Sec. II.D.2: each coherent group -- the
branches equal on every idle qubit -- transformed as one vector).

A fused run must give the state of its steps run one by one, bit for bit,
peak count included, in every storage type and key width; these tests run
the same circuits with every held run fused (SQS_FUSE_ALWAYS) and with
fusion off (SQS_FUSE_OFF), check
that fused runs actually happened (stats and trace), and compare both with
the oracle.  Runs are built to stress the group kernel: the longest run (12
steps), groups sparse and dense, several batches of groups per bucket,
controls and register-valued angles on idle qubits, steps that must break a
run, nothing pruned under eps = 0, and graph capture (steps alone).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import workloads as W
from tests.helpers import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


def _both(sqs, circ, amp32=False, merge=0):
    # FUSE_ALWAYS: every held run executes fused, also on states too small
    # for the cost estimate to choose it.
    on = sqs.State(circ["widths"], amp32=amp32, eps=circ.get("eps", 1e-14),
                   merge=merge | sqs.FUSE_ALWAYS)
    on.trace_enable(1 << 14)
    on.run(circ)
    off = sqs.State(circ["widths"], amp32=amp32, eps=circ.get("eps", 1e-14),
                    merge=merge | sqs.FUSE_OFF)
    off.run(circ)
    return on, off


def _identical(on, off):
    d1, d2 = on.to_dict(), off.to_dict()
    assert set(d1) == set(d2)
    assert all(d1[k] == d2[k] for k in d1)  # both components, exactly
    assert on.peak_nnz() == off.peak_nnz()
    return d1


def _check_oracle(circ, got, amp32):
    ref = oracle.run_circuit(circ).to_dict()
    if amp32:
        assert compare_states(got, ref, atol=1e-5, band=1e-5) >= 1 - 1e-6
    else:
        assert set(got) == set(ref)
        assert compare_states(got, ref, eps=circ.get("eps", 1e-14), atol=1e-12) >= 1 - 1e-12


def _u(rng):
    """A seeded random 2x2 unitary (QR of a complex Gaussian)."""
    z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _run_circuit(widths, seed, n_runs, run_len, with_ctrls=True, ry_reg=False):
    """Runs of interference steps on distinct targets of registers 0 and 1,
    controls (values 0 and 1) on register 2, and permutations between runs
    that entangle the registers."""
    rng = np.random.default_rng(seed)
    gates = [("h", 2, b, ()) for b in range(widths[2])]
    targets = [(r, b) for r in (0, 1) for b in range(widths[r])]
    for _ in range(n_runs):
        pick = rng.choice(len(targets), size=min(run_len, len(targets)), replace=False)
        for i in pick:
            r, b = targets[i]
            ctrls = ()
            if with_ctrls and rng.random() < 0.4:
                ctrls = ((2, int(rng.integers(widths[2])), int(rng.integers(2))),)
            kind = rng.integers(4 if ry_reg else 3)
            if kind == 0:
                gates.append(("h", r, b, ctrls))
            elif kind == 1:
                gates.append(("ry", r, b, float(rng.uniform(0, 2 * math.pi)), ctrls))
            elif kind == 2:
                gates.append(("u1q", r, b, _u(rng), ctrls))
            else:
                gates.append(("ry_reg", r, b, 2, 0.37, 0.11, ctrls))
        gates.append(("x", 1, int(rng.integers(widths[1])), ((0, int(rng.integers(widths[0])), 1),)))
        gates.append(("add", 0, 2, 0, ()))
        gates.append(("phase", ((1, 0, 1),), 0.3))
    return {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}


@pytest.mark.parametrize("amp32", [False, True])
@pytest.mark.parametrize("widths", [[6, 5, 3], [40, 40, 6]])
def test_runs_bit_identical_to_steps(sqs, widths, amp32):
    circ = _run_circuit(widths, 7 + sum(widths), n_runs=4, run_len=5, ry_reg=True)
    on, off = _both(sqs, circ, amp32)
    got = _identical(on, off)
    st = on.stats()
    assert st["runs_fused"] >= 4 and st["steps_fused"] >= 4 * 2
    assert off.stats()["runs_fused"] == 0
    names = [r[0] for r in on.trace_read()[0]]
    assert names.count("k_group") == st["runs_fused"]
    _check_oracle(circ, got, amp32)


@pytest.mark.parametrize("amp32", [False, True])
def test_longest_run_and_split(sqs, amp32):
    """RY on 14 qubits of one register from |0>: a run of 12 (the maximum)
    then a run of 2; then the inverse rotations in reverse order, which
    cancel back to one branch (the residues fall below eps)."""
    widths = [16, 4]
    th = [0.2 + 0.15 * b for b in range(14)]
    gates = [("ry", 0, b, th[b], ()) for b in range(14)]
    gates += [("x", 1, 0, ())]
    gates += [("ry", 0, b, -th[b], ()) for b in reversed(range(14))]
    circ = {"widths": widths, "eps": 1e-14 if not amp32 else 1e-6, "tables": [], "gates": gates}
    on, off = _both(sqs, circ, amp32)
    got = _identical(on, off)
    assert on.stats()["runs_fused"] == 4 and on.stats()["steps_fused"] == 28
    assert on.peak_nnz() == 2 ** 14
    assert set(got) == {1 << 16}
    _check_oracle(circ, got, amp32)


@pytest.mark.parametrize("amp32", [False, True])
def test_sparse_groups_many_batches(sqs, amp32):
    """256 groups of one branch each, then RY on 12 qubits: each group grows
    to 4096 entries, so a bucket holding more than two (four in FP32) groups
    transforms them in several batches of the dense area (2^20 branches out)."""
    widths = [12, 8]
    gates = [("h", 1, b, ()) for b in range(8)]
    gates += [("x", 0, 3, ((1, 0, 1),)), ("x", 0, 7, ((1, 1, 1),))]  # ends the run
    gates += [("ry", 0, b, 0.3 + 0.1 * b, ()) for b in range(12)]
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    on, off = _both(sqs, circ, amp32)
    _identical(on, off)
    assert on.nnz() == 2 ** 20
    assert on.stats()["runs_fused"] == 2
    # Sampled against the oracle's definition: amplitude = product over the
    # 12 rotations of the entry selected by the branch's bit (input bit from
    # the X gates), times 2^-4 from the H on register 1.
    d = on.to_dict()
    rng = np.random.default_rng(0)
    for key in rng.choice(list(d), size=200, replace=False):
        key = int(key)
        top = key >> 12
        inp = ((top & 1) << 3) | (((top >> 1) & 1) << 7)
        amp = 2.0 ** -4
        for b in range(12):
            c, s = math.cos((0.3 + 0.1 * b) / 2), math.sin((0.3 + 0.1 * b) / 2)
            m = np.array([[c, -s], [s, c]])
            amp *= m[(key >> b) & 1, (inp >> b) & 1]
        assert abs(d[key] - amp) < (1e-6 if amp32 else 1e-14)


def test_steps_that_break_a_run(sqs):
    """A step whose control sits on a target of the open run, a step on a
    target already in the run, an angle register that overlaps a target, and
    a queued permutation each end the run; the results stay bit-identical."""
    widths = [6, 6, 4]
    gates = [("h", 0, b, ()) for b in range(4)]
    gates += [("h", 1, 0, ((0, 1, 1),))]      # control on a run target: new run
    gates += [("h", 1, 1, ()), ("h", 1, 0, ())]  # target 1.0 again: new run
    gates += [("ry_reg", 2, 0, 1, 0.5, 0.0, ())]  # angle register 1 holds targets: new run
    gates += [("h", 2, 1, ()), ("x", 0, 5, ()), ("h", 2, 2, ())]  # permutation between
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    on, off = _both(sqs, circ)
    got = _identical(on, off)
    _check_oracle(circ, got, False)


def test_nothing_pruned_at_eps_zero(sqs):
    """eps = 0: the cancelling children of U^dag after U stay (as rounding
    residues or exact zeros), in a fused run as in the steps one by one."""
    r = 2 ** -0.5
    U = np.array([[r, 1j * r], [1j * r, r]])  # U[1][0] = i U[0][0]: no copy pairs
    widths = [4, 4]
    gates = [("u1q", 0, 0, U, ()), ("u1q", 0, 1, U, ()), ("x", 1, 0, ()),
             ("u1q", 0, 1, U.conj().T, ()), ("u1q", 0, 0, U.conj().T, ())]
    circ = {"widths": widths, "eps": 0.0, "tables": [], "gates": gates}
    on, off = _both(sqs, circ)
    got = _identical(on, off)
    assert len(got) == 4 and on.stats()["runs_fused"] == 2
    ref = oracle.run_circuit(circ).to_dict()
    assert set(got) == set(ref)


def test_graph_capture_runs_steps_alone(sqs):
    """A fused run waits for the group count, so a capture runs each step
    alone; the replayed state equals the fused eager one, bit for bit."""
    import torch
    widths = [8, 8, 4]
    circ = _run_circuit(widths, 3, n_runs=3, run_len=6)
    stream = torch.cuda.Stream()
    g = sqs.State(widths, stream=stream.cuda_stream, merge=sqs.FUSE_ALWAYS)
    graph = g.capture(circ, static_bound=1 << 20)
    assert g.stats()["runs_fused"] == 0
    graph.launch()
    replay = g.to_dict()
    eager = sqs.run_circuit(circ, merge=sqs.FUSE_ALWAYS)
    assert eager.stats()["runs_fused"] >= 3
    d = eager.to_dict()
    assert set(replay) == set(d) and all(replay[k] == d[k] for k in d)
    graph.close()


def test_walk_uses_fused_runs(sqs):
    """The linear-system walk's reflections about |b> are runs of H on the
    system register: fused, and the walk's state unchanged."""
    from paper_2503_15118_gb300 import qlss as Q
    cfg = Q.config4(seed=6, N=16, half_band=2, kappa=5.0, T=20)
    circ = Q.walk_circuit(cfg, n_steps=3)
    on, off = _both(sqs, circ)
    got = _identical(on, off)
    assert on.stats()["runs_fused"] >= 6
    _check_oracle(circ, got, False)


def test_config1_address_superposition_fused(sqs):
    stored = W.config1(seed=1)
    on, off = _both(sqs, stored)
    _identical(on, off)
    assert on.stats()["runs_fused"] >= 1


def test_cost_estimate_chooses(sqs):
    """By default a held run executes fused only when it moves less memory:
    a run of eight expansions on 2^16 branches over few varying qubits is
    fused; the same run on a 20-qubit state below 2^14 branches is not."""
    widths = [16, 8, 8]
    big = [("h", 0, b, ()) for b in range(16)]              # 2^16 branches
    big += [("x", 1, 0, ((0, 0, 1),))]                       # ends the run
    big += [("ry", 2, b, 0.4 + 0.1 * b, ()) for b in range(8)]
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": big}
    g = sqs.run_circuit(circ)
    g.flush()  # the last run is held until something must execute
    assert g.stats()["runs_fused"] >= 1
    small = {"widths": [4, 8, 8], "eps": 1e-14, "tables": [],
             "gates": [("h", 0, b, ()) for b in range(4)]}
    g = sqs.run_circuit(small)
    g.flush()
    assert g.stats()["runs_fused"] == 0

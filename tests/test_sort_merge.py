"""The radix-sort merge and the measured per-step merge choice.

The sort merge (SQS_MERGE_SORT) brings the members of each coherent pair
together with LSD radix passes over the pair-class key and combines
neighbours; the bucket merge finds them in shared-memory hash tables.  Both
evaluate the same 2x2 expression on the same operands, so their states must
be identical bit for bit (as sets of keys with amplitudes), and both must
match the oracle.  SQS_MERGE_TUNED times both on the first steps of each size
class and keeps the faster: its states are the same again.
"""
import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import workloads as W
from tests.helpers import compare_states

pytestmark = pytest.mark.gpu

SORT, BUCKET, TUNED = 8, 0, 32


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


KINDS = ("x", "cx", "ccx", "ry", "cry", "phase", "cphase", "h", "ch", "u1q", "cu1q", "diag",
         "adiag", "add", "sub", "swap")


@pytest.mark.parametrize("widths,seed", [([5, 5, 6], 11), ([6, 6, 6], 12), ([20, 32, 32], 13),
                                         ([16, 16, 16, 16], 14)])
@pytest.mark.parametrize("amp32", [False, True])
def test_sort_and_bucket_states_bit_identical(sqs, widths, seed, amp32):
    n_gates = 120 if sum(widths) <= 24 else 60
    kinds = KINDS if sum(widths) <= 24 else ("x", "cx", "ccx", "add", "phase") * 4 + ("h", "ry")
    circ = W.random_circuit(widths, n_gates, seed, kinds=kinds)
    a = sqs.run_circuit(circ, amp32=amp32, merge=SORT)
    b = sqs.run_circuit(circ, amp32=amp32, merge=BUCKET)
    da, db = a.to_dict(), b.to_dict()
    assert set(da) == set(db)
    assert all(da[k] == db[k] for k in da)  # exact equality of both components
    sa, sb = a.stats(), b.stats()
    assert sa["steps_hash"] == 0 and sb["steps_sort"] == 0
    assert (sa["steps_sort"] + sa["steps_expand"] + sa["steps_fold"]
            == sb["steps_hash"] + sb["steps_expand"] + sb["steps_fold"] + sb["steps_fused"])
    o = oracle.run_circuit(circ)
    f = compare_states(da, o.to_dict(), atol=1e-5 if amp32 else 1e-12,
                       band=1e-5 if amp32 else 1e-12)
    assert f >= (1 - 1e-6 if amp32 else 1 - 1e-10)


def test_sort_passes_skip_constant_bits(sqs):
    """16 superposed qubits on a 64-qubit key: the class key of a step on one
    of them varies in 15 bits, two 8-bit digits; the 48 untouched qubits are
    known constant and cost no pass."""
    widths = [8, 8, 48]
    gates = [("h", r, b, ()) for r in (0, 1) for b in range(8)]           # expand path
    gates += [("x", 1, 3, ((0, 2, 1),)), ("add", 0, 1, 0, ()), ("phase", ((1, 6, 1),), 0.4)]
    gates += [("h", 0, 5, ()), ("ry", 1, 2, 0.3, ((0, 0, 1),))]           # merge steps
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    g = sqs.State(widths, merge=SORT)
    g.trace_enable(4096)
    g.run(circ)
    recs, _ = g.trace_read()
    names = [r[0] for r in recs]
    assert names.count("k_expand") == 16
    assert names.count("k_rsort_merge") == 2
    assert names.count("k_rsort_pass") == 4  # two digits per step
    o = oracle.run_circuit(circ)
    got, ref = g.to_dict(), o.to_dict()
    assert set(got) == set(ref)
    assert compare_states(got, ref) > 1 - 1e-12


@pytest.mark.parametrize("n", [1, 2047, 2048, 2049, 65537, 300000])
@pytest.mark.parametrize("pair_fraction", [0.0, 0.5, 1.0])
def test_sort_tiles_and_ragged_tails(sqs, n, pair_fraction):
    """Imported states have no known-constant bit: 8 full passes over 63 bits,
    tiles of 2048 with a ragged last tile, one- and many-tile scans."""
    widths = [16, 16, 16, 16]
    lo, hi, amps = W.random_state(widths, n, seed=n + int(10 * pair_fraction),
                                  pair_fraction=pair_fraction, target=(2, 9))
    g = sqs.State(widths, merge=SORT)
    g.import_(lo, hi, amps)
    o = oracle.OracleState(widths)
    o.import_(lo, hi, amps)
    for gate in [("h", 2, 9, ()), ("u1q", 0, 3, np.array([[0.6, 0.8j], [0.8j, 0.6]]), ())]:
        g.apply(gate)
        o.apply(gate)
    got, ref = g.to_dict(), o.to_dict()
    assert set(got) == set(ref)
    assert compare_states(got, ref) > 1 - 1e-10
    assert g.stats()["steps_sort"] == 2


def test_sort_first_pass_applies_fused_run_with_pruning(sqs):
    """Permutations, a phase and an explicit prune queued before the step run
    inside the first radix pass (histogram and scatter), dropping branches."""
    widths = [20, 32, 32]
    lo, hi, amps = W.random_state(widths, 50000, seed=5, pair_fraction=0.5, target=(1, 7))
    amps = amps.copy()
    amps[::3] *= 1e-16  # a third of the branches fall under the threshold
    gates = [("x", 2, 4, ((0, 1, 1),)), ("add", 2, 1, 0, ()), ("phase", ((0, 3, 1),), 1.1),
             ("prune", 1e-14), ("swap", 1, 2, ()), ("h", 2, 7, ())]
    g = sqs.State(widths, merge=SORT)
    g.import_(lo, hi, amps)
    o = oracle.OracleState(widths)
    o.import_(lo, hi, amps)
    for gate in gates:
        g.apply(gate)
        o.apply(gate)
    got, ref = g.to_dict(), o.to_dict()
    assert set(got) == set(ref)
    assert compare_states(got, ref) > 1 - 1e-10


def test_tuned_choice_measures_both_paths(sqs):
    """The measured choice times each merge on the first steps of a size
    class, then keeps one; whichever it keeps, the state is the bucket
    merge's, bit for bit."""
    circ = W.config2(seed=2, n_branch=14, n_perm=200, n_cancel=4)
    # Without the host-proven shortcuts every interference step merges, so
    # size classes recur and both paths get timed.
    t = sqs.run_circuit(circ, merge=TUNED | sqs.MERGE_PLAIN)
    b = sqs.run_circuit(circ, merge=BUCKET | sqs.MERGE_PLAIN)
    st = t.stats()
    assert st["steps_sort"] >= 1 and st["steps_hash"] >= 1
    dt, db = t.to_dict(), b.to_dict()
    assert set(dt) == set(db)
    assert all(dt[k] == db[k] for k in dt)

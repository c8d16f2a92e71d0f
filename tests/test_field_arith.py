"""Register arithmetic in the fused-run interpreter, field by field.

The op-major interpreter adds and subtracts in place: the constant, or the
source register moved onto the destination's position with one shift, is
added to the masked destination field and the carries out of the field are
masked off.  These tests drive every (destination, source) pair of registers
of unequal, odd widths -- a source wider and narrower than the destination,
left of it and right of it, registers straddling the 64-bit word boundary of
two-word keys, controls on other registers -- through both places the
interpreter runs: an in-place pass (the flush) and the partition of the next
merge step.  Each state is compared with the oracle element by element.
"""
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


def _ops(widths, seed):
    rng = np.random.default_rng(seed)
    nr = len(widths)
    gates = []
    for d in range(nr):
        for s in range(nr):
            if s == d:
                continue
            other = [r for r in range(nr) if r not in (d, s)]
            ctrl = ((other[0], int(rng.integers(widths[other[0]])), int(rng.integers(2))),) \
                if other and rng.random() < 0.5 else ()
            gates.append(("add", d, s, 0, ctrl))
            gates.append(("sub", d, s, 0, ()))
        gates.append(("add", d, -1, int(rng.integers(0, 2 ** min(widths[d], 62))), ()))
        gates.append(("sub", d, -1, int(rng.integers(0, 2 ** min(widths[d], 62))), ()))
    return gates


@pytest.mark.parametrize("widths", [[7, 33, 24], [20, 32, 32], [13, 64, 5], [3, 29, 64, 31]])
@pytest.mark.parametrize("where", ["in_place", "partition"])
def test_register_add_sub_every_pair(sqs, widths, where):
    n = 70001
    lo, hi, amps = W.random_state(widths, n, seed=sum(widths), pair_fraction=0.5, target=(0, 1))
    gates = _ops(widths, seed=len(widths) * 7 + widths[0])
    if where == "partition":
        gates = gates + [("h", 0, 1, ())]  # the queued run executes inside the partition
    g = sqs.State(widths)
    g.import_(lo, hi, amps)
    o = oracle.OracleState(widths)
    o.import_(lo, hi, amps)
    for gate in gates:
        g.apply(gate)
        o.apply(gate)
    g.flush()
    got, ref = g.to_dict(), o.to_dict()
    assert set(got) == set(ref)
    assert compare_states(got, ref) > 1 - 1e-10
    if where == "partition":
        assert g.stats()["steps_hash"] == 1

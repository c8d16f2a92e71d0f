"""The stored expected values are consistent with what fixes them: the
config-2 golden (written by tests/golden/make_config2_golden.py from the
oracle alone) belongs to the current generator's gate list, holds a
normalised final state of 2^16 branches (eight exact halvings of the 2^24
peak) and a sorted sample of the 2^23-branch mid-circuit state."""
import hashlib
import os

import numpy as np

from paper_2503_15118_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def test_config2_golden_consistent():
    gold = np.load(os.path.join(HERE, "golden", "config2_seed2.npz"))
    circ = W.config2(seed=2)
    assert str(gold["gates_digest"]) == hashlib.sha256(repr(circ["gates"]).encode()).hexdigest()
    assert int(gold["after"]) == len(circ["gates"]) - 7   # right after the first cancelling H
    assert int(gold["peak"]) == 2 ** 24 and int(gold["mid_n"]) == 2 ** 23
    flo, fa = gold["final_lo"], gold["final_amp"]
    assert flo.shape[0] == 2 ** 16 and np.all(np.diff(flo.astype(np.float64)) >= 0)
    assert np.unique(flo).shape[0] == flo.shape[0]
    assert abs(np.sum(np.abs(fa) ** 2) - 1.0) < 1e-12
    mlo, ma = gold["mid_lo"], gold["mid_amp"]
    assert mlo.shape[0] == 2 ** 17 and np.unique(mlo).shape[0] == mlo.shape[0]
    assert np.all(mlo[1:] > mlo[:-1])
    # Stored branches survived pruning, and no amplitude exceeds 1.
    assert np.all(np.abs(ma) >= 1e-14) and np.all(np.abs(ma) <= 1.0)

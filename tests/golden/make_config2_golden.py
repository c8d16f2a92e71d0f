"""Writes config2_seed2.npz: expected values for the large sparse random
circuit (64 qubits in four 16-bit registers, 24 branching gates among 500
permutation and phase gates, then 8 cancelling H; peak 2^24 branches),
computed by the CPU oracle alone (std::map simulator, FP64).

Stored:
  gates_digest   SHA-256 of the gate list, so a changed generator is caught;
  after          number of gates applied for the mid-circuit point (525: the
                 state right after the first cancelling H, which takes the
                 full 2^24-branch state in);
  mid_n          branch count at that point;
  mid_lo, mid_amp  2^17 seeded samples of that state (keys ascending);
  final_lo, final_amp  the whole final state (2^16 branches, keys ascending);
  peak           the oracle's largest branch count over the circuit.

The oracle needs about three minutes on one core.

    python tests/golden/make_config2_golden.py
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2503_15118_gb300 import workloads as W  # noqa: E402

AFTER = 525
N_SAMPLE = 1 << 17
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_seed2.npz")


def gates_digest(circ):
    return hashlib.sha256(repr(circ["gates"]).encode()).hexdigest()


def main():
    circ = W.config2(seed=2)
    t0 = time.time()
    st = oracle.OracleState(circ["widths"], circ.get("eps", 1e-14))
    tables = circ.get("tables", ())
    mid = None
    for i, g in enumerate(circ["gates"]):
        st.apply(g, tables)
        if i + 1 == AFTER:
            lo, hi, amp = st.export()
            assert not hi.any()
            rng = np.random.default_rng(20250318)
            idx = np.sort(rng.choice(lo.shape[0], size=N_SAMPLE, replace=False))
            mid = (lo.shape[0], lo[idx].copy(), amp[idx].copy())
            print(f"after {AFTER} gates: {lo.shape[0]} branches ({time.time() - t0:.0f} s)")
    lo, hi, amp = st.export()
    assert not hi.any()
    np.savez_compressed(OUT, gates_digest=np.array(gates_digest(circ)), after=np.int64(AFTER),
                        mid_n=np.int64(mid[0]), mid_lo=mid[1], mid_amp=mid[2],
                        final_lo=lo, final_amp=amp, peak=np.int64(st.peak()))
    print(f"final: {lo.shape[0]} branches, peak {st.peak()} ({time.time() - t0:.0f} s) -> {OUT}")


if __name__ == "__main__":
    main()

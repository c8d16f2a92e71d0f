"""Shared test helpers: oracle-backed workload construction and comparisons."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2503_15118_gb300 import workloads as W


def build_config1(seed=1, n_gates=200, cap=4096):
    """Config 1 with its nnz cap enforced by the oracle (rejection sampling)."""
    state = {"st": None, "n": 0}

    def accept(circ, g):
        if state["st"] is None:
            state["st"] = oracle.run_circuit(circ)
            state["n"] = len(circ["gates"])
        trial = state["st"].clone()
        trial.apply(g, circ["tables"])
        if trial.nnz() > cap:
            return False
        state["st"] = trial
        return True

    return W.config1(seed=seed, n_gates=n_gates, cap=cap, accept=accept)


def as_dict(lo, hi, amps):
    return {(int(h) << 64) | int(l): complex(a) for l, h, a in zip(lo, hi, amps)}


def compare_states(got, ref, eps=1e-14, atol=1e-12, band=1e-12):
    """Keys must agree exactly except those whose |a| lies within ``band`` of
    the pruning threshold; amplitudes agree within ``atol``.  Returns the
    fidelity |<ref|got>|^2 / (<ref|ref><got|got>)."""
    def near(a):
        return abs(abs(a) - eps) <= band

    for k, a in ref.items():
        if k not in got:
            assert near(a), f"key {k:#x} missing (|a|={abs(a):.3e})"
            continue
        assert abs(got[k] - a) <= atol, f"key {k:#x}: {got[k]} vs {a}"
    for k, a in got.items():
        if k not in ref:
            assert near(a), f"extra key {k:#x} (|a|={abs(a):.3e})"
    ov = sum(np.conj(a) * got.get(k, 0) for k, a in ref.items())
    n1 = sum(abs(a) ** 2 for a in ref.values())
    n2 = sum(abs(a) ** 2 for a in got.values())
    if n1 == 0 and n2 == 0:
        return 1.0
    return float(abs(ov) ** 2 / (n1 * n2))

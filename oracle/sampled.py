"""One-by-one amplitudes of a single-qubit operation on a large sparse input.
TEST INFRASTRUCTURE ONLY.

For an input state given as arrays (keys, amplitudes) too large for the
std::map oracle, psi'(x) = sum_s U[x_t][s] psi(x with bit t := s) (the
definition the oracle's u1q follows, Sec. II.D.2) is evaluated for a chosen
set of output keys x by looking the two inputs up in the sorted key array.
Keys here are one 64-bit word.
"""
from __future__ import annotations

import numpy as np


class SortedState:
    def __init__(self, keys, amps):
        order = np.argsort(keys, kind="stable")
        self.keys = np.asarray(keys, np.uint64)[order]
        self.amps = np.asarray(amps, np.complex128)[order]

    def lookup(self, x):
        x = np.asarray(x, np.uint64)
        i = np.searchsorted(self.keys, x)
        i = np.minimum(i, self.keys.shape[0] - 1)
        hit = self.keys[i] == x
        return np.where(hit, self.amps[i], 0.0)


def u1q_amplitudes(state, t, U, xs):
    """psi'(x) for every x in xs (no controls)."""
    U = np.asarray(U, np.complex128).reshape(2, 2)
    xs = np.asarray(xs, np.uint64)
    b = np.uint64(1) << np.uint64(t)
    x0 = xs & ~b
    x1 = xs | b
    row = ((xs >> np.uint64(t)) & np.uint64(1)).astype(np.int64)
    return U[row, 0] * state.lookup(x0) + U[row, 1] * state.lookup(x1)


def pair_class_count(keys, t):
    """Number of distinct pair classes (key with bit t cleared)."""
    b = np.uint64(1) << np.uint64(t)
    return int(np.unique(np.asarray(keys, np.uint64) & ~b).shape[0])

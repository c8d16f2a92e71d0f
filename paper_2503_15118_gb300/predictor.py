"""Training traces and training of the learned capacity predictor.

Traces come from the simulator itself: circuits run in exact-sizing mode with
recording on, which stores each interference step's structural features and
its measured log2(branches after / branches before).  Training runs on the
device through sqs_predictor_train (hand-written forward, backward and Adam
kernels).
"""
from __future__ import annotations

import numpy as np

from . import sqs as S
from . import workloads as W


def training_circuits(seeds=range(100, 124)):
    """Seeded circuits shaped like the benchmark workloads (other seeds)."""
    out = []
    kinds = ("x", "cx", "ccx", "ry", "cry", "phase", "h", "ch", "u1q", "add", "swap")
    for s in seeds:
        out.append(W.config2(seed=s, n_branch=12 + s % 6, n_perm=150 + 10 * (s % 10),
                             n_cancel=4 + s % 3))
        out.append(W.random_circuit([5, 5, 6], 120, s, kinds=kinds))
        out.append(W.config3(seed=s, addr_bits=6 + s % 4, rounds=3))
    return out


def collect(circuits):
    """(X, y) of every interference step of the circuits (exact mode)."""
    Xs, ys = [], []
    for c in circuits:
        st = S.State(c["widths"], eps=c.get("eps", 1e-14))
        st.record(True)
        st.run(c)
        X, y = st.read_records()
        Xs.append(X)
        ys.append(y)
        st.close()
    return np.concatenate(Xs), np.concatenate(ys)


def train(X, y, seed=0, epochs=300, batch=128, lr=3e-3):
    p = S.Predictor(seed=seed)
    loss = p.train(X, y, epochs=epochs, batch=batch, lr=lr)
    return p, loss


def trained_predictor(seed=0):
    """Collects the standard traces and trains a predictor on them."""
    X, y = collect(training_circuits())
    p, loss = train(X, y, seed=seed)
    return p, loss, (X, y)

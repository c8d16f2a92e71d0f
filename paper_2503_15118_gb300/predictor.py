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


def walk_circuits(seeds=range(100, 132), N=1024, steps=2, kappa=10.0):
    """Linear-system walk circuits (config 4's construction) on other seeds:
    the traces the predictor learns config 4 from."""
    from . import qlss
    out = []
    for s in seeds:
        cfg = qlss.config4(seed=s, N=N, half_band=min(8, N // 4), kappa=kappa, T=2000)
        out.append(qlss.walk_circuit(cfg, n_steps=steps))
    return out


def trained_on_walks(seeds=range(100, 132), N=1024, steps=2, seed=0):
    """A predictor trained on walk traces (seeds 100..131 by default)."""
    X, y = collect(walk_circuits(seeds, N, steps))
    p, loss = train(X, y, seed=seed)
    return p, loss, (X, y)

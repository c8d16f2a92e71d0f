"""The learned capacity predictor: kernels against the FP64 reference,
training, learned-sizing parity, the overflow fallback, and what the network
gains over the exact-bound sizing."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2503_15118_gb300 import workloads as W
from tests.helpers import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs
    sqs.load()
    return sqs


@pytest.fixture(scope="module")
def trained(S):
    from paper_2503_15118_gb300 import predictor
    p, loss, data = predictor.trained_predictor(seed=1)
    return p, loss, data


def test_forward_and_gradient_match_fp64_reference(S):
    rng = np.random.default_rng(0)
    p = S.Predictor(seed=3)
    w = rng.normal(scale=0.3, size=S.PRED_PARAMS).astype(np.float32)
    p.set_params(w)
    X = rng.normal(size=(333, S.PRED_FEATURES)).astype(np.float32)
    T = rng.normal(size=333).astype(np.float32)
    y_ref, _, _ = mlp.forward(w.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(p.predict(X) - y_ref)) < 1e-4
    g, loss = p.gradient(X, T)
    g_ref = mlp.gradient(w.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel < 1e-3, rel
    assert abs(loss - mlp.loss(w, X, T)) < 1e-3 * max(1.0, loss)


def test_records_are_the_measured_growth(S):
    c = W.config2(seed=7, n_branch=10, n_perm=80, n_cancel=3)
    st = S.State(c["widths"])
    st.record(True)
    n_before = []
    for g in c["gates"]:
        if g[0] in ("h", "ry"):
            n_before.append(st.nnz())
        st.apply(g)
    X, y = st.read_records()
    assert X.shape == (len(n_before), S.PRED_FEATURES)
    # The cancelling H gates (last ones) halve the count exactly.
    assert np.allclose(y[-3:], -1.0)
    o = oracle.run_circuit(c)
    assert st.nnz() == o.nnz()


def test_training_fits_the_traces(trained):
    p, loss, (X, y) = trained
    assert X.shape[0] > 500
    base = float(np.mean((y - y.mean()) ** 2))
    assert loss < 0.25 * base, (loss, base)


def test_learned_sizing_matches_exact_and_oracle(S, trained):
    p, _, _ = trained
    c = W.config2(seed=2, n_branch=16, n_perm=300, n_cancel=6)
    o = oracle.run_circuit(c)
    g = S.State(c["widths"], learned=True)
    g.set_predictor(p)
    g.run(c)
    assert compare_states(g.to_dict(), o.to_dict()) > 1 - 1e-10
    st = g.stats()
    assert st["learned_steps"] == sum(1 for x in c["gates"] if x[0] in ("h", "ry"))


def test_overflow_falls_back_to_exact(S):
    """A predictor that always predicts a 256-fold shrink undersizes every
    merge: the device flags the overflow and the runtime re-runs the steps at
    the exact size; the result is unchanged."""
    bad = S.Predictor(seed=0)
    w = np.zeros(S.PRED_PARAMS, np.float32)
    w[-1] = -8.0
    bad.set_params(w)
    c = W.config2(seed=3, n_branch=17, n_perm=200, n_cancel=4)
    o = oracle.run_circuit(c)
    g = S.State(c["widths"], learned=True)
    g.set_predictor(bad)
    g.run(c)
    assert compare_states(g.to_dict(), o.to_dict()) > 1 - 1e-10
    assert g.stats()["overflow_reruns"] > 0


def test_learned_sizing_gains_over_exact_bound(S, trained):
    """On the 2^20-peak variant of the large random circuit, the same result
    (bit for bit) with fewer host waits than exact sizing, which must read the
    count back whenever the doubling bound outgrows the buffers, and a small
    fraction of the memory that sizing from that bound alone, without any
    count read-back, would reserve.  Both run without the host-proven
    shortcuts (the copy-pair fold keeps the exact bound tight through the
    cancelling gates, which would hide what sizing has to do)."""
    import torch
    p, _, _ = trained
    c = W.config2(seed=2, n_branch=20, n_perm=500, n_cancel=8)
    res = {}
    for mode in ("exact", "learned"):
        g = S.State(c["widths"], learned=(mode == "learned"), merge=S.MERGE_PLAIN)
        if mode == "learned":
            g.set_predictor(p)
        g.run(c)
        g.sync()
        w0 = g.stats()["host_waits"]
        g.reset()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        g.run(c)
        g.sync()
        t1.record()
        torch.cuda.synchronize()
        st = g.stats()
        res[mode] = (st, st["host_waits"] - w0, t0.elapsed_time(t1), g.to_dict())
    (se, we, te, de), (sl, wl, tl, dl) = res["exact"], res["learned"]
    assert de.keys() == dl.keys()
    assert max(abs(de[k] - dl[k]) for k in de) < 1e-12
    assert wl < we, (wl, we)
    # Sizing from the doubling bound alone: the bound after every branching gate.
    ub, peak_ub = 1, 1
    for x in c["gates"]:
        if x[0] in ("h", "ry"):
            ub = min(2 ** 64, 2 * ub)
            peak_ub = max(peak_ub, ub)
    # Buckets of 2048 slots (1024 branches each on average) plus two arrays
    # of 4096-slot segments per bucket.
    bound_bytes = peak_ub / 1024 * 24 * (2048 + 2 * 4096)
    assert sl["bytes_peak"] < bound_bytes / 100
    print(f"\nexact: {te:.2f} ms, {we} host waits, peak {se['bytes_peak'] / 2**20:.1f} MiB; "
          f"learned: {tl:.2f} ms, {wl} host waits, peak {sl['bytes_peak'] / 2**20:.1f} MiB; "
          f"bound-only sizing would reserve {bound_bytes / 2**30:.3g} GiB")


def test_learned_sizing_on_walks(S):
    """Trained on walk traces of other seeds, learned sizing runs a walk of a
    new seed to the exact-sizing state, bit for bit, with no more host waits."""
    from paper_2503_15118_gb300 import predictor, qlss
    p, loss, (X, _) = predictor.trained_on_walks(seeds=range(100, 106), N=32, steps=2)
    assert X.shape[0] > 100 and loss < 1.0
    cfg = qlss.config4(seed=4, N=32, half_band=4, kappa=10.0, T=2000)
    circ = qlss.walk_circuit(cfg, n_steps=3)
    res = {}
    for mode in ("exact", "learned"):
        g = S.State(circ["widths"], learned=(mode == "learned"))
        if mode == "learned":
            g.set_predictor(p)
        g.run(circ)
        d = g.to_dict()
        res[mode] = (d, g.stats())
    (de, se), (dl, sl) = res["exact"], res["learned"]
    assert set(de) == set(dl) and all(de[k] == dl[k] for k in de)
    assert sl["learned_steps"] > 0
    assert sl["host_waits"] <= se["host_waits"]

"""bench.py's host-side bookkeeping on the CPU, with a stand-in state (the
kernels are not involved): the workload timing loop, its units, the
interference-step roofline arithmetic, and error reporting."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Err(RuntimeError):
    pass


class _FakeState:
    """Counts branches as 1 + the number of interference gates applied."""
    closed = 0

    def __init__(self, widths, capacity_hint=0, stream=None, eps=None, amp32=False, merge=0):
        self.kw = 2 if sum(widths) > 64 else 1
        self.n = 1
        self.runs = 0

    def reset(self):
        self.n = 1

    def run(self, circ):
        for g in circ["gates"]:
            self.apply(g, circ["tables"])

    def apply(self, g, tables=()):
        if bench._interference(g):
            self.n += 1

    def flush(self):
        self.runs += 1

    def sync(self):
        pass

    def nnz(self):
        return self.n

    def peak_nnz(self):
        return self.n

    def trace_enable(self, cap):
        pass

    def trace_read(self, cap=0):
        return [("k_partition", 2, 0.5), ("k_pair", 2, 0.25), ("k_apply_inplace", 3, 9.0)], 3

    def stats(self):
        return {"runs_fused": self.runs}

    def close(self):
        _FakeState.closed += 1


def _fake_sqs(fail=False):
    m = types.SimpleNamespace(SqsError=_Err, FUSE_OFF=128)

    def make(*a, **k):
        if fail:
            raise _Err("cannot allocate")
        return _FakeState(*a, **k)
    m.State = make
    return m


def test_time_workload_units_and_roofline(monkeypatch):
    calls = []

    def fake_timed(st, step, flush, stream, steps):
        for _ in range(steps):
            step()
        calls.append(steps)
        return 2.0  # ms per step

    monkeypatch.setattr(bench, "_timed_steps", fake_timed)
    circ = {"widths": [8, 8], "eps": 1e-14, "tables": [],
            "gates": [("h", 0, 0, ()), ("x", 1, 0, ()), ("ry", 0, 1, 0.3, ()),
                      ("u1q", 1, 1, [[1, 0], [0, 1j]], ())]}  # the last one is diagonal
    args = types.SimpleNamespace(warmup=3, steps=10)
    e = bench.time_workload(_fake_sqs(), circ, 1 << 10, False, 0, types.SimpleNamespace(cuda_stream=0),
                            None, args, 1000.0)
    # Inputs per gate: 1, 2, 2, 3 (the two interference gates add a branch).
    assert e["units_per_step"] == 1 + 2 + 2 + 3
    assert e["value"] == pytest.approx(8 / 2e-3)
    assert calls == [5]
    # Interference gates h (1 -> 2) and ry (2 -> 3): (1+2 + 2+3) * 24 B over
    # 0.75 ms of merge kernels; the in-place launch is not counted.
    r = e["interference_roofline"]
    assert r["kernel_ms_per_step"] == pytest.approx(0.75)
    assert r["achieved"] == pytest.approx(8 * 24 / 0.75e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert e["key_words"] == 1


def test_time_workload_closes_the_state_and_reports_errors(monkeypatch):
    monkeypatch.setattr(bench, "_timed_steps", lambda st, step, f, s, n: 1.0)
    before = _FakeState.closed
    circ = {"widths": [8], "eps": 1e-14, "tables": [], "gates": [("h", 0, 0, ())]}
    args = types.SimpleNamespace(warmup=3, steps=4)
    bench.time_workload(_fake_sqs(), circ, 0, True, 0, types.SimpleNamespace(cuda_stream=0),
                        None, args, 1.0)
    assert _FakeState.closed == before + 1
    with pytest.raises(_Err):
        bench.time_workload(_fake_sqs(fail=True), circ, 0, True, 0,
                            types.SimpleNamespace(cuda_stream=0), None, args, 1.0)


def test_interference_classification():
    assert bench._interference(("h", 0, 0, ()))
    assert bench._interference(("ry_reg", 0, 0, 1, 0.1, 0.0, ()))
    assert not bench._interference(("u1q", 0, 0, [[0, 1], [1, 0]], ()))  # anti-diagonal
    assert not bench._interference(("phase", (), 0.3))
    assert bench._interference(("u1q", 0, 0, [[0.6, 0.8], [0.8, -0.6]], ()))


def test_fp32_error_report():
    """The FP32-against-FP64 report: equal key sets in different orders
    give the fidelity and largest difference of the matched amplitudes;
    differing key sets report the keys only one side holds."""
    import numpy as np
    rng = np.random.default_rng(3)
    n = 1000
    lo = rng.choice(1 << 40, size=n, replace=False).astype(np.uint64)
    hi = rng.integers(0, 4, size=n).astype(np.uint64)
    a = (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(2 * n)
    perm = rng.permutation(n)
    b = a.copy()
    b[5] += 1e-7
    r = bench.fp32_error((lo, hi, a), (lo[perm], hi[perm], b[perm]))
    assert r["keys_equal"] and r["n_f64"] == r["n_f32"] == n
    assert abs(r["max_abs_diff"] - 1e-7) < 1e-12
    ov = np.vdot(a, b)
    want = abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
    assert abs(r["fidelity_vs_f64"] - want) < 1e-12
    # Drop one key from the FP32 side and add one it alone holds.
    keep = np.arange(n) != 7
    lo2 = np.concatenate([lo[keep], np.array([1 << 41], np.uint64)])
    hi2 = np.concatenate([hi[keep], np.array([0], np.uint64)])
    b2 = np.concatenate([a[keep], np.array([0.5j])])
    r = bench.fp32_error((lo, hi, a), (lo2, hi2, b2))
    assert not r["keys_equal"] and r["only_f64"] == 1 and r["only_f32"] == 1
    assert abs(r["only_max_abs"] - max(abs(a[7]), 0.5)) < 1e-15
    assert r["max_abs_diff"] == 0.0


def test_cpu_baseline_repeats_its_prefix():
    """The CPU baseline times the oracle on the gate prefix whose inputs stay
    within the budget, repeating the prefix from a fresh state until at least
    min_seconds are timed; its rate counts every repetition's updates."""
    from paper_2503_15118_gb300 import workloads as W
    circ = W.random_circuit([4, 4, 4], 40, seed=3, kinds=("x", "cx", "h", "ry", "phase"))
    cb1, dt1 = bench.cpu_baseline(circ, budget_nnz=64)
    assert cb1["kind"] == "oracle" and cb1["cores"] == 1 and "1 pass(es)" in cb1["sample"]
    cb2, dt2 = bench.cpu_baseline(circ, budget_nnz=64, min_seconds=0.05)
    assert dt2 >= 0.05
    passes = int(cb2["sample"].split(" pass(es)")[0].split()[-1])
    assert passes >= 1
    upd1 = int(cb1["sample"].split(" updates in")[0].split()[-1])
    upd2 = int(cb2["sample"].split(" updates in")[0].split()[-1])
    assert upd2 == passes * upd1
    assert cb2["value"] == pytest.approx(upd2 / dt2)

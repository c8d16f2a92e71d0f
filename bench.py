#!/usr/bin/env python
"""Benchmark: nonzero-branch updates/s of the sparse-state hot path on GB300.

Workload (one step): the large sparse random circuit -- 64 qubits as four
16-bit registers in one uint64 key, 24 seeded branching gates (16 H, 8 RY)
interleaved with 500 permutation / diagonal-phase gates (CNOT, Toffoli, X,
add-mod-2^16, phase), then 8 re-applied H on the cancel qubits; peak 2^24
branches; prune threshold 1e-14; then the FP64 marginal probabilities of one
register and the norm.  The state starts from |0...0> each step.

value    = sum over gates of the branches each gate processed, divided by the
           device time of the step (CUDA events on the state's stream)
e2e      = the same units over the host wall time of the step through the C
           ABI, including the device->host read of the probabilities
roofline = the dominant kernel's algorithmic bytes / its event-timed duration
           against the measured HBM copy bandwidth
cpu_baseline / --impl reference = the CPU oracle (std::map, FP64, one core) on
           a bounded sample of the same gate list

Multi-GPU: the path does not shard; N ranks run N independent replicas
("replicas only") and value is the sum of their units over the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2503_15118_gb300 import workloads as W  # noqa: E402

METRIC = "nonzero-branch updates/s"
UNIT = "updates/s"
WORKLOAD = ("large sparse random circuit: 64 qubits (4 x 16-bit registers, uint64 keys), "
            "24 branching H/RY + 500 CNOT/Toffoli/X/add-mod-2^16/phase + 8 cancelling H, "
            "peak 2^24 branches, prune eps 1e-14, FP64 marginals of one 16-bit register")
PROB_REG = 0
L2_FLUSH_BYTES = 512 << 20


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("sqs_kernels.cu", "sqs_device.cuh", "sqs_sort.cu", "sqs_internal.h"):
        with open(os.path.join(ROOT, "paper_2503_15118_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes of the kernel's largest launch from the committed ncu
    summary, when it was captured from the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("kernel_source_sha") != kernel_source_sha():
        return None, None
    return e.get("dram_bytes"), e.get("launch")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], None, set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1].split()[0]))
                    mx = float(f[2].split()[0])
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                         "sw_power_cap"]
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# Both CPU timings (cpu_baseline in the main line and the reference arm) run
# the oracle over the same prefix: gates whose inputs hold at most this many
# branches.
CPU_BUDGET_NNZ = 1 << 19


def cpu_baseline(circ, budget_nnz=CPU_BUDGET_NNZ, min_seconds=0.0):
    """Times the oracle (as it stands, one core) on the gate-list prefix whose
    inputs stay at or below budget_nnz branches, repeating the prefix from a
    fresh state until at least min_seconds of CPU work are timed."""
    import oracle
    units, n_gates, passes, dt = 0, 0, 0, 0.0
    while passes == 0 or dt < min_seconds:
        st = oracle.OracleState(circ["widths"], circ["eps"])
        n_gates = 0
        t0 = time.perf_counter()
        for g in circ["gates"]:
            n_in = st.nnz()
            if n_in > budget_nnz:
                break
            st.apply(g, circ["tables"])
            units += n_in
            n_gates += 1
        dt += time.perf_counter() - t0
        passes += 1
        del st
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n_gates} of {len(circ['gates'])} gates of the same circuit "
                      f"(inputs <= {budget_nnz} branches), {passes} pass(es), "
                      f"{units} updates in {dt:.2f} s"}, dt


def _timed_steps(st, step, flush, stream, steps):
    import torch
    ms = []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.mean(ms)


def variants(circ, widths, stream, probs, norm, flush, args, st64):
    """The FP32-storage / learned-sizing form against the plain FP64 form on
    the same workload: updates/s of each and the fidelity of the FP32 result
    to the FP64 one."""

    from paper_2503_15118_gb300 import predictor, sqs
    units = None
    pred, loss, (X, _) = predictor.trained_predictor(seed=0)
    out = {"predictor": {"train_records": int(X.shape[0]), "train_mse": loss}}
    ref = None
    for name, amp32, learned, merge in (
            ("f64_exact", False, False, sqs.MERGE_AUTO), ("f32_exact", True, False, sqs.MERGE_AUTO),
            ("f32_learned", True, True, sqs.MERGE_AUTO), ("f64_learned", False, True, sqs.MERGE_AUTO),
            ("f64_sort_merge", False, False, sqs.MERGE_SORT),
            ("f64_cluster_merge", False, False, sqs.MERGE_CLUSTER),
            ("f64_tuned_merge", False, False, sqs.MERGE_TUNED)):
        st = sqs.State(widths, amp32=amp32, learned=learned, capacity_hint=1 << 25,
                       stream=stream.cuda_stream, eps=circ["eps"], merge=merge)
        if learned:
            st.set_predictor(pred)

        def step():
            st.reset()
            st.run(circ)
            st.probabilities_device(PROB_REG, probs.data_ptr(), norm.data_ptr())

        for _ in range(args.warmup):
            step()
        st.sync()
        s0 = st.stats()
        ms = _timed_steps(st, step, flush, stream, args.steps)
        s1 = st.stats()
        waits = (s1["host_waits"] - s0["host_waits"]) / args.steps
        paths = {k[6:]: (s1[k] - s0[k]) / args.steps
                 for k in ("steps_expand", "steps_hash", "steps_sort", "steps_cluster")}
        lo, hi, a = st.export()
        d = dict(zip(lo.tolist(), a.tolist()))
        if units is None:
            units = BENCH_UNITS[0]
        entry = {"value": units / (ms / 1e3), "ms_per_step": ms,
                 "host_waits_per_step": waits, "bytes_peak": st.stats()["bytes_peak"],
                 "overflow_reruns": st.stats()["overflow_reruns"],
                 "interference_steps_by_path": paths}
        if ref is None:
            ref = d
        else:
            ov = sum(np.conj(v) * d.get(k, 0) for k, v in ref.items())
            n1 = sum(abs(v) ** 2 for v in ref.values())
            n2 = sum(abs(v) ** 2 for v in d.values())
            entry["fidelity_vs_f64"] = float(abs(ov) ** 2 / (n1 * n2))
        out[name] = entry
        st.close()
    pred.close()
    return out


BENCH_UNITS = [0]

# Per-gate microbenchmark: one gate on a seeded random state of N branches
# (64-qubit keys, 4 x 16-bit registers), N on a log grid, with the fraction
# of branches whose partner across the target bit is present set to 0, 0.5
# or 1 for interference gates.  Bytes per unit as in the kernels' table:
# a fused pass reads and writes every branch; an interference step reads
# every input and writes every output.
PER_GATE_SIZES = (1 << 10, 1 << 14, 1 << 18, 1 << 22, 1 << 24)
PER_GATE_KINDS = (
    ("h", ("h", 2, 5, ()), (0.0, 0.5, 1.0)),
    ("ry", ("ry", 1, 9, 0.7, ()), (0.0, 1.0)),
    ("u1q", ("u1q", 3, 3, "U", ()), (0.5,)),
    ("x", ("x", 0, 7, ()), None),
    ("cnot", ("x", 0, 7, ((1, 2, 1),)), None),
    ("toffoli", ("x", 0, 7, ((1, 2, 1), (2, 3, 1))), None),
    ("add", ("add", 1, 2, 0, ()), None),
    ("swap", ("swap", 0, 3, ()), None),
    ("phase", ("phase", ((1, 4, 1),), 0.77), None),
    ("qram_load", ("qload", 0, 1, 0), None),
)


def per_gate(args):
    import numpy as np
    import torch

    from paper_2503_15118_gb300 import sqs
    widths = [16, 16, 16, 16]
    rb = 24
    U = np.array([[0.6, -0.8j], [0.8, 0.6j]])
    table = np.random.default_rng(7).integers(0, 2 ** 16, size=2 ** 16).astype(np.uint16)
    hbm, _ = peaks()
    stream = torch.cuda.Stream()
    st = sqs.State(widths, capacity_hint=1 << 25, stream=stream.cuda_stream, eps=1e-14)
    rows = []
    reps = max(3, min(args.steps, 7))
    for n in PER_GATE_SIZES:
        states = {}
        for name, gate, fracs in PER_GATE_KINDS:
            if gate[0] == "u1q":
                gate = ("u1q", gate[1], gate[2], U, gate[4])
            for pf in (fracs or (None,)):
                key = (pf, gate[1:3] if fracs else None)
                if key not in states:
                    target = (gate[1], gate[2]) if fracs else None
                    states[key] = W.random_state(widths, n, seed=n % 1000 + 17,
                                                 pair_fraction=pf or 0.0, target=target)
                lo, hi, amps = states[key]
                times, n_out = [], 0
                for rep in range(reps + 1):
                    st.import_(lo, hi, amps)
                    st.sync()
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    st.apply(gate, [table])
                    st.flush()
                    b.record(stream)
                    torch.cuda.synchronize()
                    if rep:
                        times.append(a.elapsed_time(b))
                    n_out = st.nnz()
                ms = statistics.median(times)
                byts = (n + n_out) * rb if fracs else 2 * n * rb
                gbs = byts / (ms / 1e3) / 1e9
                rows.append({"gate": name, "n": n, "pair_fraction": pf, "n_out": n_out, "ms": ms,
                             "updates_per_s": n / (ms / 1e3), "gb_per_s": gbs,
                             "frac_hbm": gbs / hbm})
    # The shortcut paths on states built by H on fresh qubits: an H on a
    # fresh (constant) qubit expands every branch (k_expand); an H on a qubit
    # expanded earlier and left untouched folds each pair from its bit-0
    # member (k_fold), alone or after m fused CNOTs on other qubits.
    for n_log2 in (20, 22, 24):
        n = 1 << n_log2
        prep = [("h", q // 16, q % 16, ()) for q in range(n_log2)]
        cases = [("expand_h", [("h", 3, 15, ())], 2 * n),
                 ("fold_h", [("h", 0, 0, ())], n // 2)]
        for m in (4, 16):
            ops = [("x", 2 + (j % 2), (j * 5) % 16, ((1 + (j % 3) // 2, (j * 7 + 3) % 16, 1),))
                   for j in range(m)]
            cases.append((f"fold_h_after_{m}_cnots", ops + [("h", 0, 0, ())], n // 2))
        for name, gates, n_expect in cases:
            times, n_out = [], 0
            for rep in range(reps + 1):
                st.reset()
                for gt in prep:
                    st.apply(gt)
                st.sync()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for gt in gates:
                    st.apply(gt)
                st.flush()
                b.record(stream)
                torch.cuda.synchronize()
                if rep:
                    times.append(a.elapsed_time(b))
                n_out = st.nnz()
            ms = statistics.median(times)
            byts = (n + n_out) * rb
            gbs = byts / (ms / 1e3) / 1e9
            rows.append({"gate": name, "n": n, "pair_fraction": None, "n_out": n_out,
                         "n_out_expected": n_expect, "ms": ms,
                         "updates_per_s": n / (ms / 1e3), "gb_per_s": gbs, "frac_hbm": gbs / hbm})
    st.close()
    print(json.dumps({"per_gate": rows, "unit": UNIT, "hbm_gbs": hbm, "reps": reps,
                      "timing": "CUDA events around one gate call and its flush, median"}),
          flush=True)
    return 0


MERGE_KERNELS = ("k_partition", "k_pair", "k_expand", "k_fold", "k_bin", "k_pair_cluster",
                 "k_rsort_pass", "k_rsort_merge")
INTERFERENCE_KERNELS = MERGE_KERNELS + ("k_group_count", "k_group")


def _interference(g):
    """Whether a gate tuple is an interference step (a merge): H, RY, a
    register-valued RY, or a u1q that is neither diagonal nor anti-diagonal."""
    if g[0] in ("h", "ry", "ry_reg"):
        return True
    if g[0] == "u1q":
        import numpy as np
        m = np.asarray(g[3]).reshape(2, 2)
        return not ((m[0, 1] == 0 and m[1, 0] == 0) or (m[0, 0] == 0 and m[1, 1] == 0))
    return False


def _sorted_on_device(lo, hi, amps):
    """The state's keys (two int64 words) and complex128 amplitudes on the
    GPU, ordered by (hi, lo)."""
    import torch
    dev = torch.device("cuda" if torch.cuda.is_available() else "cpu")
    tlo = torch.from_numpy(lo.view(np.int64)).to(dev)
    thi = torch.from_numpy(hi.view(np.int64)).to(dev)
    ta = torch.from_numpy(np.ascontiguousarray(amps)).to(dev)
    # Unsigned order from signed words: flip the sign bits.
    bias = torch.tensor(-(1 << 63), dtype=torch.int64, device=dev)
    _, o1 = torch.sort(tlo ^ bias, stable=True)
    _, o2 = torch.sort((thi ^ bias)[o1], stable=True)
    order = o1[o2]
    return tlo[order], thi[order], ta[order]


def fp32_error(ref, got):
    """The FP32-storage result against the FP64 one (both as exported
    (lo, hi, amps)): fidelity |<ref|got>|^2 / (<ref|ref><got|got>), the
    largest amplitude difference over the keys both hold, and the keys only
    one of them holds (with their largest |a|).  Computed on the GPU."""
    import torch
    rlo, rhi, ra = _sorted_on_device(*ref)
    glo, ghi, ga = _sorted_on_device(*got)
    out = {"n_f64": int(rlo.shape[0]), "n_f32": int(glo.shape[0])}
    if rlo.shape == glo.shape and bool(torch.equal(rlo, glo)) and bool(torch.equal(rhi, ghi)):
        common_r, common_g = ra, ga
        out["keys_equal"] = True
        only_r = only_g = None
    else:
        # Keys both hold: merge the two sorted lists and take adjacent equals.
        tag = torch.cat([torch.zeros_like(rlo), torch.ones_like(glo)])
        lo = torch.cat([rlo, glo])
        hi = torch.cat([rhi, ghi])
        amp = torch.cat([ra, ga])
        bias = torch.tensor(-(1 << 63), dtype=torch.int64, device=lo.device)
        _, o1 = torch.sort(lo ^ bias, stable=True)
        _, o2 = torch.sort((hi ^ bias)[o1], stable=True)
        o = o1[o2]
        lo, hi, amp, tag = lo[o], hi[o], amp[o], tag[o]
        same = (lo[1:] == lo[:-1]) & (hi[1:] == hi[:-1])
        i = torch.nonzero(same).flatten()
        first_r = tag[i] == 0
        common_r = torch.where(first_r, amp[i], amp[i + 1])
        common_g = torch.where(first_r, amp[i + 1], amp[i])
        matched = torch.zeros(lo.shape[0], dtype=torch.bool, device=lo.device)
        matched[i] = True
        matched[i + 1] = True
        only_r = amp[(~matched) & (tag == 0)]
        only_g = amp[(~matched) & (tag == 1)]
        out["keys_equal"] = False
        out["only_f64"] = int(only_r.shape[0])
        out["only_f32"] = int(only_g.shape[0])
        out["only_max_abs"] = float(max(only_r.abs().max().item() if only_r.numel() else 0.0,
                                        only_g.abs().max().item() if only_g.numel() else 0.0))
    ov = torch.sum(torch.conj(common_r) * common_g)
    n1 = torch.sum(ra.abs() ** 2)
    n2 = torch.sum(ga.abs() ** 2)
    out["fidelity_vs_f64"] = float((ov.abs() ** 2 / (n1 * n2)).item())
    out["max_abs_diff"] = float((common_r - common_g).abs().max().item()) if common_r.numel() else 0.0
    return out


def time_workload(sqs, circ, hint, amp32, fuse_off, stream, flush, args, hbm, keep=False):
    """Updates/s of one workload in one form (storage type, fused runs on or
    off), with the HBM-roofline fraction of its interference steps.  With
    keep, also returns the final state (exported)."""
    st = sqs.State(circ["widths"], capacity_hint=hint, stream=stream.cuda_stream,
                   eps=circ["eps"], amp32=amp32, merge=fuse_off)
    try:
        def step():
            st.reset()
            st.run(circ)
            st.flush()  # the operations still queued (and a held run) execute too

        for _ in range(args.warmup):
            step()
        st.sync()
        st.reset()
        n_in = []
        for g in circ["gates"]:
            n_in.append(st.nnz())
            st.apply(g, circ["tables"])
        n_in.append(st.nnz())
        units = sum(n_in[:-1])
        ms = _timed_steps(st, step, flush, stream, max(3, args.steps // 2))
        entry = {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                 "units_per_step": units, "gates": len(circ["gates"]),
                 "peak_nnz": st.peak_nnz(), "key_words": st.kw}
        # Interference-step roofline from one traced step.
        st.trace_enable(1 << 16)
        st.trace_read()
        r0 = st.stats()["runs_fused"]
        step()
        st.sync()
        entry["fused_runs_per_step"] = st.stats()["runs_fused"] - r0
        recs, _ = st.trace_read(cap=1 << 16)
        # Algorithmic bytes: every interference gate reads its input and
        # writes its output once, (N + M) * Rb, whichever kernels (and
        # however many passes, or one fused run for several gates) execute
        # it; time: every launch of those kernels.
        rb = 8 * st.kw + (8 if amp32 else 16)
        byts = sum(float(n_in[i] + n_in[i + 1]) * rb
                   for i, g in enumerate(circ["gates"]) if _interference(g))
        tms = sum(kms for kname, _, kms in recs if kname in INTERFERENCE_KERNELS)
        if tms > 0:
            gbs = byts / (tms / 1e3) / 1e9
            entry["interference_roofline"] = {"achieved": gbs, "peak": hbm, "unit": "GB/s",
                                              "frac": gbs / hbm, "kernel_ms_per_step": tms}
        if keep:
            return entry, st.export()
        return entry
    finally:
        st.close()


def extra_workloads(stream, flush, args):
    """Updates/s of the other workloads:
    - config 1 batched: 2^16 instances of the 20-qubit circuit in one state,
      each loading its own QRAM table, with the HBM-roofline fraction of its
      interference steps (every expand / merge launch: inputs read plus
      outputs written, over their event-timed duration);
    - config 3: the QRAM-heavy register workload (two-word keys, 50 rounds);
    - the linear-system walk (one system, N = 1024), 4 walk steps, for a
      positive-definite and for a non-Hermitian A;
    - the batched walk (256 systems of sizes 8..128), 2 walk steps;
    each in FP64 and FP32 storage.  A workload that fails reports its error
    instead of a rate."""
    from paper_2503_15118_gb300 import qlss, sqs
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "config1_seed1_gates.json")) as f:
        stored = json.load(f)
    cfg4 = W.config4(seed=4)
    cfg5 = qlss.config5(seed=5)
    work = (("config1_batch65536", W.config1_batch(stored, inst_bits=16), 1 << 26),
            ("config3_qram_a20_r50", W.config3(seed=3), 1 << 25),
            ("qlss_walk_N1024_4steps", qlss.walk_circuit(cfg4, n_steps=4), 1 << 23),
            ("qlss_walk_nonherm_N1024_4steps",
             qlss.walk_circuit_nh(qlss.config4_nonherm(seed=4), n_steps=4), 1 << 24),
            ("qlss_batch256_2steps", qlss.batched_circuit(cfg5, 2), 1 << 23))
    hbm, _ = peaks()
    for name, circ, hint in work:
        # The walks also run with every interference step alone, against
        # their fused runs (the reflections about |b>).  The FP32-storage
        # form reports its error against the FP64 form's final state.
        forms = [(False, 0), (True, 0)] + ([(False, sqs.FUSE_OFF)] if name.startswith("qlss") else [])
        ref = None
        for amp32, fuse_off in forms:
            key = name + ("_f32" if amp32 else "_f64") + ("_steps_alone" if fuse_off else "")
            try:
                keep = not fuse_off
                entry = time_workload(sqs, circ, hint, amp32, fuse_off, stream, flush, args, hbm,
                                      keep=keep)
                if keep:
                    entry, final = entry
                    if not amp32:
                        ref = final
                    elif ref is not None:
                        entry["fp32_error"] = fp32_error(ref, final)
                    del final
                out[key] = entry
            except sqs.SqsError as e:  # reported, not fatal to the benchmark line
                out[key] = {"error": str(e)}
        ref = None
    try:
        out["qlss_walk_N1024_4steps_learned"] = learned_walk(stream, flush, args, cfg4)
    except sqs.SqsError as e:  # reported, not fatal to the benchmark line
        out["qlss_walk_N1024_4steps_learned"] = {"error": str(e)}
    out.update(graph_workloads(stream, stored, cfg5, args))
    return out


def learned_walk(stream, flush, args, cfg4):
    """Learned against exact sizing on the N = 1024 walk (4 steps, FP64): the
    predictor is trained on the walk traces of seeds 100..131 (N = 1024, 2
    steps) and run on seed 4.  Reports updates/s, host waits per step,
    overflow re-runs, and whether the two results agree bit for bit."""
    import numpy as np

    from paper_2503_15118_gb300 import predictor, qlss, sqs
    pred, loss, (X, _) = predictor.trained_on_walks()
    circ = qlss.walk_circuit(cfg4, n_steps=4)
    out = {"predictor": {"train_records": int(X.shape[0]), "train_mse": loss,
                         "train_seeds": "100..131", "train_N": 1024}}
    states = {}
    for mode in ("exact", "learned"):
        st = sqs.State(circ["widths"], capacity_hint=1 << 23, stream=stream.cuda_stream,
                       eps=circ["eps"], learned=(mode == "learned"))
        if mode == "learned":
            st.set_predictor(pred)

        def step():
            st.reset()
            st.run(circ)
            st.flush()  # learned mode: the queued steps execute at the flush

        for _ in range(args.warmup):
            step()
        st.sync()
        units = 0
        st.reset()
        if mode == "exact":
            for g in circ["gates"]:
                units += st.nnz()
                st.apply(g, circ["tables"])
            out["units_per_step"] = units
        s0 = st.stats()
        ms = _timed_steps(st, step, flush, stream, max(3, args.steps // 2))
        s1 = st.stats()
        out[mode] = {"value": out["units_per_step"] / (ms / 1e3), "unit": UNIT,
                     "ms_per_step": ms,
                     "host_waits_per_step": (s1["host_waits"] - s0["host_waits"]) / max(3, args.steps // 2),
                     "overflow_reruns": s1["overflow_reruns"], "bytes_peak": s1["bytes_peak"]}
        lo, hi, a = st.export()
        o = np.lexsort((lo, hi))  # storage order depends on the bucket sizes
        states[mode] = (lo[o], hi[o], a[o])
        st.close()
    pred.close()
    (le, he, ae), (ll, hl, al) = states["exact"], states["learned"]
    out["bit_identical"] = bool(le.shape == ll.shape and (le == ll).all() and (he == hl).all()
                                and (ae == al).all())
    return out


def graph_workloads(stream, stored, cfg5, args):
    """The same circuit issued call by call against replayed as one captured
    CUDA graph: config 1 (one instance, launch-bound) and the 256-system
    batched walk (2 steps)."""
    import torch

    from paper_2503_15118_gb300 import qlss, sqs
    out = {}
    c1 = W.config1_from_stored(stored)
    for name, circ in (("config1_single", c1), ("qlss_batch256_2steps", qlss.batched_circuit(cfg5, 2))):
        st = sqs.State(circ["widths"], stream=stream.cuda_stream, eps=circ["eps"])
        st.run(circ)  # tables exist before the capture
        st.sync()
        st.reset()
        units = 0
        for g in circ["gates"]:
            units += st.nnz()
            st.apply(g, circ["tables"])
        peak = st.peak_nnz()
        graph = st.capture(circ, static_bound=2 * peak)
        reps = max(5, args.steps)
        res = {}
        for mode in ("eager", "graph"):
            for _ in range(3):
                if mode == "graph":
                    graph.launch()
                else:
                    st.reset()
                    st.run(circ)
            st.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                if mode == "graph":
                    graph.launch()
                else:
                    st.reset()
                    st.run(circ)
                    st.flush()  # as the capture's end, which runs what is queued
            b.record(stream)
            torch.cuda.synchronize()
            res[mode] = a.elapsed_time(b) / reps
        out[name + "_graph"] = {"value": units / (res["graph"] / 1e3), "unit": UNIT,
                                "ms_per_step": res["graph"], "eager_ms_per_step": res["eager"],
                                "eager_value": units / (res["eager"] / 1e3),
                                "units_per_step": units, "static_bound": 2 * peak}
        graph.close()
        st.close()
    return out


def _with_summary(line):
    """The line with a "summary" of the variants right after "config"."""
    v = line.get("variants", {})

    def rate(key):
        e = v.get(key, {})
        return e.get("value") if isinstance(e, dict) else None

    def frac(key):
        e = v.get(key, {})
        r = e.get("interference_roofline", {}) if isinstance(e, dict) else {}
        return r.get("frac")

    def fid(key):
        e = v.get(key, {})
        f = e.get("fp32_error", {}) if isinstance(e, dict) else {}
        return f.get("fidelity_vs_f64")

    summary = {
        "config1_batch65536_f64_updates_per_s": rate("config1_batch65536_f64"),
        "config1_batch65536_interference_frac": frac("config1_batch65536_f64"),
        "config3_f64_updates_per_s": rate("config3_qram_a20_r50_f64"),
        "config3_f32_updates_per_s": rate("config3_qram_a20_r50_f32"),
        "config3_f32_fidelity_vs_f64": fid("config3_qram_a20_r50_f32"),
        "walk_N1024_f64_updates_per_s": rate("qlss_walk_N1024_4steps_f64"),
        "walk_N1024_f32_fidelity_vs_f64": fid("qlss_walk_N1024_4steps_f32"),
        "batch256_f64_updates_per_s": rate("qlss_batch256_2steps_f64"),
        "config2_f32_vs_f64_ms": [v.get("f32_exact", {}).get("ms_per_step"),
                                  v.get("f64_exact", {}).get("ms_per_step")],
        "config2_f32_learned_vs_f64_exact_ms": [v.get("f32_learned", {}).get("ms_per_step"),
                                                v.get("f64_exact", {}).get("ms_per_step")],
    }
    out = {}
    for k, val in line.items():
        out[k] = val
        if k == "config":
            out["summary"] = summary
    return out


def slowest_rank_ms(total_ms, dist, device):
    """The timed region's length on the slowest rank (all ranks call it)."""
    if not dist:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world, units_per_step, steps, total_ms):
    """Whole-job updates/s of N replicas: every rank processes the same
    units per step, over the slowest rank's time."""
    return world * units_per_step * steps / (total_ms / 1e3)


def run_reference(args, rank):
    if rank != 0:
        return 0
    circ = W.config2(seed=2)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        cpu_baseline(circ, budget_nnz=1 << 12)
    vals, secs = [], []
    for _ in range(args.steps):
        cb, dt = cpu_baseline(circ, budget_nnz=CPU_BUDGET_NNZ)
        vals.append(cb["value"])
        secs.append(dt)
    v = statistics.median(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded prefix on the CPU oracle)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP32-storage / learned-sizing comparison")
    ap.add_argument("--profile-step", action="store_true",
                    help="run exactly one step and exit (the target of ncu captures)")
    ap.add_argument("--profile-walk", action="store_true",
                    help="run |b> and one mid-schedule step of the N = 1024 linear-system walk "
                         "(fused runs included) and exit (the target of ncu captures)")
    ap.add_argument("--amp32", dest="amp32", action="store_true")
    ap.add_argument("--per-gate", action="store_true",
                    help="per-gate microbenchmark (updates/s and HBM fraction per gate kind and size)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.per_gate:
        import torch
        torch.cuda.set_device(local)
        return per_gate(args)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2503_15118_gb300 import sqs
    sqs.load()
    if args.profile_walk:
        from paper_2503_15118_gb300 import qlss
        cfg4 = W.config4(seed=4)
        walk = {"widths": cfg4["widths"], "eps": cfg4["eps"], "tables": cfg4["tables"],
                "gates": cfg4["prep"] + qlss.walk_step(cfg4, cfg4["steps"][cfg4["T"] // 2])}
        stream = torch.cuda.Stream()
        st = sqs.State(walk["widths"], capacity_hint=1 << 23, stream=stream.cuda_stream,
                       eps=walk["eps"])
        st.run(walk)
        st.flush()
        st.sync()
        print(json.dumps({"profile_walk": st.stats()["runs_fused"], "nnz": st.nnz()}))
        st.close()
        return 0
    circ = W.config2(seed=2)
    widths = circ["widths"]
    stream = torch.cuda.Stream()
    st = sqs.State(widths, amp32=args.amp32, capacity_hint=1 << 25, stream=stream.cuda_stream,
                   eps=circ["eps"])
    probs = torch.empty(2 ** widths[PROB_REG], dtype=torch.float64, device="cuda")
    norm = torch.empty(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step():
        st.reset()
        st.run(circ)
        st.probabilities_device(PROB_REG, probs.data_ptr(), norm.data_ptr())

    if args.profile_step:
        step()
        st.sync()
        st.close()
        return 0

    for _ in range(args.warmup):
        step()
    st.sync()

    # Units: the branch count entering each gate (one untimed instrumented pass).
    st.reset()
    n_in, units = [], 0
    for g in circ["gates"]:
        n = st.nnz()
        n_in.append(n)
        units += n
        st.apply(g, circ["tables"])
    n_final = st.nnz()
    peak = st.peak_nnz()
    units += n_final  # the probability reduction reads every branch once
    BENCH_UNITS[0] = units

    # Timed region: per-step events on the state's stream; L2 flushed between steps.
    st.trace_enable(64 * (args.steps + 1) * 8)
    st.trace_read()
    launches0 = st.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i)
                evs[i][0].record(stream)
            step()
            with torch.cuda.stream(stream):
                evs[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = st.launch_count() - launches0
    recs, nrec = st.trace_read(cap=1 << 20)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.mean(step_ms)
    total_ms = sum(step_ms)
    total_ms = slowest_rank_ms(total_ms, dist, "cuda")
    value = replicas_value(world, units, args.steps, total_ms)

    # Dominant kernel (largest share of the traced device time) and the
    # roofline of its largest launch: algorithmic bytes of that launch over
    # its mean event-timed duration across the timed steps.
    per, by_call = {}, {}
    for name, call, kms in recs:
        d = per.setdefault(name, [0, 0.0])
        d[0] += 1
        d[1] += kms
        by_call.setdefault((name, call), []).append(kms)
    dom = max(per, key=lambda k: per[k][1])
    rb = 8 * (2 if sum(widths) > 64 else 1) + (8 if args.amp32 else 16)
    gates = circ["gates"]

    def alg_bytes(name, call):
        gi = call - 2  # API call c (numbered from the reset) is gate c - 2
        if not 0 <= gi < len(gates):
            return 0.0
        nin = n_in[gi]
        nout = n_in[gi + 1] if gi + 1 < len(gates) else n_final
        if name in ("k_pair", "k_fold", "k_expand", "k_rsort_merge", "k_pair_cluster"):
            return float(nin + nout) * rb  # read every input, write every output
        return 2.0 * nin * rb  # partition / fused pass: read and write every branch

    launches_dom = [(alg_bytes(n, c), statistics.mean(v), c) for (n, c), v in by_call.items()
                    if n == dom]
    big_bytes, big_ms, big_call = max(launches_dom)
    hbm, peak_kind = peaks()
    achieved = big_bytes / (big_ms / 1e3) / 1e9 if big_ms > 0 else 0.0
    agg_bytes = sum(b * len(by_call[(dom, c)]) for b, _, c in launches_dom)
    agg_ms = per[dom][1]
    traffic, traffic_launch = recorded_traffic(dom)
    clocks = clk.summary()

    # End to end through the C ABI with a host result buffer.
    e2e_times = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.reset()
        st.run(circ)
        p_host, n2 = st.probabilities(PROB_REG)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times)
    d2h = 8 * (2 ** widths[PROB_REG]) + 8

    # The headline steps are issued back to back: the host issues step i + 1
    # while the device runs step i.  The same steps with a host sync after
    # each (host issue exposed):
    sync_ms = _timed_steps(st, step, flush, stream, args.steps)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-storage/f64-math" if args.amp32 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": f"replicas{world}",
                   "l2": "L2 flushed (512 MB write) between steps; peak state 402 MB",
                   "units_per_step": units, "peak_nnz": peak, "final_nnz": n_final,
                   "gates": len(gates),
                   "step_issue": "steps issued back to back without a host sync between "
                                 "them (the host issues the next step while the device runs "
                                 "this one); synchronised steps in sync_ms_per_step"},
        "sync_ms_per_step": sync_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "kernel": dom,
                     "launch": f"gate {big_call - 2} ({n_in[big_call - 2]} branches in)",
                     "algorithmic_bytes": big_bytes, "launch_ms": big_ms,
                     "traffic_capture": traffic_launch,
                     "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "all_launches_achieved": agg_bytes / (agg_ms / 1e3) / 1e9,
                     "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in per.items()}},
        "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_variants:
        line["variants"] = variants(circ, widths, stream, probs, norm, flush, args, st)
        line["variants"].update(extra_workloads(stream, flush, args))
        # The figures read most, placed early in the line (a reader that keeps
        # only the tail of a long line still has the headline keys).
        line = _with_summary(line)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, _ = cpu_baseline(circ, min_seconds=10.0)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    st.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 storage: keys bit-exact except branches whose |a| lies within 1e-12 of
the pruning threshold, amplitudes within 1e-12 absolute, fidelity >= 1-1e-10.
FP32 storage (every child of an interference step evaluated with
compensated FP32 arithmetic, as accurate as an FP64 sum rounded once to FP32;
a component below 2^-21 of its terms' size is a storage-precision cancellation
and set to zero): fidelity >= 1-1e-6 and amplitudes within 2e-6 absolute (a
float keeps 24 bits: |a| <= 1 rounds to within 6e-8 per stored value, and a
step re-rounds once).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import workloads as W
from tests.helpers import build_config1, compare_states

pytestmark = pytest.mark.gpu

ATOL64 = 1e-12
ATOL32 = 2e-6


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


def _pair(sqs, widths, lo, hi, amps, amp32=False, eps=1e-14, merge=0):
    g = sqs.State(widths, amp32=amp32, eps=eps, merge=merge)
    g.import_(lo, hi, amps)
    o = oracle.OracleState(widths, eps=eps)
    o.import_(lo, hi, amps)
    return g, o


def _check(g, o, amp32=False, fid=None):
    got, ref = g.to_dict(), o.to_dict()
    # FP32 storage: an exact FP64 cancellation of rounded inputs leaves a residue
    # of about 2^-24 |a|, so keys are compared outside that noise floor.
    f = compare_states(got, ref, eps=o.eps, atol=ATOL32 if amp32 else ATOL64,
                       band=ATOL32 if amp32 else 1e-12)
    assert f >= (fid if fid is not None else (1 - 1e-6 if amp32 else 1 - 1e-10))
    return got, ref


W64 = [16, 16, 16, 16]
W128 = [20, 32, 32]

GATES_64 = [
    ("h", 2, 5, ()),
    ("h", 1, 3, ((0, 1, 1), (3, 7, 0))),
    ("ry", 3, 15, 1.234, ()),
    ("ry", 0, 0, -2.5, ((2, 2, 1),)),
    ("u1q", 1, 9, np.array([[0.6, -0.8j], [0.8, 0.6j]]), ()),
    ("u1q", 2, 1, np.array([[np.exp(0.3j), 0], [0, np.exp(-1.1j)]]), ((0, 0, 1),)),
    ("u1q", 2, 1, np.array([[0, np.exp(0.7j)], [np.exp(2.1j), 0]]), ()),
    ("ry_reg", 3, 4, 0, 0.0123, 0.4, ()),
    ("x", 0, 7, ()),
    ("x", 3, 63 - 48, ((0, 2, 1), (1, 5, 1))),
    ("add", 1, 2, 0, ()),
    ("sub", 0, -1, 12345, ((3, 0, 1),)),
    ("swap", 0, 3, ()),
    ("phase", ((1, 4, 1), (2, 8, 0)), 0.77),
    ("muladd", 0, 1, 2, ()),
    ("mulc", 3, 12345, ((0, 2, 1),)),
    ("divxor", 1, 2, 3, ((0, 5, 0),)),
]


MERGES = {"cluster": 16, "bucket": 0, "sort": 8, "tuned": 32}


@pytest.mark.parametrize("merge", list(MERGES))
@pytest.mark.parametrize("n", [1, 33, 2049, 70001])
@pytest.mark.parametrize("gi", range(len(GATES_64)))
def test_single_gate_64bit_keys(sqs, n, gi, merge):
    g = GATES_64[gi]
    target = (g[1], g[2]) if g[0] in ("h", "ry", "u1q", "ry_reg") else None
    lo, hi, amps = W.random_state(W64, n, seed=100 + n + gi, pair_fraction=0.5, target=target)
    gs, os_ = _pair(sqs, W64, lo, hi, amps, merge=MERGES[merge])
    gs.apply(g)
    os_.apply(g)
    _check(gs, os_)


@pytest.mark.parametrize("merge", list(MERGES))
@pytest.mark.parametrize("pair_fraction", [0.0, 1.0])
@pytest.mark.parametrize("n", [5, 4096, 30000, 300000])
def test_h_pairing_extremes(sqs, n, pair_fraction, merge):
    lo, hi, amps = W.random_state(W64, n, seed=7 * n, pair_fraction=pair_fraction, target=(1, 6))
    gs, os_ = _pair(sqs, W64, lo, hi, amps, merge=MERGES[merge])
    gs.h_gate(1, 6)
    os_.h_gate(1, 6)
    _check(gs, os_)
    assert gs.nnz() == os_.nnz()


GATES_128 = [
    ("h", 1, 31, ()),
    ("h", 2, 10, ((0, 19, 1),)),
    ("ry", 2, 31, 0.9, ()),
    ("ry_reg", 1, 2, 0, 2 * math.pi / 2 ** 20, 0.0, ()),
    ("u1q", 0, 19, np.array([[0, 1j], [1j, 0]]), ()),
    ("add", 2, 1, 0, ()),
    ("add", 2, -1, 0xFFFFFFFF, ((0, 3, 0),)),
    ("x", 2, 31, ((1, 0, 1),)),
    ("swap", 1, 2, ()),
    ("phase", ((2, 30, 1),), -1.3),
    ("muladd", 2, 0, 1, ()),
    ("divxor", 1, 2, 0, ()),
    ("mulc", 2, 0xDEADBEEF, ()),
]


@pytest.mark.parametrize("merge", list(MERGES))
@pytest.mark.parametrize("amp32", [False, True])
@pytest.mark.parametrize("n", [3, 2049, 40000])
@pytest.mark.parametrize("gi", range(len(GATES_128)))
def test_single_gate_128bit_keys(sqs, n, gi, amp32, merge):
    g = GATES_128[gi]
    target = (g[1], g[2]) if g[0] in ("h", "ry", "u1q", "ry_reg") else None
    lo, hi, amps = W.random_state(W128, n, seed=300 + n + gi, pair_fraction=0.5, target=target)
    if amp32:
        amps = amps.astype(np.complex64).astype(np.complex128)  # representable input
    gs, os_ = _pair(sqs, W128, lo, hi, amps, amp32=amp32, merge=MERGES[merge])
    gs.apply(g)
    os_.apply(g)
    _check(gs, os_, amp32=amp32)


RHO32 = 2.0 ** -19  # default storage-precision cancellation threshold of FP32 states


def _fp32_children_expected(lo, amps, bit, m):
    """For each output key of a single-qubit step: the FP64 value of every
    component and the size sum_i |u_i a_i| of its terms (the scale of the
    cancellation rule), from FP32-representable inputs."""
    m = np.asarray(m, np.complex128).reshape(2, 2)
    amp = dict(zip(lo.tolist(), amps.tolist()))
    b = 1 << bit
    out = {}
    for k in amp:
        base = k & ~b
        a0, a1 = amp.get(base, 0j), amp.get(base | b, 0j)
        for r in (0, 1):
            v = m[r, 0] * a0 + m[r, 1] * a1
            terms = (m[r, 0].real * a0.real, m[r, 0].imag * a0.imag, m[r, 1].real * a1.real,
                     m[r, 1].imag * a1.imag)
            sx = sum(abs(t) for t in terms)
            terms = (m[r, 0].real * a0.imag, m[r, 0].imag * a0.real, m[r, 1].real * a1.imag,
                     m[r, 1].imag * a1.real)
            sy = sum(abs(t) for t in terms)
            out[base | (b if r else 0)] = (v, sx, sy)
    return out


@pytest.mark.parametrize("merge", ["bucket", "sort"])
@pytest.mark.parametrize("gate", ["h", "ry", "u1q"])
def test_fp32_children_compensated(sqs, gate, merge):
    """FP32 storage: each component of each child is the FP64 value of the
    step on the stored FP32 inputs, rounded once (within one FP32 ulp, plus
    2^-40 of its terms' size for the float-float coefficients), or exactly
    zero when it lies within 2^-21 of its terms' size."""
    widths = [16, 16, 16, 16]
    bit = 16 + 6
    ms = {"h": np.array([[1, 1], [1, -1]]) / np.sqrt(2),
          "ry": np.array([[np.cos(0.35), -np.sin(0.35)], [np.sin(0.35), np.cos(0.35)]]),
          "u1q": np.array([[0.6, -0.8j], [0.8, 0.6j]])}
    m = ms[gate]
    lo, hi, amps = W.random_state(widths, 2049, seed=55, pair_fraction=0.5, target=(1, 6))
    amps = amps.astype(np.complex64).astype(np.complex128)
    st = sqs.State(widths, amp32=True, eps=1e-14, merge=MERGES[merge])
    st.import_(lo, hi, amps)
    st.u1q(1, 6, m)
    got = st.to_dict()
    want = _fp32_children_expected(lo, amps, bit, m)
    ulp = 2.0 ** -23
    n_flushed = 0
    for k, (v, sx, sy) in want.items():
        g = got.get(k, 0j)
        for gv, wv, size in ((g.real, v.real, sx), (g.imag, v.imag, sy)):
            if gv == 0.0 and abs(wv) <= RHO32 * size * (1 + 1e-6):
                n_flushed += wv != 0.0
                continue
            assert abs(gv - wv) <= ulp * abs(wv) + 2.0 ** -40 * size, (k, gv, wv, size)
    assert set(got) <= set(want)


@pytest.mark.parametrize("rho_log2,k,kept", [(-19, 15, True), (-19, 16, True), (-19, 17, True),
                                               (-19, 19, False), (-19, 21, False),
                                               (-21, 19, True), (-21, 21, False), (None, 24, True)])
def test_fp32_cancellation_threshold(sqs, rho_log2, k, kept):
    """H on |0> (amplitude 1) and |1> (amplitude -(1 - 2^-k)): the bit-0 child
    is exactly 2^-k / sqrt(2), from terms of size about sqrt(2), so it lies
    at 2^-(k+1) of its terms' size.  FP32 storage keeps it, accurate to one
    ulp, above the cancellation threshold rho (default 2^-19; 2^-21 set by
    sqs_set_fp32_cancel; the rule off with rho = 0) and sets it to zero below
    (within the rounding the stored inputs carry).  FP64 storage keeps it
    always (eps = 1e-14)."""
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    a1 = -(1.0 - 2.0 ** -k)
    true0 = 2.0 ** -k / np.sqrt(2)
    for amp32 in (True, False):
        st = sqs.State([8], amp32=amp32, eps=1e-14)
        if rho_log2 is not None:
            st.set_fp32_cancel(2.0 ** rho_log2)
        else:
            st.set_fp32_cancel(0.0)
        st.import_(np.array([0, 1], np.uint64), np.zeros(2, np.uint64),
                   np.array([1.0, a1], np.complex128))
        st.u1q(0, 0, H)
        d = st.to_dict()
        assert abs(d[1] - (1.0 - a1) / np.sqrt(2)) < 1e-7
        if amp32 and not kept:
            assert 0 not in d
        else:
            assert abs(d[0].real - true0) <= 2.0 ** -23 * true0 and d[0].imag == 0.0
        st.close()


def test_qram_load_unload(sqs):
    rng = np.random.default_rng(9)
    table8 = rng.integers(0, 256, size=300).astype(np.uint8)      # longer than 2^8: ignored tail
    table32 = rng.integers(0, 2 ** 32, size=2 ** 10, dtype=np.uint64).astype(np.uint32)
    short = rng.integers(0, 2 ** 16, size=100).astype(np.uint16)  # addresses >= 100 read 0
    for widths, tab, areg, dreg in [([8, 8, 4], table8, 0, 1), ([10, 32, 32], table32, 0, 1),
                                    ([10, 12], short, 0, 1)]:
        lo, hi, amps = W.random_state(widths, 3000, seed=len(tab))
        gs, os_ = _pair(sqs, widths, lo, hi, amps)
        for st in (gs, os_):
            st.apply(("qload", areg, dreg, 0), [tab])
        _check(gs, os_)
        for st in (gs, os_):
            st.apply(("qunload", areg, dreg, 0), [tab])
        got = gs.to_dict()
        assert got == {(int(h) << 64) | int(l): complex(a) for l, h, a in zip(lo, hi, amps)}


def _kinds_all():
    return ("x", "cx", "ccx", "ry", "cry", "phase", "cphase", "h", "ch", "u1q", "cu1q", "diag",
            "adiag", "add", "sub", "swap", "qram", "muladd", "mulc", "divxor")


# Wide registers use a mix where branching gates are rare, so the state stays small.
SPARSE_KINDS = ("x", "cx", "ccx", "add", "sub", "swap", "phase", "cphase", "qram", "muladd", "mulc",
                "divxor") * 3 + (
    "h", "ry", "cu1q")


@pytest.mark.parametrize("seed,widths,kinds", [(1, [4, 4, 4], "all"), (2, [6, 6, 4], "all"),
                                               (3, [5, 5, 6], "all"),
                                               (4, [16, 16, 16, 16], "sparse"),
                                               (5, [20, 32, 32], "sparse")])
@pytest.mark.parametrize("amp32", [False, True])
def test_random_circuits(sqs, seed, widths, kinds, amp32):
    rng = np.random.default_rng(seed)
    table = rng.integers(0, 2 ** 16, size=2 ** min(widths[0], 12)).astype(np.uint16)
    n_gates = 150 if kinds == "all" else 90
    circ = W.random_circuit(widths, n_gates, seed,
                            kinds=_kinds_all() if kinds == "all" else SPARSE_KINDS,
                            tables=[table])
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, amp32=amp32)
    f = compare_states(g.to_dict(), o.to_dict(), atol=1e-5 if amp32 else ATOL64,
                       band=1e-5 if amp32 else 1e-12)
    assert f >= (1 - 1e-6 if amp32 else 1 - 1e-10)
    assert g.peak_nnz() == o.peak() or amp32


def test_config1_full(sqs):
    circ = build_config1(seed=1)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ)
    got, ref = g.to_dict(), o.to_dict()
    assert compare_states(got, ref) >= 1 - 1e-10
    assert set(got) == set(ref)
    err = max(abs(got[k] - ref[k]) for k in ref)
    assert err <= ATOL64
    assert g.nnz() <= 4096 and g.peak_nnz() == o.peak()


def test_config1_fp32(sqs):
    circ = build_config1(seed=1)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, amp32=True)
    assert compare_states(g.to_dict(), o.to_dict(), atol=1e-5, band=1e-5) >= 1 - 1e-6


@pytest.mark.parametrize("merge", list(MERGES))
def test_config2_reduced(sqs, merge):
    circ = W.config2(seed=2, n_branch=16, n_perm=300, n_cancel=6)
    n_main = len(circ["gates"]) - 6
    o = oracle.run_circuit(circ, upto=n_main)
    g = sqs.run_circuit(circ, upto=n_main, merge=MERGES[merge])
    assert g.nnz() == o.nnz() == 2 ** 16
    _check(g, o)
    for i, gate in enumerate(circ["gates"][n_main:]):
        g.apply(gate)
        o.apply(gate)
        assert g.nnz() == o.nnz() == 2 ** 16 >> (i + 1)
    _check(g, o)


@pytest.mark.parametrize("amp32", [False, True])
def test_config3_reduced(sqs, amp32):
    circ = W.config3(seed=3, addr_bits=10, rounds=4)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, amp32=amp32)
    got, ref = g.to_dict(), o.to_dict()
    assert compare_states(got, ref, atol=1e-5 if amp32 else ATOL64,
                          band=1e-5 if amp32 else 1e-12) >= (1 - 1e-6 if amp32 else 1 - 1e-10)
    assert g.peak_nnz() == o.peak() or amp32


def test_probabilities(sqs):
    circ = build_config1(seed=1)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ)
    for reg in range(3):
        p, n2 = g.probabilities(reg)
        v, pr = o.probabilities(reg)
        want = np.zeros_like(p)
        want[v.astype(np.int64)] = pr
        assert np.max(np.abs(p - want)) < 1e-13
        assert abs(n2 - o.norm2()) < 1e-13


def test_probabilities_wide_register_128(sqs):
    circ = W.config3(seed=3, addr_bits=8, rounds=2)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ)
    p, n2 = g.probabilities(0)
    v, pr = o.probabilities(0)
    want = np.zeros_like(p)
    want[v.astype(np.int64)] = pr
    assert np.max(np.abs(p - want)) < 1e-13
    _, n2b = g.probabilities(2, with_probs=False)
    assert abs(n2b - o.norm2()) < 1e-13


# ---- edge cases ---------------------------------------------------------------
def test_empty_state_stays_empty(sqs):
    g = sqs.State([8, 8])
    g.h_gate(0, 0)
    assert g.prune(10.0, wait=True) == 0
    g.h_gate(0, 1)
    g.x(1, 3)
    g.ry(1, 2, 0.3)
    assert g.nnz() == 0
    p, n2 = g.probabilities(0)
    assert n2 == 0.0 and not p.any()


def test_full_cancellation(sqs):
    g = sqs.State([4, 4])
    for b in range(4):
        g.h_gate(0, b)
    for b in range(4):
        g.h_gate(0, b)
    assert g.to_dict().keys() == {0}
    assert abs(g.to_dict()[0] - 1) < 1e-15


def test_controls_never_hold(sqs):
    lo, hi, amps = W.random_state(W64, 5000, seed=11)
    lo &= ~np.uint64(1 << 3)  # control bit forced to 0 everywhere
    lo = np.unique(lo)
    amps = amps[: lo.shape[0]]
    gs, os_ = _pair(sqs, W64, lo, np.zeros_like(lo), amps)
    for st in (gs, os_):
        st.h_gate(1, 0, ((0, 3, 1),))
    got, _ = _check(gs, os_)
    assert len(got) == lo.shape[0]


def test_exact_capacity_growth(sqs):
    """Capacity hint far below the final size: buffers grow on demand."""
    g = sqs.State([24], capacity_hint=1)
    for b in range(20):
        g.h_gate(0, b)
    assert g.nnz() == 2 ** 20
    p, n2 = g.probabilities(0, with_probs=False)
    assert abs(n2 - 1) < 1e-12


def test_bad_arguments_leave_state_usable(sqs):
    g = sqs.State([4, 4])
    with pytest.raises(sqs.SqsError):
        g.h_gate(2, 0)
    with pytest.raises(sqs.SqsError):
        g.h_gate(0, 4)
    with pytest.raises(sqs.SqsError):
        g.h_gate(0, 1, ((0, 1, 1),))   # control on the target
    with pytest.raises(sqs.SqsError):
        g.perm([(sqs.PERM_SWAP, 0, 0, 0, 0, ())])
    g.h_gate(0, 1)
    assert g.nnz() == 2


def test_deterministic_as_a_set(sqs):
    circ = W.config2(seed=5, n_branch=14, n_perm=150, n_cancel=4)
    a = sqs.run_circuit(circ).to_dict()
    b = sqs.run_circuit(circ).to_dict()
    assert a == b  # bitwise: each output is a sum of at most two products


@pytest.mark.parametrize("then_branch", [False, True])
def test_long_fused_runs(sqs, then_branch):
    """Hundreds of queued non-interference operations: the runtime splits them
    into launch-sized lists and folds the amplitude factors into tables."""
    rng = np.random.default_rng(77)
    kinds = ("x", "cx", "ccx", "phase", "cphase", "diag", "adiag", "add", "sub", "swap")
    circ = W.random_circuit(W64, 400, 77, kinds=kinds)
    lo, hi, amps = W.random_state(W64, 9000, seed=78)
    gs, os_ = _pair(sqs, W64, lo, hi, amps)
    gates = list(circ["gates"])
    if then_branch:
        gates.append(("h", 1, 1, ()))
    for g in gates:
        gs.apply(g)
        os_.apply(g)
    _check(gs, os_)
    assert rng is not None


@pytest.mark.parametrize("merge", list(MERGES))
def test_constant_target_expand_path(sqs, merge):
    """Targets whose bit the runtime can prove constant (never touched, or
    flipped by X / CNOT whose controls are themselves constant) take the
    expand-only path; targets made non-constant by a superposed control take
    the merge.  Both must match the oracle."""
    widths = [6, 6, 4]
    gates = [
        ("h", 0, 0, ()), ("h", 0, 1, ()),                  # fresh bits: constant
        ("x", 1, 0, ()), ("h", 1, 0, ()),                  # constant after X (value 1)
        ("x", 1, 1, ((1, 2, 1),)), ("h", 1, 1, ()),        # control constant 0: unchanged
        ("x", 2, 0, ((0, 0, 1),)), ("h", 2, 0, ()),        # control superposed: merge path
        ("h", 0, 0, ()),                                   # re-applied H: pairs, merge path
        ("add", 2, 0, 0, ()), ("h", 2, 3, ()),             # arithmetic destination: merge
        ("ry", 1, 5, 0.7, ((0, 1, 1),)),                   # controlled, constant target
    ]
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    o = oracle.run_circuit(circ)
    g = sqs.State(widths, merge=MERGES[merge] | sqs.FUSE_OFF)  # every step alone
    g.trace_enable(4096)
    g.run(circ)
    recs, _ = g.trace_read()
    names = [r[0] for r in recs]
    assert names.count("k_expand") == 5
    got, ref = g.to_dict(), o.to_dict()
    assert compare_states(got, ref) > 1 - 1e-12
    assert set(got) == set(ref)


@pytest.mark.parametrize("merge", list(MERGES))
@pytest.mark.parametrize("last", ["expand", "merge"])
@pytest.mark.parametrize("then", ["prune", "diag_run"])
def test_standalone_compaction_after_wide_segments(sqs, merge, last, then):
    """The expansion, cluster and sort merges leave segments of 2^13 slots;
    a standalone pass that may drop branches (an explicit prune, or a run of
    diagonal gates split over several launches) must read them as such."""
    widths = [8, 8, 8]
    expand = [("h", 0, b, ()) for b in range(8)] + [("h", 1, b, ()) for b in range(5)]
    merge_step = [("x", 2, 0, ((0, 3, 1),)), ("h", 0, 3, ((2, 0, 1),))]
    gates = expand[:8] + merge_step + expand[8:] if last == "expand" else expand + merge_step
    if then == "prune":
        gates += [("prune", 1e-14)]
    else:
        # 12 diagonal gates on distinct bits: more selector bits than one
        # launch's factor table takes, so the first group runs on its own.
        gates += [("u1q", r, b, np.diag([np.exp(0.1j * (b + 1)), np.exp(-0.2j * r)]), ())
                  for r in (0, 1) for b in range(6)]
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, merge=MERGES[merge])
    got, ref = g.to_dict(), o.to_dict()
    assert set(got) == set(ref)
    assert compare_states(got, ref) > 1 - 1e-12


def _plain_and_fast(sqs, circ, amp32=False):
    fast = sqs.State(circ["widths"], amp32=amp32)
    fast.trace_enable(1 << 14)
    fast.run(circ)
    plain = sqs.run_circuit(circ, amp32=amp32, merge=sqs.MERGE_PLAIN)
    return fast, plain


@pytest.mark.parametrize("amp32", [False, True])
def test_copy_pair_fold(sqs, amp32):
    """A qubit expanded by an uncontrolled H-like gate and left untouched has
    every partner, with +-1 times the branch's amplitude: the next gate on it
    folds without a merge, and the state equals the merged one bit for bit."""
    widths = [8, 8, 8]
    gates = [("h", 0, b, ()) for b in range(6)] + [("x", 1, 0, ()), ("h", 1, 0, ())]
    gates += [("x", 2, 1, ((0, 2, 1),)), ("add", 2, -1, 5, ()), ("phase", ((0, 1, 1),), 0.7),
              ("x", 2, 3, ((0, 0, 1),))]
    gates += [("h", 0, 4, ()),                       # +1 pair: fold (the cancelling H)
              ("ry", 1, 0, 0.9, ((0, 5, 1),)),       # -1 pair, controlled consumer: fold
              ("h", 0, 1, ()),                       # read by the phase: merge
              ("h", 0, 0, ())]                       # read as a control: merge
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    fast, plain = _plain_and_fast(sqs, circ, amp32)
    names = [r[0] for r in fast.trace_read()[0]]
    assert names.count("k_fold") == 2
    assert fast.stats()["steps_fold"] == 2 and plain.stats()["steps_fold"] == 0
    df, dp = fast.to_dict(), plain.to_dict()
    assert set(df) == set(dp) and all(df[k] == dp[k] for k in df)
    o = oracle.run_circuit(circ)
    if amp32:
        assert compare_states(df, o.to_dict(), atol=ATOL32, band=ATOL32) >= 1 - 1e-6
    else:
        assert set(df) == set(o.to_dict())
        assert compare_states(df, o.to_dict()) >= 1 - 1e-12


def test_fold_takes_config2_cancellations(sqs):
    circ = W.config2(seed=2, n_branch=16, n_perm=300, n_cancel=6)
    fast, plain = _plain_and_fast(sqs, circ)
    assert fast.stats()["steps_fold"] == 6
    df, dp = fast.to_dict(), plain.to_dict()
    assert set(df) == set(dp) and all(df[k] == dp[k] for k in df)
    o = oracle.run_circuit(circ)
    assert fast.nnz() == o.nnz() == 2 ** 10
    assert compare_states(df, o.to_dict()) >= 1 - 1e-12


@pytest.mark.parametrize("with_ops", [False, True])
@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("amp32", [False, True])
@pytest.mark.parametrize("segmented", [False, True])
def test_uncontrolled_fold_over_many_chunks(sqs, wide, amp32, segmented, with_ops):
    """The uncontrolled copy-pair fold (bit-1 members skipped, bit-0 members
    compacted) on a ragged state of about 10^5 branches spanning many
    4096-slot chunks, on a dense input (after an expansion) and a segmented
    one (after a bucket merge), one- and two-word keys: bit for bit the state
    of the plain merge, and equal to the oracle.  Without operations fused
    into it (they are deferred past the fold) the staged kernel runs; a queued
    prune keeps them in front, so the register-fed kernel runs them."""
    widths = [16, 8, 40] + ([40] if wide else [])
    rng = np.random.default_rng(77)
    table = rng.integers(0, 256, size=1 << 16).astype(np.uint8)
    gates = [("h", 0, b, ()) for b in range(15)]
    gates += [("qload", 0, 1, 0),
              ("h", 2, 0, ((1, 0, 1),)),          # expands about half: ragged count
              ("h", 0, 15, ())]                   # constant bit: +1 copy pairs on bit 15
    gates += [("x", 2, 5, ()), ("x", 2, 7, ((1, 2, 1),)), ("add", 2, -1, 12345, ()),
              ("phase", ((1, 1, 1),), 0.3), ("ry", 2, 9, 0.7, ())]
    if segmented:
        gates += [("h", 1, 3, ())]                # no partners: bucket merge, segmented out
    gates += [("x", 2, 11, ((0, 2, 1),))]
    if with_ops:
        gates += [("prune", 1e-15)]               # nothing is that small; keeps the run in front
    gates += [("h", 0, 15, ())]                   # the fold
    circ = {"widths": widths, "eps": 1e-14, "tables": [table], "gates": gates}
    fast, plain = _plain_and_fast(sqs, circ, amp32)
    names = [r[0] for r in fast.trace_read()[0]]
    assert names.count("k_fold") == 1
    assert (fast.stats()["ops_deferred"] > 0) == (not with_ops)
    if segmented:
        assert fast.stats()["steps_hash"] >= 1
    df, dp = fast.to_dict(), plain.to_dict()
    assert len(df) > 60000 and len(df) % 2048 != 0
    assert set(df) == set(dp) and all(df[k] == dp[k] for k in df)
    o = oracle.run_circuit(circ).to_dict()
    if amp32:
        assert compare_states(df, o, atol=ATOL32, band=ATOL32) >= 1 - 1e-6
    else:
        assert set(df) == set(o)
        assert compare_states(df, o) >= 1 - 1e-12


@pytest.mark.parametrize("amp32", [False, True])
def test_ops_deferred_past_copy_pair_steps(sqs, amp32):
    """Operations queued before a step that can only merge (a copy-pair
    target) stay queued past it when they commute with it: none writes a
    control of the step and none prunes.  The plain merge path defers the
    same way, so the two states agree bit for bit; both equal the oracle,
    which applies every operation in issue order."""
    widths = [8, 8, 8]
    gates = [("h", 0, b, ()) for b in range(6)]
    ops = [("x", 1, 0, ()), ("add", 2, 1, 0, ()), ("phase", ((1, 1, 1),), 0.4),
           ("x", 2, 3, ((1, 0, 1),)), ("swap", 1, 2, ())]
    gates += ops + [("h", 0, 5, ())]              # fold, the five operations deferred
    gates += [("h", 0, 4, ())]                     # again deferred (still queued)
    gates += [("x", 1, 6, ()), ("h", 0, 3, ((1, 6, 1),))]   # writes the control: applied first
    gates += [("x", 2, 7, ()), ("prune", 1e-13), ("h", 0, 2, ())]  # a queued prune: applied first
    gates += [("h", 0, 1, ()), ("phase", ((2, 7, 1),), 1.1)]
    circ = {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates}
    fast, plain = _plain_and_fast(sqs, circ, amp32)
    sf, sp = fast.stats(), plain.stats()
    assert sf["ops_deferred"] == sp["ops_deferred"] >= 5 + 5
    assert sf["steps_fold"] >= 3 and sp["steps_fold"] == 0
    df, dp = fast.to_dict(), plain.to_dict()
    assert set(df) == set(dp) and all(df[k] == dp[k] for k in df)
    o = oracle.run_circuit(circ).to_dict()
    if amp32:
        assert compare_states(df, o, atol=ATOL32, band=ATOL32) >= 1 - 1e-6
    else:
        assert set(df) == set(o)
        assert compare_states(df, o) >= 1 - 1e-12


def test_config1_batch_sampled_instances(sqs):
    """256 instances of config 1 in one state (own QRAM table each): sampled
    instances equal config 1 run alone on the oracle, scaled by 1/16."""
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "config1_seed1_gates.json")) as f:
        stored = json.load(f)
    batch = W.config1_batch(stored, inst_bits=8)
    g = sqs.run_circuit(batch)
    lo, hi, amps = g.export()
    inst = (lo >> np.uint64(8)) & np.uint64(255)
    fresh = build_config1(seed=1)
    for i in (0, 77, 255):
        ref = oracle.run_circuit(dict(fresh, tables=[W.config1_instance_table(batch, i)])).to_dict()
        sel = inst == i
        part = {}
        for l, a in zip(lo[sel], amps[sel]):
            k = int(l)
            part[(k & 0xff) | ((k >> 16) << 8)] = complex(a)
        assert set(part) == set(ref)
        assert max(abs(part[k] - ref[k] / 16.0) for k in part) < 1e-12

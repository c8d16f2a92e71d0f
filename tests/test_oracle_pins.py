"""Pins for the CPU oracle against facts that do not come from the oracle:
the paper's printed matrices and branch counts, closed forms, an independent
dense statevector, brute-force Kronecker-product unitaries and invariants."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2503_15118_gb300 import workloads as W
from tests.helpers import build_config1, compare_states

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_matrices():
    out = {}
    s = 1 / math.sqrt(2)
    for line in open(os.path.join(GOLDEN, "gate_matrices.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, *cells = line.split()
        vals = []
        for c in cells:
            re, im = c.split(",")
            conv = lambda t: {"s": s, "-s": -s}.get(t, None)
            vals.append(complex(conv(re) if conv(re) is not None else float(re),
                                conv(im) if conv(im) is not None else float(im)))
        out[name] = np.array(vals).reshape(2, 2)
    return out


def _basis(widths, key):
    st = oracle.OracleState(widths)
    for r, w in enumerate(widths):
        off = sum(widths[:r])
        for b in range(w):
            if (key >> (off + b)) & 1:
                st.x(r, b)
    return st


@pytest.mark.parametrize("name", ["X", "Y", "Z", "H"])
def test_printed_gate_matrices(name):
    """Each column of the printed matrix is the image of |0> or |1> (Sec. II.A)."""
    M = _golden_matrices()[name]
    for col in (0, 1):
        st = _basis([1], col)
        if name == "X":
            st.x(0, 0)
        elif name == "H":
            st.h_gate(0, 0)
        elif name == "Z":
            st.phase(((0, 0, 1),), math.pi)
        else:
            st.u1q(0, 0, M)
        d = st.to_dict()
        for row in (0, 1):
            assert abs(d.get(row, 0) - M[row, col]) < 1e-15, (name, row, col)


def test_index_convention_is_row_out_col_in():
    """A non-symmetric U distinguishes U from U^T: U|0> is U's first column."""
    U = np.array([[0.6, -0.8j], [0.8, 0.6j]])
    st = _basis([3], 0)
    st.u1q(0, 1, U)
    d = st.to_dict()
    assert abs(d[0] - 0.6) < 1e-15 and abs(d[2] - 0.8) < 1e-15
    st = _basis([3], 2)
    st.u1q(0, 1, U)
    d = st.to_dict()
    assert abs(d[0] + 0.8j) < 1e-15 and abs(d[2] - 0.6j) < 1e-15


@pytest.mark.parametrize("widths", [[4], [3, 5], [8, 8, 4], [10, 6]])
def test_hadamard_power_closed_form(widths):
    """H on every qubit of |0..0> gives 2^n branches of amplitude 2^{-n/2}."""
    st = oracle.OracleState(widths)
    for r, w in enumerate(widths):
        for b in range(w):
            st.h_gate(r, b)
    n = sum(widths)
    lo, hi, a = st.export()
    assert st.nnz() == 2 ** n
    assert np.all(lo == np.arange(2 ** n))
    assert np.max(np.abs(a - 2 ** (-n / 2))) < 1e-15


@pytest.mark.parametrize("theta", [0.3, 1.7, 3.0, 5.5])
def test_ry_closed_form(theta):
    st = oracle.OracleState([2])
    st.ry(0, 1, theta)
    d = st.to_dict()
    assert abs(d[0] - math.cos(theta / 2)) < 1e-15
    assert abs(d[2] - math.sin(theta / 2)) < 1e-15
    st = _basis([2], 2)
    st.ry(0, 1, theta)
    d = st.to_dict()
    assert abs(d[0] + math.sin(theta / 2)) < 1e-15
    assert abs(d[2] - math.cos(theta / 2)) < 1e-15


def _paper_counts():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_branch_counts.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            c, q, b, _src = line.split()
            rows.append((c, int(q), int(b)))
    return rows


@pytest.mark.parametrize("row", _paper_counts())
def test_paper_branch_counts(row):
    circuit, n, branches = row
    if circuit == "ghz":
        widths = [min(64, n - 64 * i) for i in range((n + 63) // 64)]
        st = oracle.OracleState(widths)
        st.h_gate(0, 0)
        prev = (0, 0)
        for q in range(1, n):
            r, b = divmod(q, 64)
            st.x(r, b, ((prev[0], prev[1], 1),))
            prev = (r, b)
        assert st.nnz() == branches
        lo, hi, a = st.export()
        keys = sorted((int(h) << 64) | int(l) for l, h in zip(lo, hi))
        assert keys == [0, (1 << n) - 1]
        assert np.allclose(a, 1 / math.sqrt(2), atol=1e-15)
    else:
        # QRAM on a single-branch input |i>_A |0>_D -> |i>_A |d_i>_D (Eq. S1).
        rng = np.random.default_rng(0)
        table = rng.integers(0, 2 ** 10, size=2 ** 10).astype(np.uint16)
        st = oracle.OracleState([10, 10])
        i = 0b1011001110
        for b in range(10):
            if (i >> b) & 1:
                st.x(0, b)
        st.qram(0, 1, table)
        assert st.nnz() == branches
        d = st.to_dict()
        assert d == {i | (int(table[i]) << 10): 1.0}


def test_qram_truncates_to_word_length_and_reads_zero_past_table():
    table = np.array([0x1FF, 0x0F0, 0xABC], dtype=np.uint32)
    st = oracle.OracleState([2, 8])
    st.h_gate(0, 0)
    st.h_gate(0, 1)
    st.qram(0, 1, table)
    d = st.to_dict()
    want = {0 | (0xFF << 2), 1 | (0xF0 << 2), 2 | (0xBC << 2), 3}
    assert set(d) == want


def _circuits_small():
    kinds_all = ("x", "cx", "ccx", "ry", "cry", "phase", "cphase", "h", "ch", "u1q",
                 "cu1q", "diag", "adiag", "add", "sub", "swap", "qram")
    out = []
    for seed, widths in [(11, [4, 4, 2]), (12, [3, 3, 4]), (13, [5, 5, 2]), (14, [6, 6])]:
        rng = np.random.default_rng(seed)
        table = rng.integers(0, 2 ** 8, size=2 ** widths[0]).astype(np.uint8)
        out.append(W.random_circuit(widths, 60, seed, kinds=kinds_all, tables=[table]))
    return out


@pytest.mark.parametrize("circ", _circuits_small(), ids=lambda c: c["name"])
def test_oracle_matches_dense_statevector(circ):
    o = oracle.run_circuit(circ)
    d = dense.run_dense(circ)
    ref = {i: complex(a) for i, a in enumerate(d.psi) if abs(a) >= 1e-14}
    fid = compare_states(o.to_dict(), ref)
    assert fid > 1 - 1e-12


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_oracle_matches_kron_unitaries(seed):
    kinds_all = ("x", "cx", "ccx", "ry", "cry", "phase", "cphase", "h", "ch", "u1q",
                 "cu1q", "diag", "adiag", "add", "sub", "swap", "qram")
    widths = [3, 3, 2]
    rng = np.random.default_rng(seed)
    table = rng.integers(0, 8, size=8).astype(np.uint8)
    circ = W.random_circuit(widths, 30, seed, kinds=kinds_all, tables=[table])
    v = np.zeros(2 ** 8, np.complex128)
    v[0] = 1
    for g in circ["gates"]:
        v = dense.kron_unitary(widths, g, circ["tables"]) @ v
    o = oracle.run_circuit(circ)
    ref = {i: complex(a) for i, a in enumerate(v) if abs(a) >= 1e-14}
    assert compare_states(o.to_dict(), ref) > 1 - 1e-12


def test_ry_reg_matches_kron():
    widths = [2, 3, 3]
    circ = {"widths": widths, "tables": [], "eps": 1e-14, "gates": [
        ("h", 1, 0, ()), ("h", 1, 2, ()), ("ry", 0, 0, 0.4, ()),
        ("ry_reg", 0, 1, 1, 0.37, 0.1, ()), ("ry_reg", 2, 0, 1, -1.1, 0.0, ((0, 0, 1),)),
        ("h", 2, 2, ()), ("ry_reg", 0, 0, 2, 0.9, -0.2, ())]}
    v = np.zeros(2 ** 8, np.complex128)
    v[0] = 1
    for g in circ["gates"]:
        v = dense.kron_unitary(widths, g) @ v
    ref = {i: complex(a) for i, a in enumerate(v) if abs(a) >= 1e-14}
    assert compare_states(oracle.run_circuit(circ).to_dict(), ref) > 1 - 1e-12


def test_config1_matches_dense_statevector():
    circ = build_config1(seed=1)
    assert len(circ["gates"]) == 209
    o = oracle.run_circuit(circ)
    assert 0 < o.nnz() <= 4096
    d = dense.run_dense(circ)
    ref = {i: complex(a) for i, a in enumerate(d.psi) if abs(a) >= 1e-14}
    assert compare_states(o.to_dict(), ref) > 1 - 1e-10
    assert abs(o.norm2() - 1) < 1e-12


@pytest.mark.parametrize("seed", [31, 32])
def test_apply_then_inverse_restores(seed):
    kinds_all = ("x", "cx", "ccx", "ry", "cry", "phase", "cphase", "h", "ch", "u1q",
                 "cu1q", "diag", "adiag", "add", "sub", "swap", "qram")
    widths = [6, 6, 4]
    rng = np.random.default_rng(seed)
    table = rng.integers(0, 64, size=64).astype(np.uint8)
    circ = W.random_circuit(widths, 80, seed, kinds=kinds_all, tables=[table])
    st = oracle.run_circuit(circ)
    assert abs(st.norm2() - 1) < 1e-12
    for g in W.inverse_circuit(circ)["gates"]:
        st.apply(g, circ["tables"])
    d = st.to_dict()
    assert set(d) == {0}
    assert abs(d[0] - 1) < 1e-12


def test_load_unload_add_sub_swap_restore_exactly():
    rng = np.random.default_rng(5)
    table = rng.integers(0, 2 ** 32, size=2 ** 6, dtype=np.uint64).astype(np.uint32)
    st = oracle.OracleState([6, 32, 32])
    for b in range(6):
        st.ry(0, b, 0.3 + b)
    st.qram(0, 1, table)
    st.add(2, 1)
    st.add(2, -1, 0xDEADBEEF)
    before = st.to_dict()
    st.swap(1, 2)
    st.swap(1, 2)
    st.add(2, -1, 0xDEADBEEF, subtract=True)
    st.add(2, 1, subtract=True)
    st.qram(0, 1, table)
    after = st.to_dict()
    assert set(after) == set(range(64))
    st.qram(0, 1, table)
    st.add(2, 1)
    st.add(2, -1, 0xDEADBEEF)
    assert st.to_dict() == before  # bit-exact: permutations move amplitudes unchanged


def test_add_is_modular_within_register():
    st = oracle.OracleState([4, 4, 4])
    for b in range(4):
        st.x(1, b)  # reg1 = 15
    st.x(0, 0)      # reg0 = 1
    st.add(1, 0)    # 15 + 1 = 16 -> 0 mod 2^4, reg2 untouched
    assert st.to_dict() == {1: 1.0}
    st.add(1, -1, 3, subtract=True)  # 0 - 3 -> 13
    assert st.to_dict() == {1 | (13 << 4): 1.0}


def test_prune_is_strict():
    st = oracle.OracleState([2])
    st.import_(np.array([0, 1, 2], np.uint64), np.zeros(3, np.uint64),
               np.array([1e-14, 0.999e-14, 1.001e-14]))
    st.prune(1e-14)
    assert sorted(st.to_dict()) == [0, 2]


def test_config2_reduced_peak_and_exact_cancellation():
    """Scaled config 2 (12 branching gates): the re-applied H gates on the
    cancel qubits each halve the branch count."""
    circ = W.config2(seed=2, n_branch=12, n_perm=200, n_cancel=4)
    n_main = len(circ["gates"]) - 4
    st = oracle.run_circuit(circ, upto=n_main)
    peak = st.nnz()
    assert peak == 2 ** 12
    for i, g in enumerate(circ["gates"][n_main:]):
        st.apply(g)
        assert st.nnz() == peak >> (i + 1)
    assert abs(st.norm2() - 1) < 1e-12


def test_reflection_R_matches_definition():
    """R = i(2|0><0|_anc - I) (x) I written as phase operations: pi where the
    ancilla register is 0, then a global -i."""
    widths = [2, 2]
    anc = 1
    rng = np.random.default_rng(3)
    v = rng.normal(size=16) + 1j * rng.normal(size=16)
    st = oracle.OracleState(widths)
    st.import_(np.arange(16, dtype=np.uint64), np.zeros(16, np.uint64), v)
    st.phase(((anc, 0, 0), (anc, 1, 0)), math.pi)
    st.phase((), -math.pi / 2)
    P0 = np.zeros((4, 4))
    P0[0, 0] = 1
    R = 1j * np.kron(2 * P0 - np.eye(4), np.eye(4))  # anc is the high register
    want = R @ v
    got = st.to_dict()
    for i in range(16):
        assert abs(got.get(i, 0) - want[i]) < 1e-14


def test_mlp_oracle_gradient_matches_finite_differences():
    """Pins the reference network's analytic gradient against central
    differences of its forward pass (FP64)."""
    from oracle import mlp
    rng = np.random.default_rng(4)
    p = rng.normal(scale=0.3, size=mlp.N_PARAMS)
    X = rng.normal(size=(7, mlp.F))
    T = rng.normal(size=7)
    g = mlp.gradient(p, X, T)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    for i in list(idx) + [mlp.N_PARAMS - 1, 0]:
        e = np.zeros_like(p)
        e[i] = h
        num = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_mlp_oracle_forward_closed_form():
    """Zero weights: the output is the output bias whatever the input."""
    from oracle import mlp
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 0.37
    y, _, _ = mlp.forward(p, np.ones((3, mlp.F)))
    assert np.allclose(y, 0.37)


ARITH_KINDS = ("x", "cx", "h", "ry", "muladd", "mulc", "divxor", "add")


@pytest.mark.parametrize("seed", [31, 32, 33])
def test_arithmetic_oracles_match_dense(seed):
    """Multiply-add, multiply by an odd constant and divide-XOR (the arithmetic
    oracles of Sec. II.D.1) on the std::map oracle agree with the independent
    dense statevector."""
    widths = [3, 3, 3, 3]
    circ = W.random_circuit(widths, 60, seed, kinds=ARITH_KINDS)
    assert any(g[0] in ("muladd", "mulc", "divxor") for g in circ["gates"])
    o = oracle.run_circuit(circ)
    d = dense.run_dense(circ)
    got = o.to_dict()
    for k in range(1 << sum(widths)):
        assert abs(got.get(k, 0) - d.psi[k]) < 1e-12


def test_arithmetic_oracles_are_bijections_and_invert():
    widths = [4, 4, 4]
    rng = np.random.default_rng(4)
    keys = np.arange(1 << 12, dtype=np.uint64)
    amps = rng.standard_normal(1 << 12) + 1j * rng.standard_normal(1 << 12)
    for gate in [("muladd", 0, 1, 2, ()), ("mulc", 1, 11, ((0, 0, 1),)), ("divxor", 2, 0, 1, ())]:
        o = oracle.OracleState(widths)
        o.import_(keys, np.zeros_like(keys), amps)
        o.apply(gate)
        d = o.to_dict()
        assert len(d) == 1 << 12   # a bijection on the full space
        assert sorted(abs(v) for v in d.values()) == sorted(abs(a) for a in amps)
        if gate[0] != "muladd":
            o.apply(W.inverse_gate(gate))
            back = o.to_dict()
            assert all(back[int(k)] == a for k, a in zip(keys, amps))
    # multiply-add on a basis state: 5 + 3 * 7 = 26 = 10 (mod 16)
    o = oracle.OracleState(widths)
    o.import_(np.array([5 | (3 << 4) | (7 << 8)], np.uint64), np.zeros(1, np.uint64), np.ones(1))
    o.apply(("muladd", 0, 1, 2, ()))
    assert set(o.to_dict()) == {10 | (3 << 4) | (7 << 8)}
    o.apply(("divxor", 1, 2, 0, ()))           # 3 ^ (7 // 10) = 3
    o.apply(("divxor", 2, 0, 1, ()))           # 7 ^ (10 // 3) = 7 ^ 3 = 4
    assert set(o.to_dict()) == {10 | (3 << 4) | (4 << 8)}


def test_sampled_single_gate_matches_oracle_and_brute_force():
    """The one-by-one evaluator used at full size (oracle/sampled.py) against
    the std::map oracle's u1q and against a brute-force sum over the input
    list, on a random sparse state; and its pair-class count against the
    output size of an unpruned H on a state with no cancellation."""
    from oracle import sampled
    rng = np.random.default_rng(11)
    n = 3000
    keys = np.unique(rng.integers(0, 1 << 20, size=n, dtype=np.uint64))
    amps = rng.standard_normal(keys.shape[0]) + 1j * rng.standard_normal(keys.shape[0])
    z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    U, _ = np.linalg.qr(z)
    t = 7
    o = oracle.OracleState([20])
    o.import_(keys, np.zeros_like(keys), amps)
    o.u1q(0, t, U)
    ref = o.to_dict()
    st = sampled.SortedState(keys, amps)
    xs = np.array(sorted(ref)[:: max(1, len(ref) // 400)], np.uint64)
    got = sampled.u1q_amplitudes(st, t, U, xs)
    for x, g in zip(xs.tolist(), got):
        assert abs(g - ref[x]) < 1e-13
        # Brute force: sum over every input branch that maps onto x.
        bf = sum(U[(x >> t) & 1, (k >> t) & 1] * a
                 for k, a in zip(keys.tolist(), amps) if (k | (1 << t)) == (x | (1 << t)))
        assert abs(g - bf) < 1e-13
    # Every pair class yields two outputs (random amplitudes never cancel).
    assert len(ref) == 2 * sampled.pair_class_count(keys, t)


@pytest.mark.parametrize("seed", [31, 32])
def test_qram_span_address_matches_dense(seed):
    """QRAM with an address spanning consecutive registers (the first lowest)
    against the dense statevector: load, interference, unload."""
    rng = np.random.default_rng(seed)
    widths = [3, 2, 4, 3]
    table = rng.integers(0, 16, size=1 << 5).astype(np.uint8)
    gates = [("h", 0, b, ()) for b in range(3)] + [("h", 1, 0, ()), ("h", 1, 1, ())]
    gates += [("qload", (0, 2), 2, 0), ("ry", 3, 0, 0.7, ((2, 1, 1),)),
              ("h", 3, 1, ((2, 0, 1),)), ("qunload", (0, 2), 2, 0), ("h", 0, 1, ())]
    circ = {"widths": widths, "eps": 1e-14, "tables": [table], "gates": gates}
    o = oracle.run_circuit(circ)
    d = dense.run_dense(circ)
    ref = {i: complex(a) for i, a in enumerate(d.psi) if abs(a) >= 1e-14}
    assert compare_states(o.to_dict(), ref) > 1 - 1e-12
    # The address registers pick each entry: after the load alone, the data
    # register of every branch is the table entry its (addr0, addr1) select.
    st = dense.run_dense(dict(circ, gates=gates[:6]))
    addr = st._field((0, 2))
    data = st._field(2)
    live = np.abs(st.psi) > 0
    assert np.array_equal(data[live], table[addr[live]] & 15)


@pytest.mark.parametrize("circ", _circuits_small()[:3], ids=lambda c: c["name"])
def test_probabilities_match_dense_marginals(circ):
    """The oracle's marginal distribution of each register against the dense
    statevector's, and the norm."""
    o = oracle.run_circuit(circ)
    d = dense.run_dense(circ)
    for reg in range(len(circ["widths"])):
        v, p = o.probabilities(reg)
        want = d.marginal(reg)
        got = np.zeros_like(want)
        got[v.astype(np.int64)] = p
        assert np.abs(got - want).max() < 1e-12
    assert abs(o.norm2() - np.sum(np.abs(d.psi) ** 2)) < 1e-12


@pytest.mark.parametrize("circ", _circuits_small()[:2], ids=lambda c: c["name"])
def test_peak_is_the_largest_intermediate_count(circ):
    """The oracle's peak branch count against the dense statevector's count
    of amplitudes of modulus at least eps after every gate."""
    o = oracle.run_circuit(circ)
    counts = [1]
    st = dense.DenseState(circ["widths"])
    for g in circ["gates"]:
        st.apply(g, circ.get("tables", ()))
        counts.append(int(np.count_nonzero(np.abs(st.psi) >= circ.get("eps", 1e-14))))
    assert o.peak() == max(counts)
    assert o.nnz() == counts[-1]

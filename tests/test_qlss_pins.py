"""Pins of the linear-system workload (Sec. III.C, Supp. D) on the CPU oracle.

The walk's gate lists are inputs, not the method, but the oracle must run
them right, and they must be what the paper describes: the block-encoding
identity <i|<0|<0| U_A |j>|0>|0> = A_ij / ||A||_F (Supp. D), the block of
U_H(s) equal to H(s) / lambda, U_A^dag undoing U_A, and the walk driving the
flagged block towards x / ||x|| for x = A^-1 b with an error that shrinks as
the walk lengthens (Eq. of the discrete adiabatic bound, Sec. III.C).  Every
expected value here comes from numpy linear algebra on A, independent of the
oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import qlss as Q


def _basis(widths, sets):
    o = oracle.OracleState(widths)
    for reg, val in sets:
        for b in range(widths[reg]):
            if (val >> b) & 1:
                o.apply(("x", reg, b, ()))
    return o


def test_tree_angles_rebuild_the_vector():
    """The product of cos / sin factors along each root-to-leaf path of the
    angle tree is the (signed) entry of the prepared vector."""
    rng = np.random.default_rng(0)
    for n in (1, 3, 5):
        x = rng.standard_normal(1 << n)
        x[rng.integers(0, 1 << n)] = 0.0
        x /= np.linalg.norm(x)
        ang = Q.tree_angles(x)
        for i in range(1 << n):
            amp = 1.0
            for l in range(n):
                p = i >> (n - l)
                bit = (i >> (n - 1 - l)) & 1
                th = ang[l][p]
                amp *= math.sin(th / 2) if bit else math.cos(th / 2)
            assert abs(amp - x[i]) < 1e-12


def test_angle_codes_round_to_the_grid():
    th = np.array([0.0, 1e-12, math.pi, 2 * math.pi, -0.5, 4 * math.pi - 1e-12])
    c = Q.angle_code(th).astype(np.float64) * Q.ANGLE_SCALE
    d = np.mod(c - np.mod(th, 4 * math.pi) + 2 * math.pi, 4 * math.pi) - 2 * math.pi
    assert np.abs(d).max() <= Q.ANGLE_SCALE / 2 + 1e-15


@pytest.mark.parametrize("N,hb", [(4, 1), (8, 2), (16, 3)])
def test_block_encoding_identity(N, hb):
    """<i|<0|<0| U_A |j>|0>|0> = A_ij / ||A||_F (Supp. D), every i, j."""
    A = Q.spd_banded(N, hb, 6.0, np.random.default_rng(N))
    n = int(math.log2(N))
    widths, ids = Q.registers(n)
    t_l, t_r, nf = Q.tables_for(A)
    tables = t_l + t_r
    gates = Q.u_a(n, ids, list(range(n)), list(range(n, 2 * n)), ())
    off = np.cumsum([0] + widths)
    got = np.zeros((N, N))
    for j in range(N):
        o = _basis(widths, [(Q.TOP, j)])
        for g in gates:
            o.apply(g, tables)
        d = o.to_dict()
        for i in range(N):
            got[i, j] = d.get(i << int(off[Q.TOP]), 0).real
        # U_A^dag U_A = I: the input comes back, keys exactly
        for g in Q.u_a(n, ids, list(range(n)), list(range(n, 2 * n)), (), dagger=True):
            o.apply(g, tables)
        back = o.to_dict()
        assert set(back) == {j << int(off[Q.TOP])}
        assert abs(back[j << int(off[Q.TOP])] - 1.0) < 1e-12
    # 2n rotations, each within half a grid step of its angle
    assert np.abs(got - A / nf).max() < 4 * n * Q.ANGLE_SCALE


@pytest.mark.parametrize("f", [0.0, 0.37, 1.0])
def test_walk_block_encodes_h_of_s(f):
    """<0|_anc U_H(s) |0>_anc = H(s) / lambda with H(s) = [[0, A(f) Q_b],
    [Q_b A(f), 0]] and lambda = (1 - f) + f ||A||_F."""
    N, n = 4, 2
    A = Q.spd_banded(N, 1, 4.0, np.random.default_rng(2))
    widths, ids = Q.registers(n)
    t_l, t_r, nf = Q.tables_for(A)
    tables = t_l + t_r
    gates = Q.u_h(n, ids, list(range(n)), list(range(n, 2 * n)), Q.lcu_angle(f, nf))
    off = np.cumsum([0] + widths)

    def key(ah, top):
        return (ah << int(off[ids["AH"]])) | (top << int(off[Q.TOP]))

    got = np.zeros((2 * N, 2 * N), np.complex128)
    for ah in range(2):
        for j in range(N):
            o = _basis(widths, [(ids["AH"], ah), (Q.TOP, j)])
            for g in gates:
                o.apply(g, tables)
            d = o.to_dict()
            for ah2 in range(2):
                for i in range(N):
                    got[ah2 * N + i, ah * N + j] = d.get(key(ah2, i), 0)
    b = np.full(N, N ** -0.5)
    Qb = np.eye(N) - np.outer(b, b)
    Af = (1 - f) * np.eye(N) + f * A
    H = np.block([[np.zeros((N, N)), Af @ Qb], [Qb @ Af, np.zeros((N, N))]])
    lam = (1 - f) + f * nf
    assert np.abs(got - H / lam).max() < 1e-8


def test_schedule_end_points_and_monotone():
    for kappa in (2.0, 10.0, 50.0):
        s = np.linspace(0, 1, 101)
        f = np.array([Q.schedule(x, kappa) for x in s])
        assert abs(f[0]) < 1e-15 and abs(f[-1] - 1) < 1e-12
        assert np.all(np.diff(f) > 0)


def test_walk_converges_to_the_solution():
    """Sanity of the construction (not parity): the flagged block approaches
    x / ||x|| and the error falls as the walk lengthens."""
    errs = []
    for T in (50, 200, 800):
        cfg = Q.config4(seed=5, N=4, half_band=2, kappa=5.0, T=T)
        circ = Q.walk_circuit(cfg)
        o = oracle.run_circuit(circ)
        v = Q.solution_block(o.to_dict(), cfg)
        x = np.linalg.solve(cfg["A"], cfg["b"])
        x /= np.linalg.norm(x)
        p = np.vdot(v, v).real
        errs.append(1 - abs(np.vdot(x, v)) ** 2 / p)
        assert abs(o.norm2() - 1) < 1e-9
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 5e-3


def _single_instance_circuit(cfg, i, n_steps):
    """Instance i alone: INST preset to i instead of the superposition."""
    circ = Q.batched_circuit(cfg, n_steps)
    ib = cfg["inst_bits"]
    pre = [("x", cfg["ids"]["INST"], b, ()) for b in range(ib) if (i >> b) & 1]
    gates = pre + [g for g in circ["gates"][ib:]]  # drop the H on INST
    return dict(circ, gates=gates)


def test_batched_instances_are_independent():
    """The batched state restricted to instance i is 2^{-inst_bits/2} times
    the state of instance i walked alone (nothing acts on INST)."""
    cfg = Q.config5(seed=7, n_inst=4, n_min=2, n_max=3, T=6)
    o = oracle.run_circuit(Q.batched_circuit(cfg, 6))
    d = o.to_dict()
    off = np.cumsum([0] + cfg["widths"])
    sh, m = int(off[cfg["ids"]["INST"]]), (1 << cfg["inst_bits"]) - 1
    scale = 2.0 ** (-cfg["inst_bits"] / 2)
    for i in range(cfg["n_inst"]):
        alone = oracle.run_circuit(_single_instance_circuit(cfg, i, 6)).to_dict()
        part = {k: v for k, v in d.items() if (k >> sh) & m == i}
        assert set(part) == set(alone)
        assert max(abs(part[k] - scale * alone[k]) for k in part) < 1e-12


def test_batched_block_encoding_per_instance():
    """Each instance's block of the batched U_A is its own A_i / ||A_i||_F,
    whatever its size below the register width."""
    cfg = Q.config5(seed=8, n_inst=4, n_min=2, n_max=4, T=4)
    n, ids = cfg["n"], cfg["ids"]
    off = np.cumsum([0] + cfg["widths"])
    fwd = Q.u_a(n, ids, cfg["t_l"], cfg["t_r"], (), span_l=3, span_r=2)
    for i in range(cfg["n_inst"]):
        A, nf = cfg["mats"][i], cfg["norms"][i]
        N = A.shape[0]
        for j in range(N):
            o = _basis(cfg["widths"], [(ids["INST"], i), (Q.TOP, j)])
            for g in fwd:
                o.apply(g, cfg["tables"])
            d = o.to_dict()
            base = i << int(off[ids["INST"]])
            col = np.array([d.get(base | (r << int(off[Q.TOP])), 0).real for r in range(N)])
            assert np.abs(col - A[:, j] / nf).max() < 4 * n * Q.ANGLE_SCALE


def test_batched_walk_converges_per_instance():
    cfg = Q.config5(seed=5, n_inst=4, n_min=2, n_max=3, kappa=(5.0,), T=150)
    o = oracle.run_circuit(Q.batched_circuit(cfg, 150))
    d = o.to_dict()
    assert abs(o.norm2() - 1) < 1e-9
    for i in range(cfg["n_inst"]):
        v = Q.instance_block(d, cfg, i)
        A = cfg["mats"][i]
        N = A.shape[0]
        x = np.linalg.solve(A, np.full(N, N ** -0.5))
        x /= np.linalg.norm(x)
        assert abs(np.vdot(x, v)) ** 2 / np.vdot(v, v).real > 0.99


def test_config1_batch_instances_are_config1():
    """The stored config-1 gate list is what the oracle-driven rejection
    sampling produces, and instance i of the batched form equals config 1
    run alone with instance i's table, scaled by 2^{-inst_bits/2}."""
    import json
    import os

    from paper_2503_15118_gb300 import workloads as W
    from tests.helpers import build_config1
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "config1_seed1_gates.json")) as f:
        stored = json.load(f)
    fresh = build_config1(seed=1)
    assert len(stored["gates"]) == len(fresh["gates"])
    a = oracle.run_circuit(W.config1_from_stored(stored)).to_dict()
    b = oracle.run_circuit(fresh).to_dict()
    assert set(a) == set(b) and all(a[k] == b[k] for k in a)
    batch = W.config1_batch(stored, inst_bits=2)
    o = oracle.run_circuit(batch)
    d = o.to_dict()
    off_inst = 8
    for i in range(4):
        alone = dict(fresh, tables=[W.config1_instance_table(batch, i)])
        ref = oracle.run_circuit(alone).to_dict()
        # fresh uses registers (addr, data, anc); the batch (addr, inst, data, anc)
        part = {}
        for k, a in d.items():
            if (k >> off_inst) & 3 != i:
                continue
            addr = k & 0xff
            rest = k >> (off_inst + 2)
            part[addr | (rest << 8)] = a
        assert set(part) == set(ref)
        assert max(abs(part[k] - 0.5 * ref[k]) for k in part) < 1e-12


# ---- non-Hermitian variant --------------------------------------------------

def test_nonherm_matrix_shape_and_condition():
    A = Q.nonherm_banded(16, 3, 7.0, np.random.default_rng(1))
    i = np.arange(16)
    assert np.all(A[np.abs(i[:, None] - i[None, :]) > 3] == 0)
    assert np.abs(A - A.T).max() > 1e-3  # not symmetric
    sv = np.linalg.svd(A, compute_uv=False)
    assert abs(sv[0] / sv[-1] - 7.0) < 1e-9
    ev = np.linalg.eigvals(A)
    assert ev.real.min() < 0 < ev.real.max()  # indefinite


@pytest.mark.parametrize("N", [4, 8])
def test_nonherm_block_encoding_identity(N):
    """<0|_anc U_bA |0>_anc = bA / ||A||_F with bA = [[0, A], [A^T, 0]] on
    (a_1, TOP), every column."""
    cfg = Q.config4_nonherm(seed=N, N=N, half_band=2, kappa=5.0, T=10)
    n, ids, widths, A = cfg["n"], cfg["ids"], cfg["widths"], cfg["A"]
    gates = Q.u_bold_a(n, ids, cfg["tabs"], ())
    off = np.cumsum([0] + widths)
    a1 = int(off[ids["A1"]])
    bold = np.block([[np.zeros((N, N)), A], [A.T, np.zeros((N, N))]])
    got = np.zeros((2 * N, 2 * N))
    for c in range(2):
        for j in range(N):
            o = _basis(widths, [(ids["A1"], c), (Q.TOP, j)])
            for g in gates:
                o.apply(g, cfg["tables"])
            d = o.to_dict()
            for r in range(2):
                for i in range(N):
                    got[r * N + i, c * N + j] = d.get((r << a1) | (i << int(off[Q.TOP])), 0).real
    assert np.abs(got - bold / cfg["norm_f"]).max() < 4 * n * Q.ANGLE_SCALE


@pytest.mark.parametrize("f", [0.0, 0.37, 1.0])
def test_nonherm_walk_block_encodes_h_of_s(f):
    """<0|_anc U_H(s) |0>_anc = H(s) / lambda with A(f) = (1 - f) sigma_z (x) I
    + f bA and Q = I - |0><0|_{a_1} (x) |b><b|, on (AH, a_1, TOP)."""
    N = 4
    cfg = Q.config4_nonherm(seed=3, N=N, half_band=1, kappa=4.0, T=10)
    n, ids, widths, A, nf = cfg["n"], cfg["ids"], cfg["widths"], cfg["A"], cfg["norm_f"]
    gates = Q.u_h_nh(n, ids, cfg["tabs"], Q.lcu_angle(f, nf))
    off = np.cumsum([0] + widths)

    def key(ah, c, top):
        return (ah << int(off[ids["AH"]])) | (c << int(off[ids["A1"]])) | (top << int(off[Q.TOP]))

    M = 2 * N
    got = np.zeros((2 * M, 2 * M), np.complex128)
    for ah in range(2):
        for c in range(2):
            for j in range(N):
                o = _basis(widths, [(ids["AH"], ah), (ids["A1"], c), (Q.TOP, j)])
                for g in gates:
                    o.apply(g, cfg["tables"])
                d = o.to_dict()
                for ah2 in range(2):
                    for c2 in range(2):
                        for i in range(N):
                            got[ah2 * M + c2 * N + i, ah * M + c * N + j] = d.get(key(ah2, c2, i), 0)
    b = np.zeros(M)
    b[:N] = N ** -0.5
    Qb = np.eye(M) - np.outer(b, b)
    bold = np.block([[np.zeros((N, N)), A], [A.T, np.zeros((N, N))]])
    Af = (1 - f) * np.kron(np.diag([1.0, -1.0]), np.eye(N)) + f * bold
    H = np.block([[np.zeros((M, M)), Af @ Qb], [Qb @ Af, np.zeros((M, M))]])
    lam = (1 - f) + f * nf
    assert np.abs(got - H / lam).max() < 4 * n * Q.ANGLE_SCALE + 1e-12


def test_nonherm_walk_converges_to_the_solution():
    """The flagged block |0>_AH |1>_{a_1} approaches A^-1 b / ||A^-1 b||, with
    an error that falls as the walk lengthens."""
    errs = []
    for T in (50, 200, 800):
        cfg = Q.config4_nonherm(seed=5, N=4, half_band=2, kappa=5.0, T=T)
        o = oracle.run_circuit(Q.walk_circuit_nh(cfg))
        v = Q.solution_block_nh(o.to_dict(), cfg)
        x = np.linalg.solve(cfg["A"], cfg["b"])
        x /= np.linalg.norm(x)
        p = np.vdot(v, v).real
        errs.append(1 - abs(np.vdot(x, v)) ** 2 / p)
        assert abs(o.norm2() - 1) < 1e-9
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 5e-3, errs


@pytest.mark.parametrize("nonherm", [False, True])
def test_walk_error_grows_with_condition_number(nonherm):
    """At a fixed walk length the final error grows with kappa (Sec. III.C:
    the adiabatic bound scales with kappa), averaged over three systems."""
    def err(kappa, seed):
        make = Q.config4_nonherm if nonherm else Q.config4
        cfg = make(seed=seed, N=4, half_band=2, kappa=kappa, T=100)
        circ = (Q.walk_circuit_nh if nonherm else Q.walk_circuit)(cfg)
        o = oracle.run_circuit(circ)
        v = (Q.solution_block_nh if nonherm else Q.solution_block)(o.to_dict(), cfg)
        x = np.linalg.solve(cfg["A"], cfg["b"])
        x /= np.linalg.norm(x)
        return 1 - abs(np.vdot(x, v)) ** 2 / np.vdot(v, v).real
    low = np.mean([err(5.0, s) for s in (5, 6, 7)])
    high = np.mean([err(80.0, s) for s in (5, 6, 7)])
    assert low < high / 3, (low, high)

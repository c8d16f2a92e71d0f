"""The linear-system walk (Sec. III.C, Supp. D) on the CUDA path.

Small systems run the whole walk on both the CUDA path and the oracle, which
must agree element by element.  At the full size (N = 1024, half-bandwidth 8,
2^22 branches at the peak of a walk step) the oracle is too slow for a whole
step, so the tests check what holds at any size: the block-encoding identity
on sampled columns against numpy's A, U_A^dag undoing U_A, the norm kept by
every step, and the FP32-storage state against the FP64 one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2503_15118_gb300 import qlss as Q
from tests.helpers import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sqs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs as S
    S.load()
    return S


@pytest.mark.parametrize("merge", [0, 8])
@pytest.mark.parametrize("amp32", [False, True])
def test_small_walk_matches_oracle(sqs, merge, amp32):
    cfg = Q.config4(seed=6, N=8, half_band=2, kappa=5.0, T=20)
    circ = Q.walk_circuit(cfg)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, amp32=amp32, merge=merge)
    got, ref = g.to_dict(), o.to_dict()
    if amp32:
        assert compare_states(got, ref, atol=1e-5, band=1e-5) >= 1 - 1e-6
    else:
        assert compare_states(got, ref, eps=1e-14, atol=1e-12) >= 1 - 1e-10
        assert g.peak_nnz() == o.peak()


def _mid_step(cfg, step_fn):
    """|b> prepared, then one walk step at the middle of the schedule (the
    first step has f = 0, where U_A is never selected)."""
    return {"widths": cfg["widths"], "eps": cfg["eps"], "tables": cfg["tables"],
            "gates": cfg["prep"] + step_fn(cfg, cfg["steps"][cfg["T"] // 2])}


def test_one_step_n256_matches_oracle(sqs):
    cfg = Q.config4(seed=4, N=256, half_band=8, kappa=10.0, T=2000)
    circ = _mid_step(cfg, Q.walk_step)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ)
    assert g.nnz() == o.nnz()
    assert compare_states(g.to_dict(), o.to_dict(), eps=1e-14, atol=1e-12) >= 1 - 1e-10


@pytest.fixture(scope="module")
def full():
    return Q.config4(seed=4, N=1024, half_band=8, kappa=10.0, T=2000)


def test_full_size_block_encoding_columns(sqs, full):
    cfg = full
    n, ids, N = cfg["n"], cfg["ids"], 1 << cfg["n"]
    off = np.cumsum([0] + cfg["widths"])
    A, nf = cfg["A"], cfg["norm_f"]
    fwd = Q.u_a(n, ids, cfg["t_l"], cfg["t_r"], ())
    bwd = Q.u_a(n, ids, cfg["t_l"], cfg["t_r"], (), dagger=True)
    for j in (0, 517, N - 1):
        st = sqs.State(cfg["widths"])
        for b in range(n):
            if (j >> b) & 1:
                st.apply(("x", Q.TOP, b, ()))
        for gate in fwd:
            st.apply(gate, cfg["tables"])
        d = st.to_dict()
        col = np.array([d.get(i << int(off[Q.TOP]), 0) for i in range(N)])
        assert np.abs(col - A[:, j] / nf).max() < 4 * n * Q.ANGLE_SCALE
        assert abs(sum(abs(v) ** 2 for v in d.values()) - 1) < 1e-10
        for gate in bwd:
            st.apply(gate, cfg["tables"])
        back = st.to_dict()
        assert set(back) == {j << int(off[Q.TOP])}
        st.close()


def test_full_size_walk_steps_keep_norm_and_fp32_fidelity(sqs, full):
    cfg = full
    circ = Q.walk_circuit(cfg, n_steps=2)
    g64 = sqs.run_circuit(circ)
    g32 = sqs.run_circuit(circ, amp32=True)
    d64, d32 = g64.to_dict(), g32.to_dict()
    n2 = sum(abs(v) ** 2 for v in d64.values())
    assert abs(n2 - 1) < 1e-10
    assert g64.peak_nnz() <= 4 << (2 * cfg["n"])
    ov = sum(np.conj(v) * d32.get(k, 0) for k, v in d64.items())
    n32 = sum(abs(v) ** 2 for v in d32.values())
    assert abs(ov) ** 2 / (n2 * n32) >= 1 - 1e-6


@pytest.mark.parametrize("amp32", [False, True])
def test_small_batch_matches_oracle(sqs, amp32):
    cfg = Q.config5(seed=9, n_inst=8, n_min=2, n_max=3, T=10)
    circ = Q.batched_circuit(cfg, 10)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, amp32=amp32)
    got, ref = g.to_dict(), o.to_dict()
    if amp32:
        assert compare_states(got, ref, atol=1e-5, band=1e-5) >= 1 - 1e-6
    else:
        assert compare_states(got, ref, eps=1e-14, atol=1e-12) >= 1 - 1e-10
        assert g.peak_nnz() == o.peak()


def test_full_batch_instances(sqs):
    """256 instances of sizes 8..128: every instance keeps its share of the
    norm, and small instances equal their walk alone on the oracle."""
    cfg = Q.config5()
    steps = 2
    g = sqs.run_circuit(Q.batched_circuit(cfg, steps))
    lo, hi, amps = g.export()
    off = np.cumsum([0] + cfg["widths"])
    sh, m = int(off[cfg["ids"]["INST"]]), (1 << cfg["inst_bits"]) - 1
    inst = (lo >> np.uint64(sh)) & np.uint64(m)
    p = np.bincount(inst.astype(np.int64), weights=np.abs(amps) ** 2, minlength=cfg["n_inst"])
    assert np.abs(p - 1.0 / cfg["n_inst"]).max() < 1e-10
    small = [i for i in range(cfg["n_inst"]) if cfg["sizes"][i] <= 16][:3]
    assert small
    scale = 2.0 ** (-cfg["inst_bits"] / 2)
    for i in small:
        circ = Q.batched_circuit(cfg, steps)
        ib = cfg["inst_bits"]
        pre = [("x", cfg["ids"]["INST"], b, ()) for b in range(ib) if (i >> b) & 1]
        alone = oracle.run_circuit(dict(circ, gates=pre + circ["gates"][ib:])).to_dict()
        sel = inst == i
        part = {(int(h) << 64) | int(l): complex(a)
                for l, h, a in zip(lo[sel], hi[sel], amps[sel])}
        assert set(part) == set(alone)
        assert max(abs(part[k] - scale * alone[k]) for k in part) < 1e-12


@pytest.mark.parametrize("merge", [0, 8])
@pytest.mark.parametrize("amp32", [False, True])
def test_small_nonherm_walk_matches_oracle(sqs, merge, amp32):
    """The non-Hermitian variant (extra block qubit a_1, tables of A and A^T)."""
    cfg = Q.config4_nonherm(seed=6, N=8, half_band=2, kappa=5.0, T=20)
    circ = Q.walk_circuit_nh(cfg)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ, amp32=amp32, merge=merge)
    got, ref = g.to_dict(), o.to_dict()
    if amp32:
        assert compare_states(got, ref, atol=1e-5, band=1e-5) >= 1 - 1e-6
    else:
        assert compare_states(got, ref, eps=1e-14, atol=1e-12) >= 1 - 1e-10
        assert g.peak_nnz() == o.peak()


def test_nonherm_one_step_n256_matches_oracle(sqs):
    cfg = Q.config4_nonherm(seed=4, N=256, half_band=8, kappa=10.0, T=2000)
    circ = _mid_step(cfg, Q.walk_step_nh)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ)
    assert g.nnz() == o.nnz()
    assert compare_states(g.to_dict(), o.to_dict(), eps=1e-14, atol=1e-12) >= 1 - 1e-10


def test_nonherm_full_size_steps_keep_norm(sqs):
    """N = 1024: two walk steps keep the norm, and the FP32-storage state
    stays close to the FP64 one."""
    cfg = Q.config4_nonherm(seed=4, N=1024, half_band=8, kappa=10.0, T=2000)
    circ = Q.walk_circuit_nh(cfg, n_steps=2)
    g64 = sqs.run_circuit(circ)
    g32 = sqs.run_circuit(circ, amp32=True)
    d64, d32 = g64.to_dict(), g32.to_dict()
    n2 = sum(abs(v) ** 2 for v in d64.values())
    assert abs(n2 - 1) < 1e-10
    ov = sum(np.conj(v) * d32.get(k, 0) for k, v in d64.items())
    n32 = sum(abs(v) ** 2 for v in d32.values())
    assert abs(ov) ** 2 / (n2 * n32) >= 1 - 1e-6


def _flag_error(state, cfg):
    """Distance between the normalised flagged block of a walk state and
    x/||x|| for x = A^-1 b (dense solve), after removing the global phase,
    and the flagged block's probability."""
    v = Q.solution_block(state, cfg)
    x = np.linalg.solve(cfg["A"], cfg["b"])
    x = x / np.linalg.norm(x)
    pv = float(np.vdot(v, v).real)
    vn = v / math.sqrt(pv)
    ph = np.vdot(x, vn)
    return float(np.linalg.norm(vn * np.conj(ph) / abs(ph) - x)), pv


def test_full_length_walk_n16_matches_oracle(sqs):
    """The whole walk (T = 2000 steps) at N = 16, element by element against
    the oracle; the flagged block against the dense solve."""
    cfg = Q.config4(seed=4, N=16, half_band=4, kappa=10.0, T=2000)
    circ = Q.walk_circuit(cfg)
    o = oracle.run_circuit(circ)
    g = sqs.run_circuit(circ)
    ref = o.to_dict()
    got = g.to_dict()
    assert compare_states(got, ref, eps=1e-14, atol=1e-12) >= 1 - 1e-10
    assert g.peak_nnz() == o.peak()
    err, p = _flag_error(got, cfg)
    assert err <= 10 * cfg["kappa"] / cfg["T"] and p >= 0.5
    # FP32 storage over 158004 gates: the fidelity bar, and amplitudes within
    # the drift of that many roundings of 2^-24.
    g32 = sqs.run_circuit(circ, amp32=True).to_dict()
    keys = sorted(set(ref) | set(g32))
    a = np.array([ref.get(k, 0) for k in keys])
    b = np.array([g32.get(k, 0) for k in keys])
    fid = abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)
    assert fid >= 1 - 1e-6
    assert np.max(np.abs(a - b)) < 1e-4


def _walk_n1024(sqs, kappa, T, with_fp32):
    """Runs the N = 1024 walk (half-bandwidth 8, condition number kappa, T
    steps), recording at 10 schedule points: the norm (FP64) and, with
    with_fp32, the fidelity of the FP32-storage state with the FP64 one at
    every point.  Returns the final flagged-block error and probability."""
    cfg = Q.config4(seed=4, N=1024, half_band=8, kappa=kappa, T=T)
    tabs = cfg["tables"]
    states = [sqs.State(cfg["widths"], capacity_hint=1 << 23, eps=cfg["eps"])]
    if with_fp32:
        states.append(sqs.State(cfg["widths"], capacity_hint=1 << 23, eps=cfg["eps"], amp32=True))
    for g in states:
        for gate in cfg["prep"]:
            g.apply(gate, tabs)
    done = 0
    for point in cfg["points"]:
        for m in range(done, point):
            gates = Q.walk_step(cfg, cfg["steps"][m])
            for g in states:
                for gate in gates:
                    g.apply(gate, tabs)
        done = point
        lo, hi, a64 = states[0].export()
        assert abs(np.sum(np.abs(a64) ** 2) - 1.0) < 1e-9
        if with_fp32:
            lo32, hi32, a32 = states[1].export()
            assert not hi.any() and not hi32.any()
            _, i64, i32 = np.intersect1d(lo, lo32, assume_unique=True, return_indices=True)
            ov = np.vdot(a64[i64], a32[i32])
            fid = abs(ov) ** 2 / (np.sum(np.abs(a64) ** 2) * np.sum(np.abs(a32) ** 2))
            assert fid >= 1 - 1e-6, (point, fid)
    for g in states:
        g.close()
    return _flag_error(dict(zip(lo.tolist(), a64.tolist())), cfg)


def test_full_length_walk_n1024(sqs):
    """The specified walk: N = 1024, half-bandwidth 8, T = 2000 steps at 10
    schedule points, condition numbers 10, 50 and 100, FP64 and FP32 storage.
    Checked against the dense solve x = A^-1 b through the error of the
    final flagged block, along the shape of the adiabatic bound eps <= theta
    / T with theta = O(kappa) (Sec. III.C): at T = 2000 the error grows with
    kappa and stays below 10 kappa / T (a loose envelope: the oracle's own
    full walks at N = 16 give eps T / kappa between 0.3 and 1.4), and at
    kappa = 10 it is smaller at T = 2000 than at T = 500.  The norm stays 1
    and the FP32-storage state keeps fidelity >= 1 - 1e-6 with the FP64 one
    at every schedule point."""
    errs = {}
    for kappa in (10.0, 50.0, 100.0):
        err, p = _walk_n1024(sqs, kappa, 2000, with_fp32=True)
        assert p >= 0.5
        assert err <= 10 * kappa / 2000, (kappa, err)
        errs[kappa] = err
    assert errs[10.0] < errs[50.0] < errs[100.0], errs
    err500, _ = _walk_n1024(sqs, 10.0, 500, with_fp32=False)
    assert err500 > errs[10.0], (err500, errs[10.0])

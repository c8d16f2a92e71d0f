"""Seeded synthetic workloads shaped like the paper's, as gate lists.

This module only draws random numbers and writes gate descriptors: it holds
none of the simulation arithmetic, so both the CPU oracle (tests) and the CUDA
path (binding, bench) consume its output.

Gate-list format: a circuit is a dict
    {"widths": [w_0, ...], "eps": 1e-14, "tables": [np.ndarray, ...],
     "gates": [gate, ...], "name": str}
and each gate is a tuple:
    ("h", reg, bit, ctrls)                      Hadamard (Sec. II.A)
    ("ry", reg, bit, theta, ctrls)              RY(theta)
    ("u1q", reg, bit, m2x2, ctrls)              general 2x2, m[row=out][col=in]
    ("ry_reg", reg, bit, angle_reg, scale, offset, ctrls)
                                                RY(scale*value(angle_reg)+offset)
    ("x", reg, bit, ctrls)                      X / CNOT / Toffoli (FlipBool)
    ("add"|"sub", dst, src_reg, const, ctrls)   dst +-= src (src_reg<0: const)
    ("swap", r1, r2, ctrls)                     register exchange
    ("muladd", dst, a, b, ctrls)                dst += a * b (mod 2^w)
    ("mulc", dst, c, ctrls)                     dst *= c (mod 2^w), c odd
    ("divxor", dst, a, b, ctrls)                dst ^= a // b (0 when b = 0)
    ("phase", preds, phi)                       a *= e^{i phi} where preds hold
    ("qload"|"qunload", addr_reg, data_reg, t)  data ^= tables[t][addr]; addr_reg
                                                may be (first, count): the address
                                                is then consecutive registers
                                                concatenated, the first lowest
    ("prune", eps)
with ctrls / preds a tuple of (reg, bit, value) triples.
"""
from __future__ import annotations

import math

import numpy as np

BRANCHING = ("h", "ry", "u1q", "ry_reg")


def _qubits(widths):
    return [(r, b) for r, w in enumerate(widths) for b in range(w)]


def random_circuit(widths, n_gates, seed, kinds=("x", "cx", "ccx", "ry", "phase", "h"),
                   tables=(), eps=1e-14, max_ctrl=2):
    """Uniform random gates over distinct qubits (no capacity control)."""
    rng = np.random.default_rng(seed)
    qs = _qubits(widths)
    gates = []
    for _ in range(n_gates):
        gates.append(_draw_gate(rng, kinds, qs, widths, len(tables), max_ctrl))
    return {"widths": list(widths), "eps": eps, "tables": list(tables), "gates": gates,
            "name": f"random-{seed}"}


def _draw_gate(rng, kinds, qs, widths, n_tables, max_ctrl=2):
    k = kinds[rng.integers(len(kinds))]
    pick = rng.choice(len(qs), size=min(len(qs), 3), replace=False)
    t, c1, c2 = (qs[i] for i in pick) if len(pick) == 3 else (qs[pick[0]],) * 3
    if k == "x":
        return ("x", t[0], t[1], ())
    if k == "cx":
        return ("x", t[0], t[1], ((c1[0], c1[1], 1),))
    if k == "ccx":
        return ("x", t[0], t[1], ((c1[0], c1[1], 1), (c2[0], c2[1], 1)))
    if k == "ry":
        return ("ry", t[0], t[1], float(rng.uniform(0, 2 * math.pi)), ())
    if k == "cry":
        return ("ry", t[0], t[1], float(rng.uniform(0, 2 * math.pi)), ((c1[0], c1[1], 1),))
    if k == "phase":
        return ("phase", ((t[0], t[1], 1),), float(rng.uniform(0, 2 * math.pi)))
    if k == "cphase":
        return ("phase", ((t[0], t[1], 1), (c1[0], c1[1], int(rng.integers(2)))),
                float(rng.uniform(0, 2 * math.pi)))
    if k == "h":
        return ("h", t[0], t[1], ())
    if k == "ch":
        return ("h", t[0], t[1], ((c1[0], c1[1], int(rng.integers(2))),))
    if k == "u1q":
        return ("u1q", t[0], t[1], random_unitary(rng), ())
    if k == "cu1q":
        return ("u1q", t[0], t[1], random_unitary(rng), ((c1[0], c1[1], 1),))
    if k == "diag":
        a, b = rng.uniform(0, 2 * math.pi, 2)
        return ("u1q", t[0], t[1], np.array([[np.exp(1j * a), 0], [0, np.exp(1j * b)]]), ())
    if k == "adiag":
        a, b = rng.uniform(0, 2 * math.pi, 2)
        return ("u1q", t[0], t[1], np.array([[0, np.exp(1j * a)], [np.exp(1j * b), 0]]), ())
    if k in ("add", "sub"):
        dst = int(rng.integers(len(widths)))
        others = [r for r in range(len(widths)) if r != dst]
        if others and rng.integers(2):
            src = int(others[rng.integers(len(others))])
            return (k, dst, src, 0, ())
        return (k, dst, -1, int(rng.integers(0, 2 ** min(widths[dst], 62))), ())
    if k == "swap":
        eq = [(a, b) for a in range(len(widths)) for b in range(len(widths))
              if a < b and widths[a] == widths[b]]
        a, b = eq[rng.integers(len(eq))]
        return ("swap", a, b, ())
    if k == "qram":
        return ("qload", 0, 1, int(rng.integers(n_tables)))
    if k in ("muladd", "divxor"):
        if len(widths) < 3:
            return ("x", t[0], t[1], ())
        dst, a, b = (int(r) for r in rng.choice(len(widths), size=3, replace=False))
        return (k, dst, a, b, ())
    if k == "mulc":
        dst = int(rng.integers(len(widths)))
        return ("mulc", dst, int(rng.integers(0, 2 ** min(widths[dst], 62))) | 1, ())
    raise ValueError(k)


def random_unitary(rng):
    """Haar-ish 2x2 unitary from a QR decomposition of a complex Gaussian."""
    z = (rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def inverse_gate(g):
    """Adjoint of one gate (for apply-then-inverse checks)."""
    op = g[0]
    if op == "h" or op == "x" or op == "swap" or op in ("qload", "qunload"):
        return g
    if op == "ry":
        return ("ry", g[1], g[2], -g[3], g[4])
    if op == "u1q":
        return ("u1q", g[1], g[2], np.conj(np.asarray(g[3], np.complex128)).T, g[4])
    if op == "ry_reg":
        return ("ry_reg", g[1], g[2], g[3], -g[4], -g[5], g[6])
    if op == "add":
        return ("sub",) + tuple(g[1:])
    if op == "sub":
        return ("add",) + tuple(g[1:])
    if op == "phase":
        return ("phase", g[1], -g[2])
    if op == "divxor":
        return g
    if op == "mulc":
        # the inverse of an odd c modulo 2^64 is its inverse modulo 2^w too
        return ("mulc", g[1], pow(int(g[2]), -1, 2 ** 64), g[3])
    raise ValueError(op)


def inverse_circuit(circ):
    out = dict(circ)
    out["gates"] = [inverse_gate(g) for g in reversed(circ["gates"]) if g[0] != "prune"]
    out["name"] = circ.get("name", "") + "-inverse"
    return out


# ---------------------------------------------------------------------------
# Config 1: 20 qubits in 3 registers (addr 8, data 8, anc 4), uint64 keys, FP64.
# ---------------------------------------------------------------------------
CFG1_WIDTHS = [8, 8, 4]
CFG1_KINDS = ("x", "cx", "ccx", "ry", "phase", "h")


def config1_prefix(seed=1):
    """H on all 8 addr bits, then QRAM load of a seeded 256-entry uint8 table."""
    rng = np.random.default_rng(seed)
    table = rng.integers(0, 256, size=256, dtype=np.uint64).astype(np.uint8)
    gates = [("h", 0, b, ()) for b in range(8)]
    gates.append(("qload", 0, 1, 0))
    return {"widths": list(CFG1_WIDTHS), "eps": 1e-14, "tables": [table], "gates": gates,
            "name": f"config1-seed{seed}"}, rng


def config1_candidates(rng):
    """One seeded candidate gate for the 200-gate body of config 1."""
    return _draw_gate(rng, CFG1_KINDS, _qubits(CFG1_WIDTHS), CFG1_WIDTHS, 1)


def config1(seed=1, n_gates=200, cap=4096, accept=None):
    """Config 1 with its nnz cap.

    The cap is enforced by rejection: ``accept(circuit_so_far, gate)`` returns
    True when the gate keeps the state's branch count <= cap.  The caller passes
    a simulator-backed predicate (the tests pass the oracle); without one every
    drawn gate is accepted.
    """
    circ, rng = config1_prefix(seed)
    while len(circ["gates"]) < 9 + n_gates:
        g = config1_candidates(rng)
        if accept is None or accept(circ, g):
            circ["gates"].append(g)
    return circ


def _decode_gate(g, remap):
    """A stored gate (JSON lists) as a gate tuple, registers renumbered."""
    def ctrls(cs):
        return tuple((remap[c[0]], c[1], c[2]) for c in cs)
    op = g[0]
    if op in ("h", "x"):
        return (op, remap[g[1]], g[2], ctrls(g[3]))
    if op == "ry":
        return (op, remap[g[1]], g[2], float(g[3]), ctrls(g[4]))
    if op == "phase":
        return (op, ctrls(g[1]), float(g[2]))
    raise ValueError(f"config 1 has no gate {op!r}")


def config1_batch(stored, inst_bits=16, seed=1):
    """2^inst_bits instances of config 1 in one state.

    Every instance runs the same stored gate list (config 1, seed 1, its nnz
    cap enforced on the oracle); instance i loads its own seeded 256-entry
    uint8 table (instance 0: the seed-1 table), so the instances' states
    differ.  Registers: addr 8, inst, data 8, anc 4 -- the instance register
    sits next to addr so that the QRAM address (addr, inst) spans consecutive
    registers; the instances start in uniform superposition (H on every
    instance qubit).  `stored` is the dict of tests/golden/config1_seed1_gates.json.
    """
    remap = {0: 0, 1: 2, 2: 3}
    widths = [8, inst_bits, 8, 4]
    n_inst = 1 << inst_bits
    base = config1_prefix(seed)[0]["tables"][0]
    rng = np.random.default_rng(seed + 1000)
    table = rng.integers(0, 256, size=n_inst * 256, dtype=np.uint64).astype(np.uint8)
    table[:256] = base
    gates = [("h", 1, b, ()) for b in range(inst_bits)]
    for g in stored["gates"]:
        if g[0] == "qload":
            gates.append(("qload", (0, 2), remap[g[2]], 0))
        else:
            gates.append(_decode_gate(g, remap))
    return {"widths": widths, "eps": stored["eps"], "tables": [table], "gates": gates,
            "n_inst": n_inst, "inst_bits": inst_bits,
            "name": f"config1-batch{n_inst}-seed{seed}"}


def config1_from_stored(stored, seed=1):
    """Config 1 itself from the stored gate list (registers addr, data, anc)."""
    ident = {0: 0, 1: 1, 2: 2}
    gates = [("qload", 0, 1, 0) if g[0] == "qload" else _decode_gate(g, ident)
             for g in stored["gates"]]
    table = config1_prefix(seed)[0]["tables"][0]
    return {"widths": list(stored["widths"]), "eps": stored["eps"], "tables": [table],
            "gates": gates, "name": f"config1-seed{seed}"}


def config1_instance_table(batch, i):
    """The 256-entry table instance i of a config-1 batch loads."""
    return batch["tables"][0][i * 256:(i + 1) * 256]


# ---------------------------------------------------------------------------
# Config 2: 64 qubits = four 16-bit registers in one uint64 key, FP64.
# 24 branching gates (16 H of which 8 on reserved cancel qubits, 8 RY) interleaved
# with 500 permutation / phase gates, then 8 re-applied H on the cancel qubits.
# ---------------------------------------------------------------------------
CFG2_WIDTHS = [16, 16, 16, 16]


def config2(seed=2, n_branch=24, n_perm=500, n_cancel=8, widths=None):
    """Large sparse random circuit.

    The n_cancel "cancel qubits" are bits of the last register.  Each gets one H
    among the branching gates and a second H at the end; no other gate touches
    or reads them in between, so every re-applied H merges all pairs and halves
    the branch count exactly.  The other branching gates (H, then RY) hit
    distinct qubits never branched before; the peak is 2^n_branch when none of
    them finds partner branches."""
    widths = list(widths or CFG2_WIDTHS)
    rng = np.random.default_rng(seed)
    last = len(widths) - 1
    cancel_bits = rng.choice(widths[last], size=n_cancel, replace=False)
    cancel = [(last, int(b)) for b in cancel_bits]
    cset = set(cancel)
    free = [q for q in _qubits(widths) if q not in cset]
    n_h = 16 * n_branch // 24
    fresh_idx = rng.choice(len(free), size=n_branch - n_cancel, replace=False)
    fresh = [free[i] for i in fresh_idx]
    branch = [("h", q[0], q[1], ()) for q in cancel]
    for q in fresh:
        if len(branch) < n_h:
            branch.append(("h", q[0], q[1], ()))
        else:
            branch.append(("ry", q[0], q[1], float(rng.uniform(0.1, 2 * math.pi - 0.1)), ()))
    order = rng.permutation(len(branch))
    branch = [branch[i] for i in order]
    slots = np.sort(rng.choice(n_perm + 1, size=n_branch, replace=True))
    gates = []
    bi = 0
    for p in range(n_perm + 1):
        while bi < n_branch and slots[bi] == p:
            gates.append(branch[bi])
            bi += 1
        if p == n_perm:
            break
        gates.append(_perm_gate(rng, widths, free))
    for q in cancel:
        gates.append(("h", q[0], q[1], ()))
    return {"widths": widths, "eps": 1e-14, "tables": [], "gates": gates,
            "name": f"config2-seed{seed}-b{n_branch}-p{n_perm}", "cancel": cancel}


def _perm_gate(rng, widths, free):
    """CNOT / Toffoli / X / add-mod-2^16 / phase, never touching a cancel qubit
    (free lists the allowed qubits; add-mod only between registers that hold no
    cancel qubit)."""
    k = ("cx", "ccx", "x", "add", "phase")[rng.integers(5)]
    pick = rng.choice(len(free), size=3, replace=False)
    t, c1, c2 = (free[i] for i in pick)
    if k == "x":
        return ("x", t[0], t[1], ())
    if k == "cx":
        return ("x", t[0], t[1], ((c1[0], c1[1], 1),))
    if k == "ccx":
        return ("x", t[0], t[1], ((c1[0], c1[1], 1), (c2[0], c2[1], 1)))
    if k == "phase":
        return ("phase", ((t[0], t[1], 1),), float(rng.uniform(0, 2 * math.pi)))
    # add-mod-2^w on registers: both must be free of cancel qubits so that the
    # cancel qubits stay untouched between their two H gates.
    free_set = set(free)
    clean = [r for r in range(len(widths))
             if all((r, b) in free_set for b in range(widths[r]))]
    if len(clean) >= 2:
        dst, src = rng.choice(clean, size=2, replace=False)
        return ("add", int(dst), int(src), 0, ())
    if len(clean) == 1:
        return ("add", int(clean[0]), -1, int(rng.integers(1, 2 ** widths[clean[0]])), ())
    # No register is free of cancel qubits: a controlled X instead.
    return ("x", t[0], t[1], ((c1[0], c1[1], 1),))


# ---------------------------------------------------------------------------
# Config 3: QRAM-heavy, 128-bit keys: addr 20 / data 32 / acc 32.
# ---------------------------------------------------------------------------
def config3(seed=3, addr_bits=20, rounds=50, ry_bits=4):
    rng = np.random.default_rng(seed)
    widths = [addr_bits, 32, 32]
    table = rng.integers(0, 2 ** 32, size=2 ** addr_bits, dtype=np.uint64).astype(np.uint32)
    gates = [("h", 0, b, ()) for b in range(addr_bits)]
    for _ in range(rounds):
        gates.append(("qload", 0, 1, 0))
        gates.append(("add", 2, 1, 0, ()))
        bits = rng.choice(32, size=ry_bits, replace=False)
        thetas = rng.uniform(0.1, 2 * math.pi - 0.1, size=ry_bits)
        for b, th in zip(bits, thetas):
            gates.append(("ry", 1, int(b), float(th), ()))
        for b, th in reversed(list(zip(bits, thetas))):
            gates.append(("ry", 1, int(b), float(-th), ()))
        gates.append(("qunload", 0, 1, 0))
    return {"widths": widths, "eps": 1e-14, "tables": [table], "gates": gates,
            "name": f"config3-seed{seed}-a{addr_bits}-r{rounds}"}


def random_state(widths, n, seed, pair_fraction=0.5, target=None):
    """A seeded sparse input state of n distinct keys over sum(widths) bits with
    complex Gaussian amplitudes (not normalised).  When ``target`` = (reg, bit)
    is given, a fraction ``pair_fraction`` of the keys come with their partner
    across that bit.  Returns (lo, hi, amps) in a seeded random order."""
    rng = np.random.default_rng(seed)
    total = sum(widths)
    words = 2 if total > 64 else 1
    mask_lo = np.uint64((1 << min(total, 64)) - 1)
    mask_hi = np.uint64((1 << max(total - 64, 0)) - 1)
    bpos = None if target is None else sum(widths[: target[0]]) + target[1]
    n_base = n if bpos is None else int(math.ceil(n / (1.0 + pair_fraction)))
    n_pair = n - n_base
    base_lo = np.zeros(0, np.uint64)
    base_hi = np.zeros(0, np.uint64)
    while base_lo.shape[0] < n_base:
        m = 2 * (n_base - base_lo.shape[0]) + 16
        lo = rng.integers(0, 2 ** 64, size=m, dtype=np.uint64, endpoint=False) & mask_lo
        hi = (rng.integers(0, 2 ** 64, size=m, dtype=np.uint64, endpoint=False) & mask_hi
              if words == 2 else np.zeros(m, np.uint64))
        if bpos is not None:
            if bpos < 64:
                lo &= ~np.uint64(1 << bpos)
            else:
                hi &= ~np.uint64(1 << (bpos - 64))
        lo = np.concatenate([base_lo, lo])
        hi = np.concatenate([base_hi, hi])
        if words == 1:
            _, first = np.unique(lo, return_index=True)
        else:
            both = np.stack([hi, lo], axis=1)
            _, first = np.unique(both, axis=0, return_index=True)
        first = np.sort(first)
        base_lo, base_hi = lo[first], hi[first]
    base_lo, base_hi = base_lo[:n_base], base_hi[:n_base]
    lo_all, hi_all = [base_lo], [base_hi]
    if n_pair > 0:
        sel = rng.choice(n_base, size=n_pair, replace=False)
        plo, phi = base_lo[sel].copy(), base_hi[sel].copy()
        if bpos < 64:
            plo |= np.uint64(1 << bpos)
        else:
            phi |= np.uint64(1 << (bpos - 64))
        lo_all.append(plo)
        hi_all.append(phi)
    lo = np.concatenate(lo_all)
    hi = np.concatenate(hi_all)
    perm = rng.permutation(n)
    amps = (rng.normal(size=n) + 1j * rng.normal(size=n)) / math.sqrt(2 * max(n, 1))
    return lo[perm], hi[perm], amps


def config4(seed=4, N=1024, half_band=8, kappa=10.0, T=2000, n_points=10):
    """The quantum linear-system walk (Sec. III.C, Supp. D) on one seeded
    symmetric positive-definite banded system; see qlss.config4."""
    from . import qlss
    return qlss.config4(seed=seed, N=N, half_band=half_band, kappa=kappa, T=T,
                        n_points=n_points)

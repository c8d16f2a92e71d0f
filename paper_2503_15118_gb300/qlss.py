"""The quantum linear-system workload (Sec. III.C, Supp. D) as gate lists.

An adiabatic walk W(s) = R U_H(s) (Supp. D, Fig. S1(c)) for a symmetric
positive-definite A: the block-encoding U_H(s) of
    H(s) = [[0, A(f) Q_b], [Q_b A(f), 0]],  A(f) = (1 - f) I + f A,
    Q_b = I - |b><b|,
built from the block-encoding U_A of A (Supp. D: U_A = U_SWAP U_R^dag U_L, with
U_L and U_R preparing columns and column norms from rotation-angle trees held
in QRAM and applied as register-valued RY rotations), the state-preparation
U_b of b, and R = i(2|0><0|_anc - I) (Supp. D).  Like workloads.py, this
module only builds inputs (matrices, angle tables, gate tuples); the
simulation arithmetic lives in the simulators that consume them.

Registers (low bits first):
    BOT (n)  the ancilla register of U_A, where U_L prepares a column
    TOP (n)  the system register |j>, where U_R acts
    [INST]   batched instances only: the instance id (never acted on)
    C (1)    LCU ancilla of A(f) = (1-f) I + f A
    A2 (1)   LCU ancilla of Q_b = (I + R_b) / 2
    AH (1)   the block qubit a_h of H(s)
    Q (32)   QRAM data register: rotation angles, 4 pi * v / 2^32
The block-encoding ancillas ("anc" of R) are C, A2, BOT and Q; the system of
H(s) is AH and TOP.

Readings (the paper prints U_A and R but not the circuits of Fig. S1(a)):
  * U_{A(f)}: one ancilla C prepared by RY(theta_f) with cos^2(theta_f/2)
    proportional to (1 - f) and sin^2 to f ||A||_F; U_A controlled on C = 1;
    RY(-theta_f).  Normalisation lambda = (1 - f) + f ||A||_F.
  * U_Q: H on A2, then R_b = U_b (I - 2|0><0|) U_b^dag controlled on A2 = 1,
    then H on A2, so that <0|U_Q|0> = (I + R_b) / 2 = Q_b.  U_b = H on every
    TOP qubit (b is the normalised all-ones vector, Sec. III.C).
  * U_H = X_AH (|0><0|_AH (x) U_M^dag + |1><1|_AH (x) U_M), U_M = U_{A(f)} U_Q,
    so that <0|_anc U_H |0>_anc = H(s) / lambda.
  * Schedule f(s): the AQC(p) schedule of An and Lin with p = 1.5,
    f(s) = kappa / (kappa - 1) * (1 - (1 + s (kappa^(p-1) - 1))^(1 / (1 - p))).
  * A: S = (B + B^T) / 2 for B with N(0, 1) entries on |i - j| <= half_band,
    then A = alpha S + beta I maps spec(S) onto [1 / kappa, 1].
  * Angle trees: level l rotates qubit n-1-l (most significant first) by an
    angle looked up at the prefix already prepared; internal levels split the
    subtree masses, the last level carries the signs of the entries.
"""
from __future__ import annotations

import math

import numpy as np

ANGLE_BITS = 32
ANGLE_SCALE = 4.0 * math.pi / float(1 << ANGLE_BITS)  # RY has period 4 pi

BOT, TOP = 0, 1


def registers(n, inst_bits=0, nonherm=False):
    """Widths and register ids for system size 2^n (and an instance register;
    nonherm adds the block qubit a_1 of the non-Hermitian embedding)."""
    widths = [n, n]
    ids = {"BOT": 0, "TOP": 1}
    if inst_bits:
        ids["INST"] = len(widths)
        widths.append(inst_bits)
    extra = (("A1", 1),) if nonherm else ()
    for name, w in (("C", 1), ("A2", 1), ("AH", 1)) + extra + (("Q", ANGLE_BITS),):
        ids[name] = len(widths)
        widths.append(w)
    return widths, ids


def spd_banded(N, half_band, kappa, rng):
    """Symmetric positive-definite banded matrix with condition number kappa."""
    i = np.arange(N)
    band = np.abs(i[:, None] - i[None, :]) <= half_band
    B = rng.standard_normal((N, N)) * band
    S = 0.5 * (B + B.T)
    ev = np.linalg.eigvalsh(S)
    lo, hi = float(ev[0]), float(ev[-1])
    if hi - lo < 1e-12:
        return np.eye(N)
    alpha = (1.0 - 1.0 / kappa) / (hi - lo)
    beta = 1.0 / kappa - alpha * lo
    return alpha * S + beta * np.eye(N)


def angle_code(theta):
    """uint32 codes of angles theta (radians), taken modulo 4 pi."""
    t = np.mod(np.asarray(theta, np.float64), 4.0 * math.pi)
    return (np.rint(t / ANGLE_SCALE).astype(np.uint64) % (1 << ANGLE_BITS)).astype(np.uint32)


def tree_angles(x):
    """Angles (radians) of the rotation tree preparing the real unit vector x
    (length 2^n) from |0>: angles[l][p] for level l and prefix p (l bits)."""
    x = np.asarray(x, np.float64)
    n = int(round(math.log2(x.shape[0])))
    mass = x * x
    out = []
    for l in range(n):
        size = 1 << (n - l)
        if l < n - 1:
            m = mass.reshape(1 << l, size)
            m0 = m[:, : size // 2].sum(axis=1)
            m1 = m[:, size // 2:].sum(axis=1)
            out.append(2.0 * np.arctan2(np.sqrt(m1), np.sqrt(m0)))
        else:
            pair = x.reshape(1 << l, 2)
            out.append(2.0 * np.arctan2(pair[:, 1], pair[:, 0]))
    return out


def tables_for(A):
    """QRAM angle tables of U_L (address = (BOT, TOP) span, N * N entries) and
    U_R (address = TOP, N entries) per level, and ||A||_F."""
    N = A.shape[0]
    n = int(round(math.log2(N)))
    col = np.linalg.norm(A, axis=0)
    nf = float(np.linalg.norm(A))
    tl = [np.zeros(N * N, np.uint32) for _ in range(n)]
    tr = [np.zeros(N, np.uint32) for _ in range(n)]
    # The entry of level l depends only on the prefix (the l bits above the
    # rotated qubit): the rotation changes the target bit between load and
    # unload, and the lower bits are whatever the input holds, so every
    # address with the same prefix reads the same angle and unload always
    # restores the data register.
    m = np.arange(N, dtype=np.int64)
    for k in range(N):
        if col[k] == 0.0:
            continue
        ang = tree_angles(A[:, k] / col[k])
        for l in range(n):
            tl[l][k * N: (k + 1) * N] = angle_code(ang[l])[m >> (n - l)]
    ang = tree_angles(col / nf)
    for l in range(n):
        tr[l][:] = angle_code(ang[l])[m >> (n - l)]
    return tl, tr, nf


def u_l(n, ids, t_l, ctrls, dagger=False, span=2):
    Q, sc = ids["Q"], (-ANGLE_SCALE if dagger else ANGLE_SCALE)
    g = []
    for l in (reversed(range(n)) if dagger else range(n)):
        g += [("qload", (BOT, span), Q, t_l[l]),
              ("ry_reg", BOT, n - 1 - l, Q, sc, 0.0, tuple(ctrls)),
              ("qunload", (BOT, span), Q, t_l[l])]
    return g


def u_r(n, ids, t_r, ctrls, dagger=False, span=1):
    Q, sc = ids["Q"], (-ANGLE_SCALE if dagger else ANGLE_SCALE)
    addr = TOP if span == 1 else (TOP, span)
    g = []
    for l in (reversed(range(n)) if dagger else range(n)):
        g += [("qload", addr, Q, t_r[l]),
              ("ry_reg", TOP, n - 1 - l, Q, sc, 0.0, tuple(ctrls)),
              ("qunload", addr, Q, t_r[l])]
    return g


def u_a(n, ids, t_l, t_r, ctrls, dagger=False, span_l=2, span_r=1):
    """U_A = U_SWAP U_R^dag U_L (Supp. D), all controlled by ctrls."""
    c = tuple(ctrls)
    if not dagger:
        return (u_l(n, ids, t_l, c, False, span_l) + u_r(n, ids, t_r, c, True, span_r)
                + [("swap", TOP, BOT, c)])
    return ([("swap", TOP, BOT, c)] + u_r(n, ids, t_r, c, False, span_r)
            + u_l(n, ids, t_l, c, True, span_l))


def lcu_angle(f, norm):
    """theta with cos^2(theta/2) : sin^2(theta/2) = (1 - f) : f * norm."""
    return 2.0 * math.atan2(math.sqrt(f * norm), math.sqrt(1.0 - f))


def u_af(n, ids, t_l, t_r, theta, ctrls, dagger=False, theta_gate=None, **kw):
    """Block-encoding of A(f) = (1 - f) I + f A by an LCU on C.  theta_gate,
    when given, replaces the fixed RY(theta) preparation (batched instances
    take their angle from a table)."""
    C = ids["C"]
    c = tuple(ctrls)
    prep = theta_gate(False, c) if theta_gate else [("ry", C, 0, theta, c)]
    unprep = theta_gate(True, c) if theta_gate else [("ry", C, 0, -theta, c)]
    return prep + u_a(n, ids, t_l, t_r, c + ((C, 0, 1),), dagger, **kw) + unprep


def u_q(n, ids, ctrls):
    """Block-encoding of Q_b = I - |b><b| (Hermitian and self-inverse)."""
    A2 = ids["A2"]
    g = [("h", A2, 0, ())] + [("h", TOP, b, ()) for b in range(n)]
    pred = ((A2, 0, 1),) + tuple((TOP, b, 0) for b in range(n)) + tuple(ctrls)
    g += [("phase", pred, math.pi)]
    g += [("h", TOP, b, ()) for b in range(n)] + [("h", A2, 0, ())]
    return g


def u_h(n, ids, t_l, t_r, theta, theta_gate=None, **kw):
    """U_H = X_AH (|0><0| (x) U_M^dag + |1><1| (x) U_M), U_M = U_{A(f)} U_Q."""
    AH = ids["AH"]
    on, off = ((AH, 0, 1),), ((AH, 0, 0),)
    return (u_q(n, ids, on)
            + u_af(n, ids, t_l, t_r, theta, off, dagger=True, theta_gate=theta_gate, **kw)
            + u_af(n, ids, t_l, t_r, theta, on, dagger=False, theta_gate=theta_gate, **kw)
            + u_q(n, ids, off)
            + [("x", AH, 0, ())])


def reflection(n, ids):
    """R = i (2|0><0|_anc - I): -i everywhere, then -1 where every ancilla is 0."""
    pred = ((ids["C"], 0, 0), (ids["A2"], 0, 0)) + tuple((BOT, b, 0) for b in range(n)) \
        + tuple((ids["Q"], b, 0) for b in range(ANGLE_BITS))
    return [("phase", (), -0.5 * math.pi), ("phase", pred, math.pi)]


def schedule(s, kappa, p=1.5):
    """AQC(p) schedule f(s) (An and Lin), f(0) = 0, f(1) = 1."""
    if kappa <= 1.0:
        return s
    return kappa / (kappa - 1.0) * (1.0 - (1.0 + s * (kappa ** (p - 1.0) - 1.0)) ** (1.0 / (1.0 - p)))


def prepare_b(n):
    """|psi_0> = |0>_AH |b>_TOP |0>_anc with b the normalised all-ones vector."""
    return [("h", TOP, b, ()) for b in range(n)]


def config4(seed=4, N=1024, half_band=8, kappa=10.0, T=2000, n_points=10):
    """The linear-system walk on one seeded SPD banded system.  Returns the
    circuit pieces: widths, tables, eps, "prep" (b), "steps" (f of every walk
    step), "points" (steps after which the state is recorded) and A, b."""
    rng = np.random.default_rng(seed)
    n = int(round(math.log2(N)))
    if 1 << n != N:
        raise ValueError("N must be a power of two")
    A = spd_banded(N, half_band, kappa, rng)
    widths, ids = registers(n)
    t_l, t_r, nf = tables_for(A)
    tables = t_l + t_r
    ti_l, ti_r = list(range(n)), list(range(n, 2 * n))
    steps = [schedule(m / T, kappa) for m in range(T)]
    points = [int(round((i + 1) * T / n_points)) for i in range(n_points)]
    return {"widths": widths, "ids": ids, "n": n, "eps": 1e-14, "tables": tables,
            "t_l": ti_l, "t_r": ti_r, "norm_f": nf, "A": A, "b": np.full(N, N ** -0.5),
            "kappa": kappa, "T": T, "steps": steps, "points": points,
            "prep": prepare_b(n), "name": f"qlss-N{N}-k{kappa:g}-T{T}"}


def walk_step(cfg, f):
    """Gates of one walk step W(s) = R U_H(s) at schedule value f."""
    n, ids = cfg["n"], cfg["ids"]
    theta = lcu_angle(f, cfg["norm_f"])
    return u_h(n, ids, cfg["t_l"], cfg["t_r"], theta) + reflection(n, ids)


def walk_circuit(cfg, n_steps=None):
    """The whole walk (or its first n_steps steps) as one gate list."""
    steps = cfg["steps"] if n_steps is None else cfg["steps"][:n_steps]
    gates = list(cfg["prep"])
    for f in steps:
        gates += walk_step(cfg, f)
    return {"widths": cfg["widths"], "eps": cfg["eps"], "tables": cfg["tables"],
            "gates": gates, "name": cfg["name"]}


def solution_block(state, cfg):
    """The normalised flagged block of a walk state: amplitudes of |0>_AH |j>_TOP
    with every ancilla 0, as a vector over j (state: dict key -> amplitude)."""
    n, ids = cfg["n"], cfg["ids"]
    off = np.cumsum([0] + cfg["widths"])
    top_off = off[TOP]
    v = np.zeros(1 << n, np.complex128)
    keep_mask = ((1 << n) - 1) << top_off
    for k, a in state.items():
        if k & ~keep_mask:
            continue
        v[(k >> top_off) & ((1 << n) - 1)] = a
    return v


# ---- batched instances (config 5) ------------------------------------------
#
# Many independent systems share one state: an instance register INST (never
# acted on) selects the system, every instance-dependent quantity is a QRAM
# table indexed by INST, and instance i of size N_i = 2^{n_i} <= 2^n lives in
# the low n_i bits of TOP and BOT (the higher bits stay 0: levels of the angle
# trees above n_i carry angle 0, the identity).  A step register STEP counts
# walk steps (one "add" per step), so that the gates of every walk step are
# the same list and only the counter selects the schedule value f_i(s).

def batched_registers(n, inst_bits, step_bits):
    widths = [n, n, inst_bits, step_bits]
    ids = {"BOT": 0, "TOP": 1, "INST": 2, "STEP": 3}
    for name, w in (("C", 1), ("A2", 1), ("AH", 1), ("Q", ANGLE_BITS)):
        ids[name] = len(widths)
        widths.append(w)
    return widths, ids


def batched_tables(mats, n, inst_bits):
    """Per-level U_L tables (address BOT, TOP, INST) and U_R tables (address
    TOP, INST) for the instance matrices mats[i] (sizes 2^{n_i} <= 2^n)."""
    N = 1 << n
    n_inst = 1 << inst_bits
    tl = [np.zeros(n_inst * N * N, np.uint32) for _ in range(n)]
    tr = [np.zeros(n_inst * N, np.uint32) for _ in range(n)]
    norms = np.zeros(n_inst)
    m = np.arange(N, dtype=np.int64)
    for i, A in enumerate(mats):
        Ni = A.shape[0]
        ni = int(round(math.log2(Ni)))
        col = np.linalg.norm(A, axis=0)
        norms[i] = float(np.linalg.norm(A))
        for l in range(n):
            b = n - 1 - l  # the rotated qubit of global level l
            if b >= ni:
                continue  # above the instance's size: identity
            li = ni - 1 - b  # the instance's own level
            for k in range(Ni):
                if col[k] == 0.0:
                    continue
                ang = tree_angles(A[:, k] / col[k])
                base = (i * N + k) * N
                tl[l][base: base + N] = angle_code(ang[li])[(m >> (b + 1)) & ((1 << li) - 1)]
            ang = tree_angles(col / norms[i])
            tr[l][i * N: (i + 1) * N] = angle_code(ang[li])[(m >> (b + 1)) & ((1 << li) - 1)]
    return tl, tr, norms


def config5(seed=5, n_inst=256, n_min=3, n_max=7, kappa=(10.0, 50.0, 100.0), T=2000,
            max_half_band=16):
    """Batched linear-system walks: n_inst seeded SPD banded systems of sizes
    2^{U[n_min, n_max]}, half-bandwidths U{1 .. min(16, N/4)} and condition
    numbers drawn from `kappa`, all walked at once in one state."""
    rng = np.random.default_rng(seed)
    inst_bits = max(1, int(math.ceil(math.log2(n_inst))))
    step_bits = max(1, int(math.ceil(math.log2(T + 1))))
    n = n_max
    widths, ids = batched_registers(n, inst_bits, step_bits)
    mats, sizes, kap, hbs = [], [], [], []
    for _ in range(n_inst):
        ni = int(rng.integers(n_min, n_max + 1))
        Ni = 1 << ni
        hb = int(rng.integers(1, max(1, min(max_half_band, Ni // 4)) + 1))
        k = float(kappa[int(rng.integers(0, len(kappa)))])
        mats.append(spd_banded(Ni, hb, k, rng))
        sizes.append(Ni), kap.append(k), hbs.append(hb)
    tl, tr, norms = batched_tables(mats, n, inst_bits)
    # LCU angle of A(f) per (step, instance): address (INST, STEP).
    tf = np.zeros((1 << step_bits) << inst_bits, np.uint32)
    for mstep in range(T):
        s = mstep / T
        th = [lcu_angle(schedule(s, kap[i]), norms[i]) for i in range(n_inst)]
        tf[(mstep << inst_bits) + np.arange(n_inst)] = angle_code(th)
    # U_b: RY(pi / 2) on the instance's own TOP qubits, identity above.
    tb = [np.zeros(1 << inst_bits, np.uint32) for _ in range(n)]
    for b in range(n):
        tb[b][:n_inst] = angle_code([math.pi / 2 if b < int(math.log2(sizes[i])) else 0.0
                                     for i in range(n_inst)])
    tables = tl + tr + [tf] + tb
    cfg = {"widths": widths, "ids": ids, "n": n, "inst_bits": inst_bits, "step_bits": step_bits,
           "eps": 1e-14, "tables": tables, "t_l": list(range(n)),
           "t_r": list(range(n, 2 * n)), "t_f": 2 * n, "t_b": list(range(2 * n + 1, 3 * n + 1)),
           "mats": mats, "sizes": sizes, "kappa": kap, "half_band": hbs, "norms": norms,
           "n_inst": n_inst, "T": T, "name": f"qlss-batch{n_inst}-T{T}"}
    return cfg


def _batched_ub(cfg, dagger, ctrls):
    """U_b (or its inverse) with per-instance angles."""
    ids, n = cfg["ids"], cfg["n"]
    Qr, INST = ids["Q"], ids["INST"]
    sc = -ANGLE_SCALE if dagger else ANGLE_SCALE
    g = []
    for b in range(n):
        t = cfg["t_b"][b]
        g += [("qload", INST, Qr, t), ("ry_reg", TOP, b, Qr, sc, 0.0, tuple(ctrls)),
              ("qunload", INST, Qr, t)]
    return g


def batched_prep(cfg):
    """Uniform superposition over the instances, then |b_i> on every instance."""
    g = [("h", cfg["ids"]["INST"], b, ()) for b in range(cfg["inst_bits"])]
    return g + _batched_ub(cfg, False, ())


def _batched_uq(cfg, ctrls):
    ids, n = cfg["ids"], cfg["n"]
    A2 = ids["A2"]
    pred = ((A2, 0, 1),) + tuple((TOP, b, 0) for b in range(n)) + tuple(ctrls)
    return ([("h", A2, 0, ())] + _batched_ub(cfg, True, ()) + [("phase", pred, math.pi)]
            + _batched_ub(cfg, False, ()) + [("h", A2, 0, ())])


def batched_walk_step(cfg):
    """One walk step for every instance; identical for every step (the STEP
    register selects the schedule value and is incremented at the end)."""
    ids, n = cfg["ids"], cfg["n"]
    INST, STEP, C, Qr, AH = ids["INST"], ids["STEP"], ids["C"], ids["Q"], ids["AH"]
    span_l, span_r = 3, 2  # (BOT, TOP, INST) and (TOP, INST)

    def theta_gate(dagger, c):
        sc = -ANGLE_SCALE if dagger else ANGLE_SCALE
        return [("qload", (INST, 2), Qr, cfg["t_f"]), ("ry_reg", C, 0, Qr, sc, 0.0, c),
                ("qunload", (INST, 2), Qr, cfg["t_f"])]

    on, off = ((AH, 0, 1),), ((AH, 0, 0),)
    kw = {"span_l": span_l, "span_r": span_r}
    g = (_batched_uq(cfg, on)
         + u_af(n, ids, cfg["t_l"], cfg["t_r"], None, off, dagger=True, theta_gate=theta_gate,
                **kw)
         + u_af(n, ids, cfg["t_l"], cfg["t_r"], None, on, dagger=False, theta_gate=theta_gate,
                **kw)
         + _batched_uq(cfg, off)
         + [("x", AH, 0, ())])
    return g + reflection(n, ids) + [("add", STEP, -1, 1, ())]


def batched_circuit(cfg, n_steps):
    step = batched_walk_step(cfg)
    gates = batched_prep(cfg)
    for _ in range(n_steps):
        gates += step
    return {"widths": cfg["widths"], "eps": cfg["eps"], "tables": cfg["tables"],
            "gates": gates, "name": cfg["name"]}


def instance_block(state, cfg, i):
    """Flagged block of instance i: amplitudes of |0>_AH |j>_TOP |i>_INST with
    every ancilla 0 (any step count), over j < N_i."""
    ids = cfg["ids"]
    off = np.cumsum([0] + cfg["widths"])
    Ni = cfg["sizes"][i]
    mask_keep = (((1 << cfg["n"]) - 1) << int(off[TOP])) | \
        (((1 << cfg["inst_bits"]) - 1) << int(off[ids["INST"]])) | \
        (((1 << cfg["step_bits"]) - 1) << int(off[ids["STEP"]]))
    v = np.zeros(Ni, np.complex128)
    for k, a in state.items():
        if k & ~mask_keep:
            continue
        if (k >> int(off[ids["INST"]])) & ((1 << cfg["inst_bits"]) - 1) != i:
            continue
        j = (k >> int(off[TOP])) & ((1 << cfg["n"]) - 1)
        if j < Ni:
            v[j] = a
    return v


# ---- the non-Hermitian variant (Supp. D, second column of the table) --------
#
# A general (non-symmetric) A enters through the Hermitian embedding
#     bA = [[0, A], [A^T, 0]]   on (a_1, TOP),  |b_bold> = |0>_{a_1} |b>,
# with A(f) = (1 - f) (sigma_z (x) I) + f bA, so that A(0) gives H_0 and A(1)
# gives H_1, and the final flagged state |0>_AH |1>_{a_1} |A^-1 b> / norm
# (bA^-1 maps |0>|b> to |1>|A^-1 b>).
#   * U_bA = X_{a_1} (|0><0|_{a_1} (x) U_{A^T} + |1><1|_{a_1} (x) U_A): its
#     block is |1><0| (x) A^T / a + |0><1| (x) A / a = bA / a, a = ||A||_F
#     (A and A^T share the Frobenius norm).  U_{A^T} is U_A built from the
#     angle trees of A^T.
#   * U_{A(f)}: the LCU on C selects sigma_z on a_1 (a phase pi on a_1 = 1)
#     when C = 0 and U_bA when C = 1; lambda = (1 - f) + f ||A||_F as before.
#   * U_Q reflects about |0>_{a_1} U_b|0>: the phase predicate adds a_1 = 0.
# The ancillas of R are unchanged (C, A2, BOT, Q); a_1 belongs to the system.

def nonherm_banded(N, half_band, kappa, rng):
    """Banded, non-symmetric, indefinite A = D S with condition number kappa:
    S the symmetric positive-definite banded matrix of spd_banded and D a
    seeded diagonal of +-1 (orthogonal, so A has the singular values of S)."""
    S = spd_banded(N, half_band, kappa, rng)
    d = rng.choice(np.array([-1.0, 1.0]), size=N)
    if N > 1 and np.all(d == d[0]):
        d[-1] = -d[0]
    return d[:, None] * S


def u_bold_a(n, ids, tabs, ctrls, dagger=False):
    """U_bA = X_{a_1} (|0><0| (x) U_{A^T} + |1><1| (x) U_A), all under ctrls.
    tabs = (t_l(A), t_r(A), t_l(A^T), t_r(A^T)) as table-index lists."""
    A1 = ids["A1"]
    c = tuple(ctrls)
    t_l, t_r, t_l2, t_r2 = tabs
    sel = (u_a(n, ids, t_l2, t_r2, c + ((A1, 0, 0),), dagger)
           + u_a(n, ids, t_l, t_r, c + ((A1, 0, 1),), dagger))
    flip = [("x", A1, 0, c)]
    return sel + flip if not dagger else flip + sel


def u_af_nh(n, ids, tabs, theta, ctrls, dagger=False):
    """Block-encoding of A(f) = (1 - f) (sigma_z (x) I) + f bA (LCU on C)."""
    C, A1 = ids["C"], ids["A1"]
    c = tuple(ctrls)
    z = [("phase", c + ((C, 0, 0), (A1, 0, 1)), math.pi)]
    return ([("ry", C, 0, theta, c)] + z + u_bold_a(n, ids, tabs, c + ((C, 0, 1),), dagger)
            + [("ry", C, 0, -theta, c)])


def u_q_nh(n, ids, ctrls):
    """Block-encoding of Q_b_bold = I - |0><0|_{a_1} (x) |b><b|."""
    A2, A1 = ids["A2"], ids["A1"]
    g = [("h", A2, 0, ())] + [("h", TOP, b, ()) for b in range(n)]
    pred = ((A2, 0, 1), (A1, 0, 0)) + tuple((TOP, b, 0) for b in range(n)) + tuple(ctrls)
    g += [("phase", pred, math.pi)]
    g += [("h", TOP, b, ()) for b in range(n)] + [("h", A2, 0, ())]
    return g


def u_h_nh(n, ids, tabs, theta):
    """U_H = X_AH (|0><0| (x) U_M^dag + |1><1| (x) U_M), U_M = U_{A(f)} U_Q."""
    AH = ids["AH"]
    on, off = ((AH, 0, 1),), ((AH, 0, 0),)
    return (u_q_nh(n, ids, on)
            + u_af_nh(n, ids, tabs, theta, off, dagger=True)
            + u_af_nh(n, ids, tabs, theta, on, dagger=False)
            + u_q_nh(n, ids, off)
            + [("x", AH, 0, ())])


def config4_nonherm(seed=4, N=1024, half_band=8, kappa=10.0, T=2000, n_points=10):
    """The linear-system walk on one seeded non-Hermitian banded system (the
    pieces of config4, with A = D S and the tables of A and A^T)."""
    rng = np.random.default_rng(seed)
    n = int(round(math.log2(N)))
    if 1 << n != N:
        raise ValueError("N must be a power of two")
    A = nonherm_banded(N, half_band, kappa, rng)
    widths, ids = registers(n, nonherm=True)
    t_l, t_r, nf = tables_for(A)
    t_l2, t_r2, nf2 = tables_for(A.T)
    tables = t_l + t_r + t_l2 + t_r2
    tabs = tuple(list(range(i * n, (i + 1) * n)) for i in range(4))
    steps = [schedule(m / T, kappa) for m in range(T)]
    points = [int(round((i + 1) * T / n_points)) for i in range(n_points)]
    return {"widths": widths, "ids": ids, "n": n, "eps": 1e-14, "tables": tables,
            "tabs": tabs, "norm_f": nf, "A": A, "b": np.full(N, N ** -0.5),
            "kappa": kappa, "T": T, "steps": steps, "points": points,
            "prep": prepare_b(n), "nonherm": True,
            "name": f"qlss-nonherm-N{N}-k{kappa:g}-T{T}"}


def walk_step_nh(cfg, f):
    n, ids = cfg["n"], cfg["ids"]
    theta = lcu_angle(f, cfg["norm_f"])
    return u_h_nh(n, ids, cfg["tabs"], theta) + reflection(n, ids)


def walk_circuit_nh(cfg, n_steps=None):
    steps = cfg["steps"] if n_steps is None else cfg["steps"][:n_steps]
    gates = list(cfg["prep"])
    for f in steps:
        gates += walk_step_nh(cfg, f)
    return {"widths": cfg["widths"], "eps": cfg["eps"], "tables": cfg["tables"],
            "gates": gates, "name": cfg["name"]}


def solution_block_nh(state, cfg):
    """Amplitudes of |0>_AH |1>_{a_1} |j>_TOP with every ancilla 0, over j."""
    n = cfg["n"]
    off = np.cumsum([0] + cfg["widths"])
    top_off, a1 = int(off[TOP]), 1 << int(off[cfg["ids"]["A1"]])
    keep_mask = ((1 << n) - 1) << top_off
    v = np.zeros(1 << n, np.complex128)
    for k, a in state.items():
        if k & a1 and not (k & ~keep_mask & ~a1):
            v[(k >> top_off) & ((1 << n) - 1)] = a
    return v

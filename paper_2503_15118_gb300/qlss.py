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


def registers(n, inst_bits=0):
    """Widths and register ids for system size 2^n (and an instance register)."""
    widths = [n, n]
    ids = {"BOT": 0, "TOP": 1}
    if inst_bits:
        ids["INST"] = len(widths)
        widths.append(inst_bits)
    for name, w in (("C", 1), ("A2", 1), ("AH", 1), ("Q", ANGLE_BITS)):
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

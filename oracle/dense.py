"""Dense references used to pin the std::map oracle.  TEST INFRASTRUCTURE ONLY.

Both are written from the textbook definitions, independently of
``sqs_oracle.cpp``:

* :class:`DenseState` -- a full statevector of 2^n complex128 amplitudes
  (Schroedinger picture, Sec. II.B).  A single-qubit gate is applied pairwise:
  for every index x with bit t = 0 whose controls hold,
  (psi[x], psi[x|b]) <- U (psi[x], psi[x|b]).
* :func:`kron_unitary` -- the full 2^n x 2^n matrix of one gate built from
  Kronecker products, with |i> = |i_{n-1}> (x) ... (x) |i_0> (Eq. 4) and the
  controlled form CU = |0><0| (x) I + |1><1| (x) U (Sec. II.A), generalised to
  several controls as  I - P_C + P_C . U_t  with P_C the projector onto the
  required control values.  Permutations are built as 0/1 matrices from the
  map's definition.

Neither prunes: their results are compared to the oracle with a tolerance that
covers the amplitudes below the oracle's pruning threshold.
"""
from __future__ import annotations

import numpy as np

H_MAT = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)


def ry_mat(theta):
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def gate_matrix(g):
    """2x2 matrix of a single-qubit gate tuple."""
    if g[0] == "h":
        return H_MAT
    if g[0] == "ry":
        return ry_mat(g[3])
    if g[0] == "u1q":
        return np.asarray(g[3], dtype=np.complex128).reshape(2, 2)
    raise ValueError(g[0])


def _offsets(widths):
    off, o = [], 0
    for w in widths:
        off.append(o)
        o += w
    return off, o


class DenseState:
    """Full statevector over sum(widths) <= 22 qubits, index = packed key."""

    def __init__(self, widths):
        self.widths = list(widths)
        self.off, self.n = _offsets(self.widths)
        assert self.n <= 22, "dense reference limited to 22 qubits"
        self.psi = np.zeros(2 ** self.n, dtype=np.complex128)
        self.psi[0] = 1.0
        self.idx = np.arange(2 ** self.n, dtype=np.int64)

    def _field(self, reg):
        """Value of register reg, or of (first, count): the consecutive
        registers first .. first + count - 1 read as one number, the first
        one lowest."""
        if isinstance(reg, tuple):
            first, count = reg
            w = sum(self.widths[first:first + count])
            return (self.idx >> self.off[first]) & ((1 << w) - 1)
        return (self.idx >> self.off[reg]) & ((1 << self.widths[reg]) - 1)

    def marginal(self, reg):
        """p(v) = sum of |psi(x)|^2 over the x whose register reg holds v."""
        p = np.zeros(1 << self.widths[reg])
        np.add.at(p, self._field(reg), np.abs(self.psi) ** 2)
        return p

    def _ctrl_mask(self, ctrls):
        m = np.ones(self.idx.shape, dtype=bool)
        for c in ctrls or ():
            val = c[2] if len(c) > 2 else 1
            m &= ((self.idx >> (self.off[c[0]] + c[1])) & 1) == val
        return m

    def single(self, reg, bit, U, ctrls=()):
        q = self.off[reg] + bit
        b = 1 << q
        sel = self._ctrl_mask(ctrls) & (((self.idx >> q) & 1) == 0)
        x0 = self.idx[sel]
        x1 = x0 | b
        a0, a1 = self.psi[x0].copy(), self.psi[x1].copy()
        self.psi[x0] = U[0, 0] * a0 + U[0, 1] * a1
        self.psi[x1] = U[1, 0] * a0 + U[1, 1] * a1

    def permute(self, new_index):
        out = np.zeros_like(self.psi)
        out[new_index] = self.psi
        self.psi = out

    def apply(self, g, tables=()):
        op = g[0]
        if op in ("h", "ry", "u1q"):
            ctrls = g[4] if op != "h" else g[3]
            self.single(g[1], g[2], gate_matrix(g), ctrls)
        elif op == "ry_reg":
            _, reg, bit, areg, scale, offset, ctrls = g
            q = self.off[reg] + bit
            b = 1 << q
            sel = self._ctrl_mask(ctrls) & (((self.idx >> q) & 1) == 0)
            x0 = self.idx[sel]
            x1 = x0 | b
            theta = scale * self._field(areg)[sel].astype(np.float64) + offset
            c, s = np.cos(theta / 2), np.sin(theta / 2)
            a0, a1 = self.psi[x0].copy(), self.psi[x1].copy()
            self.psi[x0] = c * a0 - s * a1
            self.psi[x1] = s * a0 + c * a1
        elif op == "x":
            _, reg, bit, ctrls = g
            m = self._ctrl_mask(ctrls)
            self.permute(np.where(m, self.idx ^ (1 << (self.off[reg] + bit)), self.idx))
        elif op in ("add", "sub"):
            _, dst, src, const, ctrls = g
            w = self.widths[dst]
            d = self._field(dst)
            v = self._field(src) if src >= 0 else np.int64(const % (1 << w))
            r = (d + v) % (1 << w) if op == "add" else (d - v) % (1 << w)
            new = (self.idx & ~(((1 << w) - 1) << self.off[dst])) | (r << self.off[dst])
            self.permute(np.where(self._ctrl_mask(ctrls), new, self.idx))
        elif op == "swap":
            _, r1, r2, ctrls = g
            v1, v2 = self._field(r1), self._field(r2)
            clear = ~((((1 << self.widths[r1]) - 1) << self.off[r1])
                      | (((1 << self.widths[r2]) - 1) << self.off[r2]))
            new = (self.idx & clear) | (v2 << self.off[r1]) | (v1 << self.off[r2])
            self.permute(np.where(self._ctrl_mask(ctrls), new, self.idx))
        elif op in ("muladd", "mulc", "divxor"):
            # Arithmetic oracles (Sec. II.D.1), in Python integers per basis state.
            dst = g[1]
            w = self.widths[dst]
            d = self._field(dst)
            if op == "mulc":
                r = np.array([(int(x) * int(g[2])) % (1 << w) for x in d], np.int64)
                ctrls = g[3]
            else:
                a, bb = self._field(g[2]), self._field(g[3])
                if op == "muladd":
                    r = np.array([(int(x) + int(y) * int(z)) % (1 << w)
                                  for x, y, z in zip(d, a, bb)], np.int64)
                else:
                    r = np.array([(int(x) ^ (int(y) // int(z) if z else 0)) % (1 << w)
                                  for x, y, z in zip(d, a, bb)], np.int64)
                ctrls = g[4]
            new = (self.idx & ~(((1 << w) - 1) << self.off[dst])) | (r << self.off[dst])
            self.permute(np.where(self._ctrl_mask(ctrls), new, self.idx))
        elif op == "phase":
            _, preds, phi = g
            self.psi[self._ctrl_mask(preds)] *= np.exp(1j * phi)
        elif op in ("qload", "qunload"):
            _, areg, dreg, ti = g
            t = np.asarray(tables[ti]).astype(np.int64)
            a = self._field(areg)
            d = np.where(a < t.shape[0], t[np.minimum(a, t.shape[0] - 1)], 0)
            d &= (1 << self.widths[dreg]) - 1
            self.permute(self.idx ^ (d << self.off[dreg]))
        elif op == "prune":
            pass
        else:
            raise ValueError(op)


def run_dense(circ, upto=None):
    st = DenseState(circ["widths"])
    tables = circ.get("tables", ())
    for g in circ["gates"] if upto is None else circ["gates"][:upto]:
        st.apply(g, tables)
    return st


def kron_unitary(widths, g, tables=()):
    """Full 2^n x 2^n matrix of one gate (n = sum(widths) <= 10)."""
    off, n = _offsets(widths)
    assert n <= 10
    dim = 2 ** n
    I2 = np.eye(2, dtype=np.complex128)

    def one_qubit(q, A):
        # |i> = |i_{n-1}> (x) ... (x) |i_0>: qubit n-1 is the leftmost factor.
        return np.kron(np.kron(np.eye(2 ** (n - 1 - q)), A), np.eye(2 ** q))

    def projector(ctrls):
        P = np.eye(dim, dtype=np.complex128)
        for c in ctrls or ():
            val = c[2] if len(c) > 2 else 1
            Pv = np.diag([1.0, 0.0] if val == 0 else [0.0, 1.0]).astype(np.complex128)
            P = P @ one_qubit(off[c[0]] + c[1], Pv)
        return P

    op = g[0]
    if op in ("h", "ry", "u1q"):
        ctrls = g[3] if op == "h" else g[4]
        P = projector(ctrls)
        Ut = one_qubit(off[g[1]] + g[2], gate_matrix(g))
        return np.eye(dim) - P + P @ Ut
    if op == "phase":
        P = projector(g[1])
        return np.eye(dim) - P + np.exp(1j * g[2]) * P
    if op == "ry_reg":
        _, reg, bit, areg, scale, offset, ctrls = g
        M = np.zeros((dim, dim), dtype=np.complex128)
        q = off[reg] + bit
        for x in range(dim):
            ok = all(((x >> (off[c[0]] + c[1])) & 1) == (c[2] if len(c) > 2 else 1)
                     for c in ctrls or ())
            if not ok:
                M[x, x] = 1
                continue
            v = (x >> off[areg]) & ((1 << widths[areg]) - 1)
            R = ry_mat(scale * v + offset)
            xt = (x >> q) & 1
            for r in (0, 1):
                y = (x & ~(1 << q)) | (r << q)
                M[y, x] += R[r, xt]
        return M
    # Permutations: column x has a single 1 at row pi(x).
    M = np.zeros((dim, dim), dtype=np.complex128)
    for x in range(dim):
        M[_perm_image(widths, off, g, x, tables), x] = 1.0
    return M


def _perm_image(widths, off, g, x, tables):
    def field(r):
        return (x >> off[r]) & ((1 << widths[r]) - 1)

    def with_field(y, r, v):
        m = ((1 << widths[r]) - 1) << off[r]
        return (y & ~m) | ((v & ((1 << widths[r]) - 1)) << off[r])

    def ctrl_ok(ctrls):
        return all(((x >> (off[c[0]] + c[1])) & 1) == (c[2] if len(c) > 2 else 1)
                   for c in ctrls or ())

    op = g[0]
    if op == "x":
        return x ^ (1 << (off[g[1]] + g[2])) if ctrl_ok(g[3]) else x
    if op in ("add", "sub"):
        _, dst, src, const, ctrls = g
        if not ctrl_ok(ctrls):
            return x
        v = field(src) if src >= 0 else const
        return with_field(x, dst, field(dst) + v if op == "add" else field(dst) - v)
    if op == "swap":
        _, r1, r2, ctrls = g
        if not ctrl_ok(ctrls):
            return x
        return with_field(with_field(x, r1, field(r2)), r2, field(r1))
    if op == "muladd":
        _, dst, a, b, ctrls = g
        return with_field(x, dst, field(dst) + field(a) * field(b)) if ctrl_ok(ctrls) else x
    if op == "mulc":
        _, dst, c, ctrls = g
        return with_field(x, dst, field(dst) * c) if ctrl_ok(ctrls) else x
    if op == "divxor":
        _, dst, a, b, ctrls = g
        if not ctrl_ok(ctrls):
            return x
        q = field(a) // field(b) if field(b) else 0
        return with_field(x, dst, field(dst) ^ q)
    if op in ("qload", "qunload"):
        _, areg, dreg, ti = g
        t = tables[ti]
        a = field(areg)
        d = int(t[a]) if a < len(t) else 0
        return with_field(x, dreg, field(dreg) ^ d)
    raise ValueError(op)

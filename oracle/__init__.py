"""CPU oracle for the sparse register-level state simulator (arXiv 2503.15118).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the CUDA library and its
Python binding never import it.

Two independent references live here:

* ``sqs_oracle.cpp`` -- a std::map<key, complex<double>> simulator (FP64) that
  follows the paper's statement of each operation; wrapped by ``OracleState``.
* ``dense.py`` -- a dense statevector and a brute-force Kronecker-product
  unitary, written separately in numpy, used to pin the std::map simulator.

The library is compiled in-tree by :func:`build` with g++ (plain C++17).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sqs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


class _Ctrl(ctypes.Structure):
    _fields_ = [("reg", ctypes.c_uint32), ("bit", ctypes.c_uint32), ("value", ctypes.c_uint32)]


def build(extra_flags=(), out_path=None, force=False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    out = out_path or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC) \
            and not extra_flags:
        return out
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", *extra_flags, _SRC,
           "-o", out]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    P = ctypes.c_void_p
    u32, u64, i32, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
    CP = ctypes.POINTER(_Ctrl)
    sig = {
        "or_create": (P, [ctypes.POINTER(u32), u32]),
        "or_clone": (P, [P]),
        "or_destroy": (None, [P]),
        "or_set_eps": (None, [P, dbl]),
        "or_nnz": (u64, [P]),
        "or_peak": (u64, [P]),
        "or_apply_u1q": (None, [P, u32, u32, ctypes.POINTER(dbl), CP, u32]),
        "or_apply_h": (None, [P, u32, u32, CP, u32]),
        "or_apply_ry": (None, [P, u32, u32, dbl, CP, u32]),
        "or_apply_ry_reg": (None, [P, u32, u32, u32, dbl, dbl, CP, u32]),
        "or_apply_x": (None, [P, u32, u32, CP, u32]),
        "or_apply_add": (None, [P, u32, i32, u64, i32, CP, u32]),
        "or_apply_swap": (None, [P, u32, u32, CP, u32]),
        "or_apply_mul_add": (None, [P, u32, u32, u32, CP, u32]),
        "or_apply_mul_const": (None, [P, u32, u64, CP, u32]),
        "or_apply_div_xor": (None, [P, u32, u32, u32, CP, u32]),
        "or_apply_phase": (None, [P, CP, u32, dbl]),
        "or_qram": (None, [P, u32, u32, P, u64, u32]),
        "or_qram_span": (None, [P, u32, u32, u32, P, u64, u32]),
        "or_prune": (None, [P, dbl]),
        "or_export": (u64, [P, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(dbl), u64]),
        "or_import": (None, [P, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(dbl), u64]),
        "or_probabilities": (u64, [P, u32, ctypes.POINTER(u64), ctypes.POINTER(dbl), u64]),
        "or_norm2": (dbl, [P]),
        "or_amplitude": (None, [P, u64, u64, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(path=None):
    """Load (building if needed) the oracle library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ctrls(ctrls):
    ctrls = list(ctrls or ())
    arr = (_Ctrl * max(1, len(ctrls)))()
    for i, c in enumerate(ctrls):
        reg, bit = int(c[0]), int(c[1])
        val = int(c[2]) if len(c) > 2 else 1
        arr[i] = _Ctrl(reg, bit, val)
    return arr, len(ctrls)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class OracleState:
    """One std::map state; starts in |0...0> with amplitude 1."""

    def __init__(self, widths, eps=1e-14, lib=None, _handle=None):
        self.lib = lib or load()
        self.widths = [int(w) for w in widths]
        if _handle is not None:
            self.h = _handle
        else:
            w = (ctypes.c_uint32 * len(self.widths))(*self.widths)
            self.h = self.lib.or_create(w, len(self.widths))
        self.eps = eps
        self.lib.or_set_eps(self.h, float(eps))
        self._tables = {}

    def __del__(self):
        try:
            if self.h:
                self.lib.or_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def clone(self):
        o = OracleState(self.widths, self.eps, self.lib, _handle=self.lib.or_clone(self.h))
        return o

    # --- operations -------------------------------------------------------
    def u1q(self, reg, bit, m, ctrls=()):
        m = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(2, 2))
        flat = np.empty(8, dtype=np.float64)
        flat[0::2] = m.reshape(-1).real
        flat[1::2] = m.reshape(-1).imag
        c, n = _ctrls(ctrls)
        self.lib.or_apply_u1q(self.h, reg, bit, _ptr(flat, ctypes.c_double), c, n)

    def h_gate(self, reg, bit, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_h(self.h, reg, bit, c, n)

    def ry(self, reg, bit, theta, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_ry(self.h, reg, bit, float(theta), c, n)

    def ry_reg(self, reg, bit, angle_reg, scale, offset=0.0, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_ry_reg(self.h, reg, bit, angle_reg, float(scale), float(offset), c, n)

    def x(self, reg, bit, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_x(self.h, reg, bit, c, n)

    def add(self, dst, src_reg, const=0, subtract=False, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_add(self.h, dst, int(src_reg), int(const) & (2**64 - 1),
                              1 if subtract else 0, c, n)

    def swap(self, r1, r2, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_swap(self.h, r1, r2, c, n)

    def phase(self, preds, phi):
        c, n = _ctrls(preds)
        self.lib.or_apply_phase(self.h, c, n, float(phi))

    def mul_add(self, dst, src1, src2, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_mul_add(self.h, dst, src1, src2, c, n)

    def mul_const(self, dst, const, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_mul_const(self.h, dst, int(const) & (2 ** 64 - 1), c, n)

    def div_xor(self, dst, src1, src2, ctrls=()):
        c, n = _ctrls(ctrls)
        self.lib.or_apply_div_xor(self.h, dst, src1, src2, c, n)

    def qram(self, addr_reg, data_reg, table):
        """addr_reg: a register, or (first, count): the address is then the
        concatenation of consecutive registers, the first one lowest."""
        t = np.ascontiguousarray(table)
        if isinstance(addr_reg, tuple):
            self.lib.or_qram_span(self.h, addr_reg[0], addr_reg[1], data_reg,
                                  t.ctypes.data_as(ctypes.c_void_p), t.shape[0], t.dtype.itemsize)
        else:
            self.lib.or_qram(self.h, addr_reg, data_reg, t.ctypes.data_as(ctypes.c_void_p),
                             t.shape[0], t.dtype.itemsize)

    def prune(self, eps):
        self.lib.or_prune(self.h, float(eps))

    # --- readout ----------------------------------------------------------
    def nnz(self):
        return int(self.lib.or_nnz(self.h))

    def peak(self):
        return int(self.lib.or_peak(self.h))

    def export(self):
        """Returns (keys as python ints, amplitudes complex128), ascending keys."""
        n = self.nnz()
        lo = np.zeros(max(n, 1), np.uint64)
        hi = np.zeros(max(n, 1), np.uint64)
        am = np.zeros(2 * max(n, 1), np.float64)
        n = self.lib.or_export(self.h, _ptr(lo, ctypes.c_uint64), _ptr(hi, ctypes.c_uint64),
                               _ptr(am, ctypes.c_double), n)
        return lo[:n], hi[:n], am[: 2 * n].view(np.complex128)

    def to_dict(self):
        lo, hi, a = self.export()
        return {(int(h) << 64) | int(l): complex(v) for l, h, v in zip(lo, hi, a)}

    def import_(self, lo, hi, amps):
        lo = np.ascontiguousarray(lo, np.uint64)
        hi = np.ascontiguousarray(hi, np.uint64)
        am = np.ascontiguousarray(np.asarray(amps, np.complex128)).view(np.float64)
        self.lib.or_import(self.h, _ptr(lo, ctypes.c_uint64), _ptr(hi, ctypes.c_uint64),
                           _ptr(am, ctypes.c_double), lo.shape[0])

    def probabilities(self, reg):
        cap = max(self.nnz(), 1)
        v = np.zeros(cap, np.uint64)
        p = np.zeros(cap, np.float64)
        n = self.lib.or_probabilities(self.h, reg, _ptr(v, ctypes.c_uint64),
                                      _ptr(p, ctypes.c_double), cap)
        return v[:n], p[:n]

    def norm2(self):
        return float(self.lib.or_norm2(self.h))

    def amplitude(self, key):
        re, im = ctypes.c_double(), ctypes.c_double()
        self.lib.or_amplitude(self.h, key & (2**64 - 1), key >> 64, ctypes.byref(re),
                              ctypes.byref(im))
        return complex(re.value, im.value)

    # --- gate lists ---------------------------------------------------------
    def apply(self, g, tables=()):
        """Applies one gate tuple of the shared gate-list format."""
        op = g[0]
        if op == "h":
            self.h_gate(g[1], g[2], g[3])
        elif op == "ry":
            self.ry(g[1], g[2], g[3], g[4])
        elif op == "u1q":
            self.u1q(g[1], g[2], g[3], g[4])
        elif op == "ry_reg":
            self.ry_reg(g[1], g[2], g[3], g[4], g[5], g[6])
        elif op == "x":
            self.x(g[1], g[2], g[3])
        elif op == "add":
            self.add(g[1], g[2], g[3], False, g[4])
        elif op == "sub":
            self.add(g[1], g[2], g[3], True, g[4])
        elif op == "swap":
            self.swap(g[1], g[2], g[3])
        elif op == "phase":
            self.phase(g[1], g[2])
        elif op == "muladd":
            self.mul_add(g[1], g[2], g[3], g[4])
        elif op == "mulc":
            self.mul_const(g[1], g[2], g[3])
        elif op == "divxor":
            self.div_xor(g[1], g[2], g[3], g[4])
        elif op in ("qload", "qunload"):
            self.qram(g[1], g[2], tables[g[3]])
        elif op == "prune":
            self.prune(g[1])
        else:
            raise ValueError(f"unknown gate {op!r}")


def run_circuit(circ, lib=None, upto=None):
    """Runs a gate-list circuit (see paper_2503_15118_gb300.workloads) on the oracle."""
    st = OracleState(circ["widths"], circ.get("eps", 1e-14), lib=lib)
    gates = circ["gates"] if upto is None else circ["gates"][:upto]
    tables = circ.get("tables", ())
    for g in gates:
        st.apply(g, tables)
    return st

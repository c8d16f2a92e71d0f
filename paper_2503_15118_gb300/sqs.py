"""ctypes binding of the C ABI in include/sqs.h (argument marshalling only).

Every operation runs in the CUDA library ``_build/libsqs.so``; this module
only converts Python arguments and maps status codes to exceptions.  PyTorch
supplies device memory (its caching allocator, through the ABI's allocator
callbacks) and the CUDA stream.  If the library is missing and cannot be
built, importing the binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
AMP_FP64, AMP_FP32 = 0, 1
SIZING_EXACT, SIZING_LEARNED = 0, 2
MERGE_AUTO, MERGE_HASH, MERGE_SORT, MERGE_CLUSTER, MERGE_TUNED, MERGE_PLAIN = 0, 4, 8, 16, 32, 64
FUSE_OFF, FUSE_ALWAYS = 128, 256
AUTOTUNE = 512
(PERM_X, PERM_ADD_REG, PERM_SUB_REG, PERM_ADD_CONST, PERM_SUB_CONST, PERM_SWAP, PERM_MUL_ADD,
 PERM_MUL_CONST, PERM_DIV_XOR) = range(9)
MAX_CTRL = 8     # controls inline in one permutation operation
MAX_PRED = 128   # controls / predicates passed as an array


class SqsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sqs status {status}: {msg}")
        self.status = status


class Ctrl(ctypes.Structure):
    _fields_ = [("reg", ctypes.c_uint32), ("bit", ctypes.c_uint32), ("value", ctypes.c_uint32)]


class PermOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("reg", ctypes.c_uint32), ("bit", ctypes.c_uint32),
                ("src_reg", ctypes.c_uint32), ("constant", ctypes.c_uint64),
                ("n_ctrl", ctypes.c_uint32), ("ctrl", Ctrl * MAX_CTRL),
                ("src2_reg", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("host_waits", ctypes.c_uint64), ("overflow_reruns", ctypes.c_uint64),
                ("learned_steps", ctypes.c_uint64), ("bytes_live", ctypes.c_uint64),
                ("bytes_peak", ctypes.c_uint64), ("steps_expand", ctypes.c_uint64),
                ("steps_hash", ctypes.c_uint64), ("steps_sort", ctypes.c_uint64),
                ("steps_cluster", ctypes.c_uint64), ("steps_fold", ctypes.c_uint64),
                ("runs_fused", ctypes.c_uint64), ("steps_fused", ctypes.c_uint64),
                ("ops_deferred", ctypes.c_uint64)]


PRED_FEATURES, PRED_HIDDEN, PRED_PARAMS = 16, 32, 1633


class TraceRecord(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_uint32), ("call", ctypes.c_uint32), ("ms", ctypes.c_float),
                ("pad", ctypes.c_uint32)]


KERNEL_NAMES = {0: "k_init", 1: "k_apply_inplace", 2: "k_apply_compact", 3: "k_partition",
                4: "k_pair", 5: "k_probabilities", 6: "k_convert", 7: "k_expand", 8: "k_bin",
                9: "k_pair_cluster", 10: "k_rsort_pass", 11: "k_rsort_merge", 12: "k_fold",
                13: "k_group_count", 14: "k_group"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN)]


# Names and signatures of every entry point declared in include/sqs.h.
_P = ctypes.c_void_p
_u32, _u64, _dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
_S = ctypes.c_int
_CP = ctypes.POINTER(Ctrl)
_DP = ctypes.POINTER(ctypes.c_double)
_UP = ctypes.POINTER(ctypes.c_uint64)
_FP = ctypes.POINTER(ctypes.c_float)
SIGNATURES = {
    "sqs_state_create": (_S, [ctypes.POINTER(_u32), _u32, _u32, _u64,
                              ctypes.POINTER(Allocator), _P, ctypes.POINTER(_P)]),
    "sqs_state_destroy": (None, [_P]),
    "sqs_state_reset": (_S, [_P]),
    "sqs_set_prune_eps": (_S, [_P, _dbl]),
    "sqs_apply_u1q": (_S, [_P, _u32, _u32, _DP, _CP, _u32]),
    "sqs_apply_h": (_S, [_P, _u32, _u32, _CP, _u32]),
    "sqs_apply_ry": (_S, [_P, _u32, _u32, _dbl, _CP, _u32]),
    "sqs_apply_ry_reg": (_S, [_P, _u32, _u32, _u32, _dbl, _dbl, _CP, _u32]),
    "sqs_apply_perm": (_S, [_P, ctypes.POINTER(PermOp), _u32]),
    "sqs_apply_phase": (_S, [_P, _CP, _u32, _dbl]),
    "sqs_table_create": (_S, [_P, _P, _u64, _u32, ctypes.POINTER(_P)]),
    "sqs_qram_load": (_S, [_P, _u32, _u32, _P]),
    "sqs_qram_unload": (_S, [_P, _u32, _u32, _P]),
    "sqs_qram_load_span": (_S, [_P, _u32, _u32, _u32, _P]),
    "sqs_capture_begin": (_S, [_P, _u64]),
    "sqs_capture_end": (_S, [_P, ctypes.POINTER(ctypes.c_void_p)]),
    "sqs_graph_launch": (_S, [_P, _P]),
    "sqs_graph_destroy": (None, [_P]),
    "sqs_qram_unload_span": (_S, [_P, _u32, _u32, _u32, _P]),
    "sqs_prune": (_S, [_P, _dbl, _UP]),
    "sqs_probabilities": (_S, [_P, _u32, _DP, _DP]),
    "sqs_probabilities_device": (_S, [_P, _u32, _P, _P]),
    "sqs_probabilities_sparse": (_S, [_P, _u32, _UP, _DP, _u64, _UP, _DP]),
    "sqs_state_set_wait_test": (_S, [_P, _u32, ctypes.c_int32]),
    "sqs_set_fp32_cancel": (_S, [_P, ctypes.c_double]),
    "sqs_tune_export": (_S, [_P, ctypes.c_char_p, _u64, _UP]),
    "sqs_tune_import": (_S, [_P, ctypes.c_char_p]),
    "sqs_nnz": (_S, [_P, _UP]),
    "sqs_peak_nnz": (_S, [_P, _UP]),
    "sqs_export": (_S, [_P, _UP, _DP, _u64, _UP]),
    "sqs_import": (_S, [_P, _UP, _DP, _u64]),
    "sqs_sync": (_S, [_P]),
    "sqs_flush": (_S, [_P]),
    "sqs_key_words": (_u32, [_P]),
    "sqs_launch_count": (_u64, [_P]),
    "sqs_trace_enable": (_S, [_P, _u32]),
    "sqs_trace_read": (_S, [_P, ctypes.POINTER(TraceRecord), _u32, ctypes.POINTER(_u32)]),
    "sqs_last_error": (ctypes.c_char_p, [_P]),
    "sqs_version": (ctypes.c_char_p, []),
    "sqs_apply_u1q_noalloc": (_S, [ctypes.POINTER(_u32), _u32, _u32, _u32, _DP, _CP, _u32, _dbl,
                                   _P, _P, _P, _u64, _P, _P, _P, _u64, _P, _P]),
    "sqs_noalloc_last_error": (ctypes.c_char_p, []),
    "sqs_noalloc_scratch_bytes": (_u64, []),
    "sqs_predictor_create": (_S, [_u64, _P, ctypes.POINTER(_P)]),
    "sqs_predictor_destroy": (None, [_P]),
    "sqs_predictor_get_params": (_S, [_P, _FP]),
    "sqs_predictor_set_params": (_S, [_P, _FP]),
    "sqs_predictor_predict": (_S, [_P, _FP, _u32, _FP]),
    "sqs_predictor_gradient": (_S, [_P, _FP, _FP, _u32, _FP, _FP]),
    "sqs_predictor_train": (_S, [_P, _FP, _FP, _u32, _u32, _u32, ctypes.c_float, _FP]),
    "sqs_state_set_predictor": (_S, [_P, _P]),
    "sqs_state_record": (_S, [_P, _u32]),
    "sqs_state_read_records": (_S, [_P, _FP, _FP, _u32, ctypes.POINTER(_u32)]),
    "sqs_state_stats": (_S, [_P, ctypes.POINTER(Stats)]),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Loads libsqs.so (building it with nvcc when absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; run paper_2503_15118_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ctrls(ctrls):
    ctrls = list(ctrls or ())
    if len(ctrls) > MAX_PRED:
        raise ValueError("too many controls")
    arr = (Ctrl * max(1, len(ctrls)))()
    for i, c in enumerate(ctrls):
        arr[i] = Ctrl(int(c[0]), int(c[1]), int(c[2]) if len(c) > 2 else 1)
    return arr, len(ctrls)


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch
        self._alloc = ALLOC_FN(self.alloc)
        self._free = FREE_FN(self.free)
        self.struct = Allocator(None, self._alloc, self._free)

    def alloc(self, ctx, nbytes, stream):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def free(self, ctx, ptr, stream):
        try:
            self.torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass


class State:
    """One sparse state on the current CUDA device (see sqs_state_create)."""

    def __init__(self, widths, amp32=False, learned=False, merge=MERGE_AUTO, capacity_hint=0,
                 stream=None, torch_allocator=True, eps=None):
        self.lib = load()
        self.widths = [int(w) for w in widths]
        flags = (AMP_FP32 if amp32 else 0) | (SIZING_LEARNED if learned else 0) | merge
        self._alloc = None
        alloc_ptr = None
        if stream is None or torch_allocator:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        if torch_allocator:
            self._alloc = _TorchAllocator()
            alloc_ptr = ctypes.byref(self._alloc.struct)
        self.stream = int(stream or 0)
        h = ctypes.c_void_p()
        w = (ctypes.c_uint32 * len(self.widths))(*self.widths)
        st = self.lib.sqs_state_create(w, len(self.widths), flags, int(capacity_hint), alloc_ptr,
                                       ctypes.c_void_p(self.stream), ctypes.byref(h))
        if st != OK:
            raise SqsError(st, "sqs_state_create failed")
        self.h = h
        self.kw = int(self.lib.sqs_key_words(self.h))
        self._tables = {}
        if eps is not None:
            self.set_prune_eps(eps)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sqs_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, status):
        if status != OK:
            raise SqsError(status, self.lib.sqs_last_error(self.h).decode())

    # --- operations -------------------------------------------------------
    def reset(self):
        self._chk(self.lib.sqs_state_reset(self.h))

    def tune_export(self):
        """The autotuner's choices (SQS_AUTOTUNE) as a parsed JSON object."""
        import json
        n = ctypes.c_uint64()
        self.lib.sqs_tune_export(self.h, None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(int(n.value) + 1)
        self._chk(self.lib.sqs_tune_export(self.h, buf, int(n.value) + 1, ctypes.byref(n)))
        return json.loads(buf.value.decode())

    def tune_import(self, obj):
        import json
        text = obj if isinstance(obj, str) else json.dumps(obj)
        self._chk(self.lib.sqs_tune_import(self.h, text.encode()))

    def set_fp32_cancel(self, rho):
        self._chk(self.lib.sqs_set_fp32_cancel(self.h, float(rho)))

    def set_prune_eps(self, eps):
        self._chk(self.lib.sqs_set_prune_eps(self.h, float(eps)))

    def h_gate(self, reg, bit, ctrls=()):
        c, n = _ctrls(ctrls)
        self._chk(self.lib.sqs_apply_h(self.h, reg, bit, c, n))

    def ry(self, reg, bit, theta, ctrls=()):
        c, n = _ctrls(ctrls)
        self._chk(self.lib.sqs_apply_ry(self.h, reg, bit, float(theta), c, n))

    def ry_reg(self, reg, bit, angle_reg, scale, offset=0.0, ctrls=()):
        c, n = _ctrls(ctrls)
        self._chk(self.lib.sqs_apply_ry_reg(self.h, reg, bit, angle_reg, float(scale),
                                            float(offset), c, n))

    def u1q(self, reg, bit, m, ctrls=()):
        m = np.asarray(m, dtype=np.complex128).reshape(2, 2)
        flat = np.empty(8, np.float64)
        flat[0::2] = m.reshape(-1).real
        flat[1::2] = m.reshape(-1).imag
        c, n = _ctrls(ctrls)
        self._chk(self.lib.sqs_apply_u1q(self.h, reg, bit,
                                         flat.ctypes.data_as(_DP), c, n))

    def perm(self, ops):
        """ops: (kind, reg, bit, src_reg, constant, ctrls[, src2_reg]) tuples."""
        arr = (PermOp * max(1, len(ops)))()
        for i, op in enumerate(ops):
            kind, reg, bit, src, const, ctrls = op[:6]
            arr[i].kind, arr[i].reg, arr[i].bit = kind, reg, bit
            arr[i].src_reg, arr[i].constant = src, int(const) & (2 ** 64 - 1)
            arr[i].src2_reg = op[6] if len(op) > 6 else 0
            arr[i].n_ctrl = len(ctrls)
            for j, c in enumerate(ctrls):
                arr[i].ctrl[j] = Ctrl(int(c[0]), int(c[1]), int(c[2]) if len(c) > 2 else 1)
        self._chk(self.lib.sqs_apply_perm(self.h, arr, len(ops)))

    def x(self, reg, bit, ctrls=()):
        self.perm([(PERM_X, reg, bit, 0, 0, tuple(ctrls or ()))])

    def phase(self, preds, phi):
        c, n = _ctrls(preds)
        self._chk(self.lib.sqs_apply_phase(self.h, c, n, float(phi)))

    def table(self, entries):
        key = id(entries)
        if key in self._tables:
            return self._tables[key][0]
        t = np.ascontiguousarray(entries)
        if t.dtype.kind not in "ui" or t.dtype.itemsize not in (1, 2, 4, 8):
            raise ValueError("QRAM tables hold 1, 2, 4 or 8-byte unsigned integers")
        out = ctypes.c_void_p()
        self._chk(self.lib.sqs_table_create(self.h, t.ctypes.data_as(ctypes.c_void_p),
                                            t.shape[0], t.dtype.itemsize, ctypes.byref(out)))
        self._tables[key] = (out, entries)
        return out

    def qram_load(self, addr_reg, data_reg, entries):
        """addr_reg: a register, or (first, count) for an address spanning
        consecutive registers."""
        if isinstance(addr_reg, tuple):
            self._chk(self.lib.sqs_qram_load_span(self.h, addr_reg[0], addr_reg[1], data_reg,
                                                  self.table(entries)))
        else:
            self._chk(self.lib.sqs_qram_load(self.h, addr_reg, data_reg, self.table(entries)))

    def qram_unload(self, addr_reg, data_reg, entries):
        if isinstance(addr_reg, tuple):
            self._chk(self.lib.sqs_qram_unload_span(self.h, addr_reg[0], addr_reg[1], data_reg,
                                                    self.table(entries)))
        else:
            self._chk(self.lib.sqs_qram_unload(self.h, addr_reg, data_reg, self.table(entries)))

    def prune(self, eps, wait=False):
        n = ctypes.c_uint64()
        self._chk(self.lib.sqs_prune(self.h, float(eps), ctypes.byref(n) if wait else None))
        return int(n.value) if wait else None

    # --- readout ----------------------------------------------------------
    def nnz(self):
        n = ctypes.c_uint64()
        self._chk(self.lib.sqs_nnz(self.h, ctypes.byref(n)))
        return int(n.value)

    def peak_nnz(self):
        n = ctypes.c_uint64()
        self._chk(self.lib.sqs_peak_nnz(self.h, ctypes.byref(n)))
        return int(n.value)

    def sync(self):
        self._chk(self.lib.sqs_sync(self.h))

    def flush(self):
        self._chk(self.lib.sqs_flush(self.h))

    def launch_count(self):
        return int(self.lib.sqs_launch_count(self.h))

    def set_predictor(self, pred):
        self._pred = pred
        self._chk(self.lib.sqs_state_set_predictor(self.h, pred.h if pred is not None else None))

    def record(self, enable=True):
        self._chk(self.lib.sqs_state_record(self.h, 1 if enable else 0))

    def read_records(self, cap=1 << 16):
        X = np.zeros((cap, PRED_FEATURES), np.float32)
        y = np.zeros(cap, np.float32)
        n = ctypes.c_uint32()
        self._chk(self.lib.sqs_state_read_records(self.h, X.ctypes.data_as(_FP),
                                                  y.ctypes.data_as(_FP), cap, ctypes.byref(n)))
        k = min(int(n.value), cap)
        return X[:k], y[:k]

    def stats(self):
        s = Stats()
        self._chk(self.lib.sqs_state_stats(self.h, ctypes.byref(s)))
        return {f: int(getattr(s, f)) for f, _ in Stats._fields_}

    def trace_enable(self, max_records):
        self._chk(self.lib.sqs_trace_enable(self.h, int(max_records)))

    def trace_read(self, cap=1 << 16):
        """List of (kernel name, api call index, device ms) since the last read."""
        buf = (TraceRecord * max(1, cap))()
        n = ctypes.c_uint32()
        self._chk(self.lib.sqs_trace_read(self.h, buf, cap, ctypes.byref(n)))
        return [(KERNEL_NAMES.get(buf[i].kernel, str(buf[i].kernel)), int(buf[i].call),
                 float(buf[i].ms)) for i in range(min(int(n.value), cap))], int(n.value)

    def probabilities(self, reg, with_probs=True):
        w = self.widths[reg]
        probs = np.zeros(2 ** w if with_probs else 1, np.float64)
        n2 = ctypes.c_double()
        self._chk(self.lib.sqs_probabilities(self.h, reg,
                                             probs.ctypes.data_as(_DP) if with_probs else None,
                                             ctypes.byref(n2)))
        return (probs if with_probs else None), float(n2.value)

    def probabilities_device(self, reg, probs_ptr, norm_ptr):
        self._chk(self.lib.sqs_probabilities_device(self.h, reg, ctypes.c_void_p(probs_ptr),
                                                    ctypes.c_void_p(norm_ptr)))

    def probabilities_sparse(self, reg):
        """(values, probs, norm2): the distinct values of register ``reg``
        ascending and the summed |a|^2 of each (sqs_probabilities_sparse)."""
        cnt = ctypes.c_uint64()
        n2 = ctypes.c_double()
        st = self.lib.sqs_probabilities_sparse(self.h, reg, None, None, 0, ctypes.byref(cnt),
                                               ctypes.byref(n2))
        if st not in (OK, ERR_ARG):
            self._chk(st)
        c = int(cnt.value)
        vals = np.zeros(max(c, 1), np.uint64)
        probs = np.zeros(max(c, 1), np.float64)
        self._chk(self.lib.sqs_probabilities_sparse(self.h, reg, vals.ctypes.data_as(_UP),
                                                    probs.ctypes.data_as(_DP), c,
                                                    ctypes.byref(cnt), ctypes.byref(n2)))
        c = int(cnt.value)
        return vals[:c], probs[:c], float(n2.value)

    def export(self):
        """(lo, hi, amps): key words and complex128 amplitudes, ascending keys."""
        n = ctypes.c_uint64()
        st = self.lib.sqs_export(self.h, None, None, 0, ctypes.byref(n))
        if st not in (OK, ERR_ARG):
            self._chk(st)
        cnt = int(n.value)
        keys = np.zeros(max(cnt, 1) * self.kw, np.uint64)
        amps = np.zeros(2 * max(cnt, 1), np.float64)
        self._chk(self.lib.sqs_export(self.h, keys.ctypes.data_as(_UP), amps.ctypes.data_as(_DP),
                                      cnt, ctypes.byref(n)))
        cnt = int(n.value)
        keys = keys[: cnt * self.kw].reshape(cnt, self.kw)
        lo = keys[:, 0].copy()
        hi = keys[:, 1].copy() if self.kw == 2 else np.zeros(cnt, np.uint64)
        return lo, hi, amps[: 2 * cnt].view(np.complex128)

    def to_dict(self):
        lo, hi, a = self.export()
        return {(int(h) << 64) | int(l): complex(v) for l, h, v in zip(lo, hi, a)}

    def import_(self, lo, hi, amps):
        lo = np.asarray(lo, np.uint64)
        n = lo.shape[0]
        keys = np.empty((n, self.kw), np.uint64)
        keys[:, 0] = lo
        if self.kw == 2:
            keys[:, 1] = np.asarray(hi, np.uint64)
        keys = np.ascontiguousarray(keys.reshape(-1))
        am = np.ascontiguousarray(np.asarray(amps, np.complex128)).view(np.float64)
        self._chk(self.lib.sqs_import(self.h, keys.ctypes.data_as(_UP), am.ctypes.data_as(_DP),
                                      n))

    # --- gate lists ---------------------------------------------------------
    def apply(self, g, tables=()):
        """Applies one gate tuple of the gate-list format (workloads.py)."""
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
            self.perm([(PERM_X, g[1], g[2], 0, 0, tuple(g[3]))])
        elif op in ("add", "sub"):
            if g[2] >= 0:
                kind = PERM_ADD_REG if op == "add" else PERM_SUB_REG
                self.perm([(kind, g[1], 0, g[2], 0, tuple(g[4]))])
            else:
                kind = PERM_ADD_CONST if op == "add" else PERM_SUB_CONST
                self.perm([(kind, g[1], 0, 0, g[3], tuple(g[4]))])
        elif op == "swap":
            self.perm([(PERM_SWAP, g[1], 0, g[2], 0, tuple(g[3]))])
        elif op == "phase":
            self.phase(g[1], g[2])
        elif op == "muladd":
            self.perm([(PERM_MUL_ADD, g[1], 0, g[2], 0, tuple(g[4]), g[3])])
        elif op == "mulc":
            self.perm([(PERM_MUL_CONST, g[1], 0, 0, g[2], tuple(g[3]))])
        elif op == "divxor":
            self.perm([(PERM_DIV_XOR, g[1], 0, g[2], 0, tuple(g[4]), g[3])])
        elif op == "qload":
            self.qram_load(g[1], g[2], tables[g[3]])
        elif op == "qunload":
            self.qram_unload(g[1], g[2], tables[g[3]])
        elif op == "prune":
            self.prune(g[1])
        else:
            raise ValueError(f"unknown gate {op!r}")

    # --- CUDA-graph capture (include/sqs.h) -----------------------------------
    def capture_begin(self, static_bound):
        self._chk(self.lib.sqs_capture_begin(self.h, int(static_bound)))

    def capture_end(self):
        g = ctypes.c_void_p()
        self._chk(self.lib.sqs_capture_end(self.h, ctypes.byref(g)))
        return Graph(self, g)

    def capture(self, circ, static_bound):
        """Captures |0...0> followed by the circuit's gates as one graph."""
        self.capture_begin(static_bound)
        try:
            self.run(circ)
        except SqsError:
            try:
                self.capture_end()
            except SqsError:
                pass
            raise
        return self.capture_end()

    def run(self, circ, upto=None):
        tables = circ.get("tables", ())
        for g in circ["gates"] if upto is None else circ["gates"][:upto]:
            self.apply(g, tables)
        return self


class Graph:
    """A captured circuit (sqs_capture_begin / _end); launch() replays it."""

    def __init__(self, state, handle):
        self.state, self.h = state, handle

    def launch(self):
        self.state._chk(self.state.lib.sqs_graph_launch(self.state.h, self.h))

    def close(self):
        if getattr(self, "h", None):
            self.state.lib.sqs_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Predictor:
    """The learned capacity predictor (include/sqs.h, sqs_predictor_*)."""

    def __init__(self, seed=0, stream=None):
        self.lib = load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        st = self.lib.sqs_predictor_create(int(seed), ctypes.c_void_p(int(stream or 0)),
                                           ctypes.byref(h))
        if st != OK:
            raise SqsError(st, "sqs_predictor_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.sqs_predictor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        w = np.zeros(PRED_PARAMS, np.float32)
        self._chk(self.lib.sqs_predictor_get_params(self.h, w.ctypes.data_as(_FP)))
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, np.float32)
        assert w.shape == (PRED_PARAMS,)
        self._chk(self.lib.sqs_predictor_set_params(self.h, w.ctypes.data_as(_FP)))

    def predict(self, X):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, PRED_FEATURES)
        Y = np.zeros(X.shape[0], np.float32)
        self._chk(self.lib.sqs_predictor_predict(self.h, X.ctypes.data_as(_FP), X.shape[0],
                                                 Y.ctypes.data_as(_FP)))
        return Y

    def gradient(self, X, T):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, PRED_FEATURES)
        T = np.ascontiguousarray(T, np.float32)
        g = np.zeros(PRED_PARAMS, np.float32)
        loss = ctypes.c_float()
        self._chk(self.lib.sqs_predictor_gradient(self.h, X.ctypes.data_as(_FP),
                                                  T.ctypes.data_as(_FP), X.shape[0],
                                                  g.ctypes.data_as(_FP), ctypes.byref(loss)))
        return g, float(loss.value)

    def train(self, X, T, epochs=200, batch=256, lr=3e-3):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, PRED_FEATURES)
        T = np.ascontiguousarray(T, np.float32)
        loss = ctypes.c_float()
        self._chk(self.lib.sqs_predictor_train(self.h, X.ctypes.data_as(_FP),
                                               T.ctypes.data_as(_FP), X.shape[0], epochs, batch,
                                               float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def _chk(self, status):
        if status != OK:
            raise SqsError(status, "predictor call failed")


def run_circuit(circ, amp32=False, learned=False, merge=MERGE_AUTO, capacity_hint=0, upto=None,
                predictor=None):
    st = State(circ["widths"], amp32=amp32, learned=learned, merge=merge,
               capacity_hint=capacity_hint, eps=circ.get("eps", 1e-14))
    if predictor is not None:
        st.set_predictor(predictor)
    return st.run(circ, upto=upto)


def version():
    return load().sqs_version().decode()

"""sqs_apply_u1q_noalloc, the entry point that allocates no device memory.

It is for callers that cannot allocate: a host framework that owns all device
memory through its own arena, or a latency-bound caller that cannot afford the
synchronisation cudaMalloc may bring.  The test calls it through the C ABI on
device buffers the caller owns (torch tensors) and compares its output with
the state-based sqs_apply_u1q / sqs_apply_h on the same input, twice in a row
(the second call reuses the static scratch the first one left behind).  This
file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_15118_gb300 import workloads as W
from tests.helpers import compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_15118_gb300 import sqs
    return torch, sqs, sqs.load()


def _noalloc(torch, sqs, lib, widths, lo, hi, amps, reg, bit, m, ctrls=(), eps=1e-14):
    dev = torch.device("cuda")
    n = lo.shape[0]
    k_lo = torch.from_numpy(lo.astype(np.uint64).view(np.int64)).to(dev)
    k_hi = torch.from_numpy(hi.astype(np.uint64).view(np.int64)).to(dev)
    a = torch.from_numpy(np.ascontiguousarray(amps, np.complex128).view(np.float64)).to(dev)
    cap = 2 * n
    o_lo = torch.empty(cap, dtype=torch.int64, device=dev)
    o_hi = torch.empty(cap, dtype=torch.int64, device=dev)
    o_a = torch.empty(2 * cap, dtype=torch.float64, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    w = (ctypes.c_uint32 * len(widths))(*widths)
    mm = np.asarray(m, np.complex128).reshape(2, 2)
    flat = np.empty(8, np.float64)
    flat[0::2], flat[1::2] = mm.reshape(-1).real, mm.reshape(-1).imag
    c, nc = sqs._ctrls(ctrls)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.sqs_apply_u1q_noalloc(
        w, len(widths), reg, bit, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), c, nc,
        eps, ctypes.c_void_p(k_lo.data_ptr()), ctypes.c_void_p(k_hi.data_ptr()),
        ctypes.c_void_p(a.data_ptr()), n, ctypes.c_void_p(o_lo.data_ptr()),
        ctypes.c_void_p(o_hi.data_ptr()), ctypes.c_void_p(o_a.data_ptr()), cap,
        ctypes.c_void_p(n_out.data_ptr()), ctypes.c_void_p(stream))
    assert st == 0, lib.sqs_noalloc_last_error().decode()
    torch.cuda.synchronize()
    cnt = int(n_out.item())
    assert 0 <= cnt <= cap
    lo_o = o_lo[:cnt].cpu().numpy().view(np.uint64)
    hi_o = o_hi[:cnt].cpu().numpy().view(np.uint64) if sum(widths) > 64 else np.zeros(cnt, np.uint64)
    a_o = o_a[: 2 * cnt].cpu().numpy().view(np.complex128)
    return {(int(h) << 64) | int(l): complex(v) for l, h, v in zip(lo_o, hi_o, a_o)}


def _reference(sqs, widths, lo, hi, amps, reg, bit, m, ctrls=()):
    st = sqs.State(widths, eps=1e-14)
    st.import_(lo, hi, amps)
    st.u1q(reg, bit, m, ctrls)
    out = st.to_dict()
    st.close()
    return out


H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
U = np.array([[0.6, -0.8j], [0.8, 0.6j]])


@pytest.mark.parametrize("widths,target,m,ctrls", [
    ([16, 16, 16, 16], (2, 5), H, ()),
    ([20, 32, 32], (1, 31), U, ((0, 3, 1),)),
])
def test_noalloc_matches_state_entry_point_twice(env, widths, target, m, ctrls):
    torch, sqs, lib = env
    assert lib.sqs_noalloc_scratch_bytes() < 16 << 20
    for call, n in enumerate([5000, 40000]):  # two calls in a row on the shared scratch
        lo, hi, amps = W.random_state(widths, n, seed=900 + call + n, pair_fraction=0.5,
                                      target=target)
        got = _noalloc(torch, sqs, lib, widths, lo, hi, amps, target[0], target[1], m, ctrls)
        ref = _reference(sqs, widths, lo, hi, amps, target[0], target[1], m, ctrls)
        assert compare_states(got, ref, atol=1e-12) > 1 - 1e-10
        assert set(got) == set(ref)


def test_noalloc_rejects_oversized_input(env):
    torch, sqs, lib = env
    w = (ctypes.c_uint32 * 1)(16)
    flat = (ctypes.c_double * 8)(*([0.0] * 8))
    n = lib.sqs_apply_u1q_noalloc(w, 1, 0, 0, flat, None, 0, 1e-14, ctypes.c_void_p(1),
                                  None, ctypes.c_void_p(1), (1 << 16) + 1, ctypes.c_void_p(1),
                                  None, ctypes.c_void_p(1), 1 << 20, ctypes.c_void_p(1), None)
    assert n == sqs.ERR_ARG
    assert "MAX_BRANCHES" in lib.sqs_noalloc_last_error().decode()


def test_noalloc_overflow_writes_nothing_past_out_cap(env):
    """A bucket overflow (here forced by repeated keys, which break the
    distinct-keys contract) must report an all-ones count and leave the
    caller's output untouched, even though the previous call left large
    output-segment counts in the shared scratch."""
    torch, sqs, lib = env
    dev = torch.device("cuda")
    widths = [16, 16, 16, 16]
    # First call: 65536 unpaired branches, so every output segment is full.
    lo, hi, amps = W.random_state(widths, 65536, seed=4242, pair_fraction=0.0, target=(2, 5))
    _noalloc(torch, sqs, lib, widths, lo, hi, amps, 2, 5, H)
    # Second call: 3073 copies of one key land in one bucket of 2048 slots.
    n = 2 * 1536 + 1
    cap = 2 * n
    guard = 1 << 16
    k_in = torch.full((n,), 12345, dtype=torch.int64, device=dev)
    a_in = torch.full((2 * n,), 0.01, dtype=torch.float64, device=dev)
    o_lo = torch.full((cap + guard,), -7, dtype=torch.int64, device=dev)
    o_a = torch.full((2 * (cap + guard),), -7.0, dtype=torch.float64, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    w = (ctypes.c_uint32 * 4)(*widths)
    flat = np.empty(8, np.float64)
    flat[0::2], flat[1::2] = H.reshape(-1).real, H.reshape(-1).imag
    st = lib.sqs_apply_u1q_noalloc(
        w, 4, 2, 5, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0, 1e-14,
        ctypes.c_void_p(k_in.data_ptr()), None, ctypes.c_void_p(a_in.data_ptr()), n,
        ctypes.c_void_p(o_lo.data_ptr()), None, ctypes.c_void_p(o_a.data_ptr()), cap,
        ctypes.c_void_p(n_out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.sqs_noalloc_last_error().decode()
    torch.cuda.synchronize()
    assert int(n_out.item()) == -1  # all ones: the device-side check failed
    assert bool((o_lo == -7).all()), "output keys written after an overflow"
    assert bool((o_a == -7.0).all()), "output amplitudes written after an overflow"
    # The scratch is usable again: a valid call right after gives the right result.
    lo, hi, amps = W.random_state(widths, 3000, seed=4243, pair_fraction=0.5, target=(2, 5))
    got = _noalloc(torch, sqs, lib, widths, lo, hi, amps, 2, 5, H)
    ref = _reference(sqs, widths, lo, hi, amps, 2, 5, H)
    assert set(got) == set(ref)
    assert compare_states(got, ref, atol=1e-12) > 1 - 1e-10

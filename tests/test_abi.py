"""CPU checks of the C ABI: the library builds, loads and exports every entry
point that include/sqs.h declares, and the binding knows each of them.  No
call here touches a GPU."""
import ctypes
import os
import re

from paper_2503_15118_gb300 import build, sqs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sqs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sqs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["sqs_state_create", "sqs_apply_h", "sqs_apply_ry", "sqs_apply_u1q",
                 "sqs_apply_perm", "sqs_apply_phase", "sqs_qram_load", "sqs_qram_unload",
                 "sqs_probabilities", "sqs_prune", "sqs_export", "sqs_nnz"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert sorted(sqs.SIGNATURES) == _declared()


def test_version_string():
    assert "sm_103a" in sqs.version()


def test_only_the_c_abi_is_exported():
    out = os.popen(f"nm -D --defined-only {build.build()}").read().split("\n")
    text = [l.split()[-1] for l in out if " T " in l]
    assert text and all(n.startswith("sqs_") for n in text)

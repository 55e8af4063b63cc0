"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every symbol
include/cleora.h declares (no compute call: there is no GPU here)."""
import os
import re

import paper_2102_02302_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cleora_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    names = _declared("cleora.h")
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    names = _declared("cleora.h")
    missing = [n for n in names if not hasattr(pkg, n) and n not in pkg.cleora.SIGNATURES]
    assert not missing, missing
    assert set(pkg.cleora.SIGNATURES) >= set(names)


def test_status_strings_without_a_device():
    lib = pkg.load()
    assert lib.cleora_status_string(0) == b"ok"
    assert lib.cleora_status_string(-4) == b"call out of order"


def test_library_is_built_for_sm_103a_only():
    flags = " ".join(pkg.build_native.ARCH)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert flags.count("-gencode") == 1

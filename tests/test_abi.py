"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every symbol
include/cleora.h declares (no compute call: there is no GPU here)."""
import os
import re

import ctypes

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


def test_noalloc_refuses_misaligned_or_overlapping_buffers_before_any_cuda_call():
    # The allocation-free step moves 16-byte vectors of T: misaligned (or overlapping) buffers
    # are refused by host checks that run before any CUDA call, so fake addresses are safe
    # here; only rejected combinations are passed.
    lib = pkg.load()
    f = lambda rp, c, v, tin, tout: lib.cleora_propagate_noalloc(rp, c, v, 4, 10, tin, tout, 8, 0, 0, None)
    assert f(0x10000, 0x20000, None, 0x30004, 0x40000) == pkg.CLEORA_ERR_INVALID_ARG  # T_in
    assert f(0x10000, 0x20000, None, 0x30000, 0x40008) == pkg.CLEORA_ERR_INVALID_ARG  # T_out
    assert f(0x10004, 0x20000, None, 0x30000, 0x40000) == pkg.CLEORA_ERR_INVALID_ARG  # rowptr
    assert f(0x10000, 0x20002, None, 0x30000, 0x40000) == pkg.CLEORA_ERR_INVALID_ARG  # col
    assert f(0x10000, 0x20000, 0x50001, 0x30000, 0x40000) == pkg.CLEORA_ERR_INVALID_ARG  # val
    assert f(0x10000, 0x20000, None, 0x30000, 0x30010) == pkg.CLEORA_ERR_INVALID_ARG  # overlap
    assert f(0x10000, 0x20000, None, 0x30000, None) == pkg.CLEORA_ERR_INVALID_ARG


def test_library_is_built_for_sm_103a_only():
    flags = " ".join(pkg.build_native.ARCH)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert flags.count("-gencode") == 1


def _job(E, d=128, storage="f32", directed=False, weighted=False, nodes_hint=0):
    job = pkg.cleora.cleora_job()
    job.num_edges = E
    job.directed = int(directed)
    job.d = d
    job.iters = 4
    job.storage = pkg.cleora.DTYPES[storage]
    job.nodes_hint = nodes_hint
    job.weights = 1 if weighted else None  # only its presence is read
    return job


def test_serving_memory_estimate_model():
    """The admission estimate (host arithmetic, no device): it covers the resident CSR and both
    embedding buffers, grows with edges, d, FP32 storage and weights, and adds the transient
    of the hot-first row partition once T is larger than twice the 72 MiB hot-row budget."""
    est = lambda **kw: pkg.cleora.load().cleora_serve_estimate(ctypes.byref(_job(**kw)))
    assert pkg.cleora.load().cleora_serve_estimate(None) == -1
    n, E = 1_000_000, 10_000_000
    base = est(E=E, nodes_hint=n)
    m = 2 * E
    assert base >= m * 8 + 2 * n * 128 * 4  # CSR entries, ping-pong FP32 T
    assert est(E=2 * E, nodes_hint=n) > base
    assert est(E=E, nodes_hint=n, d=256) > base
    assert est(E=E, nodes_hint=n, storage="bf16") < base
    assert est(E=E, nodes_hint=n, weighted=True) > base
    assert est(E=E, nodes_hint=n, directed=True) < base
    # T of 100k x 128 BF16 (25.6 MB) fits twice in the hot budget: no partition term; at
    # 2M nodes (512 MB) the partition's copy of the column array is counted
    small_t = est(E=E, nodes_hint=100_000, storage="bf16")
    big_t = est(E=E, nodes_hint=2_000_000, storage="bf16")
    assert big_t - small_t > m * 4


def test_server_config_is_checked_before_any_cuda_call():
    """Out-of-range slot counts and short-job limits are refused on the host."""
    lib = pkg.cleora.load()
    for kw in ({"short_slots": -1}, {"short_slots": 65}, {"short_job_seconds": -1.0},
               {"short_job_seconds": float("nan")}, {"max_slots": -1}, {"queue_capacity": -1}):
        cfg = pkg.cleora.cleora_server_config(0, 0, 2, 0, 0, 0, 0.0)
        for k, v in kw.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        assert lib.cleora_serve_create(ctypes.byref(h), ctypes.byref(cfg)) == pkg.CLEORA_ERR_INVALID_ARG
        assert not h.value


def _header_structs():
    """Field names and C types of every `typedef struct { ... } name;` in the header."""
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "cleora.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"((?:const )?\w+\s*\**)\s*(.+)", decl)
            ctype, names = m.group(1).replace(" ", ""), m.group(2)
            for n in names.split(","):
                n = n.strip()
                ptr = n.startswith("*")
                fields.append((n.lstrip("*").strip(), ctype + ("*" if ptr else "")))
        out[name] = fields
    return out


_C_SIZES = {"int": 4, "float": 4, "double": 8, "int64_t": 8, "uint64_t": 8, "cleora_dtype": 4}


def _c_layout_size(fields):
    off, align = 0, 1
    for _, t in fields:
        sz = 8 if t.endswith("*") else _C_SIZES[t.replace("const", "")]
        off = (off + sz - 1) // sz * sz + sz
        align = max(align, sz)
    return (off + align - 1) // align * align


def test_binding_structs_match_the_header():
    """Every struct the binding mirrors has the header's fields in the header's order, and the
    same size under the C layout rules (no device needed)."""
    structs = _header_structs()
    assert {"cleora_graph_desc", "cleora_server_config", "cleora_job", "cleora_result"} <= set(structs)
    for name, fields in structs.items():
        mirror = getattr(pkg.cleora, name)
        assert [f[0] for f in mirror._fields_] == [f[0] for f in fields], name
        assert ctypes.sizeof(mirror) == _c_layout_size(fields), name

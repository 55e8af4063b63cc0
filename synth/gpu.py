"""GPU edge-list generator for large power-law graphs (input generation only).

``libsynth_gpu.so`` implements ``synth.chung_lu_undirected_idx`` and ``synth.node_ids`` with
the same integer draws, so a graph generated here equals the numpy one bit for bit; it is
used where the host would take minutes (1.4 billion edges).  Outputs are torch CUDA tensors
(int64 holding the uint64 ids).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import shutil
import subprocess

import numpy as np

from . import ID_KEY, cdf_thresholds, solve_i0

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gen_gpu.cu")
LIB = os.path.join(HERE, "libsynth_gpu.so")
_lib = None


def build(force: bool = False) -> str:
    stamp_path = LIB + ".stamp"
    h = hashlib.sha256(open(SRC, "rb").read() + platform.machine().encode()).hexdigest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp_path) \
            and open(stamp_path).read() == h:
        return LIB
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", "-o", tmp, SRC],
                   check=True)
    os.replace(tmp, LIB)
    with open(stamp_path, "w") as f:
        f.write(h)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.synth_undirected_keys.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                              ctypes.c_int, ctypes.POINTER(P),
                                              ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_uint64)]
        lib.synth_undirected_keys.restype = ctypes.c_int
        lib.synth_keys_to_ids.argtypes = [P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, P, P]
        lib.synth_keys_to_ids.restype = ctypes.c_int
        lib.synth_free.argtypes = [P]
        lib.synth_free.restype = None
        _lib = lib
    return _lib


def chung_lu_undirected(n: int, E: int, gamma: float, seed: int, max_deg: float,
                        max_rounds: int = 64):
    """(src, dst) as CUDA int64 tensors of uint64 ids, plus metadata; equals
    ``synth.chung_lu_undirected`` for the same arguments."""
    import torch
    lib = _load()
    i0 = solve_i0(n, gamma, 2 * E, max_deg)
    thr = np.ascontiguousarray(cdf_thresholds(n, gamma, i0))
    keys = ctypes.c_void_p()
    count = ctypes.c_int64()
    cend = ctypes.c_uint64()
    torch.cuda.synchronize()
    rc = lib.synth_undirected_keys(thr.ctypes.data, n, E, seed & (2**64 - 1), max_rounds,
                                   ctypes.byref(keys), ctypes.byref(count), ctypes.byref(cend))
    if rc != 0:
        raise RuntimeError(f"GPU generator failed (cudaError {rc})")
    try:
        src = torch.empty(count.value, dtype=torch.int64, device="cuda")
        dst = torch.empty(count.value, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        rc = lib.synth_keys_to_ids(keys, count.value, seed & (2**64 - 1), ID_KEY,
                                   src.data_ptr(), dst.data_ptr())
        if rc != 0:
            raise RuntimeError(f"GPU generator failed (cudaError {rc})")
    finally:
        lib.synth_free(keys)
    return src, dst, {"i0": i0, "rounds_counter_end": cend.value, "edges": count.value}

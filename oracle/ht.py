"""Python face of the Hopcroft-Tarjan oracle (``ht_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The GPU library never
does, and nothing here imports the GPU library.

``solve(offsets, adj)`` runs the single-threaded C oracle and returns the
canonical outputs defined in ``ht_oracle.c`` (edge id = rank of the src<dst arc in
CSR order; BCCs numbered by their smallest edge id; head = shallowest vertex with
every connected component rooted at its smallest vertex id, section 4.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfbcc_oracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "ok", 1: "malformed CSR", 2: "not simple or not symmetric", 3: "out of host memory"}


def build(src: str = _SRC, out: str = _LIB, extra_flags=()) -> str:
    """Compile the oracle with gcc into ``out`` (skipped when up to date)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src) and not extra_flags:
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags, src, "-o", tmp])
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """Load (building first if needed) the oracle library; returns the ctypes handle."""
    global _lib
    with _lock:
        if path is not None:
            lib = ctypes.CDLL(path)
        elif _lib is not None:
            return _lib
        else:
            lib = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.fbcc_oracle_solve.argtypes = [i64, i64, p, p, p, p, p, p, p]
        lib.fbcc_oracle_solve.restype = ctypes.c_int
        lib.fbcc_oracle_check_csr.argtypes = [i64, i64, p, p]
        lib.fbcc_oracle_check_csr.restype = ctypes.c_int
        if path is None:
            _lib = lib
        return lib


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle rejected the input: {STATUS.get(code, code)}")
        self.code = code


def check_csr(offsets, adj) -> int:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    a = np.ascontiguousarray(adj, dtype=np.int32)
    n = off.size - 1
    return load().fbcc_oracle_check_csr(n, int(off[-1]) // 2, off.ctypes.data, a.ctypes.data)


def solve(offsets, adj, lib=None) -> dict:
    """Canonical BCC outputs of an undirected simple graph given as symmetric CSR.

    Returns a dict with ``edge_bcc`` (int32 per arc), ``bcc_head`` (int32, n_bcc),
    ``is_ap`` (uint8 per vertex), ``is_bridge`` (uint8 per arc) and the counts
    ``n_bcc``, ``n_ap``, ``n_bridge``, ``n_cc``. Raises OracleError on bad input.
    """
    lib = lib or load()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    a = np.ascontiguousarray(adj, dtype=np.int32)
    n = off.size - 1
    nnz = int(off[-1])
    if nnz % 2:
        raise OracleError(1)
    m = nnz // 2
    edge_bcc = np.empty(nnz, np.int32)
    bcc_head = np.empty(max(n, 1), np.int32)
    is_ap = np.empty(max(n, 1), np.uint8)
    is_bridge = np.empty(max(nnz, 1), np.uint8)
    stats = np.zeros(4, np.int64)
    rc = lib.fbcc_oracle_solve(n, m, off.ctypes.data, a.ctypes.data, edge_bcc.ctypes.data,
                               bcc_head.ctypes.data, is_ap.ctypes.data, is_bridge.ctypes.data,
                               stats.ctypes.data)
    if rc:
        raise OracleError(rc)
    nb = int(stats[0])
    return {
        "edge_bcc": edge_bcc,
        "bcc_head": bcc_head[:nb].copy(),
        "is_ap": is_ap[:n].copy(),
        "is_bridge": is_bridge[:nnz].copy(),
        "n_bcc": nb,
        "n_ap": int(stats[1]),
        "n_bridge": int(stats[2]),
        "n_cc": int(stats[3]),
    }

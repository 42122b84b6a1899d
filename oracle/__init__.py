"""TEST INFRASTRUCTURE ONLY: the CPU oracle for Expected Force (EF_2).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

Three independent computations live here:

* ``alg1``     -- Algorithm 1 (Section 4) written out literally in C, FP64:
  materialise every cluster (i, v, j), take its degree, update the
  histograms of its members (weights 1, 1, 2), then take the entropy of
  each histogram per Eq. 1.
* ``vertex``   -- the vertex-centric formulation (Section 4): per seed, visit
  every cluster credited to it and build its histogram (C, FP64, OpenMP).
* ``brute``    -- ordered two-step transmission sequences with the cluster
  out-degree counted edge by edge (Section 3.3's definition), pure Python,
  for tiny graphs only (``oracle.brute``).

Beside them: ``oracle.surrogate`` (the learned ranking path's features,
network and metrics), ``oracle.shard`` (Algorithm 1's loop over a range of
middle nodes, the sharded form) and ``oracle.sir`` (the SIR simulation of
Section 3.1 with Philox4x32-10 draws).

Graphs are passed as (row_ptr, col_idx) int32 numpy arrays of a symmetric
CSR with sorted rows, or any object carrying those two attributes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ef_oracle.c")
_LIB = os.path.join(_HERE, "libeforacle.so")
_lib = None


def build_lib(force: bool = False) -> str:
    """Compile ef_oracle.c (gcc -O2, OpenMP when the compiler has it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:2] + ["-fopenmp"] + base[2:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        lib.ef_oracle_alg1.argtypes = [ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp]
        lib.ef_oracle_vertex.argtypes = [ctypes.c_int32, vp, vp, ctypes.c_int64, vp, ctypes.c_int32,
                                         vp, vp, vp, vp, vp, vp]
        lib.ef_oracle_vertex_hist.argtypes = [ctypes.c_int32, vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
        lib.ef_oracle_alg1_hist.argtypes = [ctypes.c_int32, vp, vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
        lib.ef_oracle_triangles.argtypes = [ctypes.c_int32, vp, vp, vp]
        for f in ("ef_oracle_alg1", "ef_oracle_vertex", "ef_oracle_vertex_hist", "ef_oracle_alg1_hist",
                  "ef_oracle_triangles", "ef_oracle_num_threads"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _csr(g, col_idx=None):
    if col_idx is None:
        row_ptr, col_idx = g.row_ptr, g.col_idx
    else:
        row_ptr = g
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    return rp, ci, rp.shape[0] - 1


def _p(a):
    return a.ctypes.data


def alg1(g, col_idx=None) -> dict:
    """Algorithm 1 for every node: N, S (int64), T, EF (float64), flag (uint8)."""
    rp, ci, n = _csr(g, col_idx)
    out = dict(N=np.zeros(n, np.int64), S=np.zeros(n, np.int64), T=np.zeros(n, np.float64),
               EF=np.zeros(n, np.float64), flag=np.zeros(n, np.uint8))
    rc = _load().ef_oracle_alg1(n, _p(rp), _p(ci), _p(out["N"]), _p(out["S"]), _p(out["T"]),
                                _p(out["EF"]), _p(out["flag"]))
    if rc != 0:
        raise RuntimeError(f"ef_oracle_alg1 failed ({rc})")
    return out


def vertex(g, nodes=None, threads: int = 0, col_idx=None) -> dict:
    """Vertex-centric EF of the given seeds (all nodes when None); adds t = triangles."""
    rp, ci, n = _csr(g, col_idx)
    nodes = np.arange(n, dtype=np.int32) if nodes is None else np.ascontiguousarray(nodes, dtype=np.int32)
    k = nodes.shape[0]
    out = dict(N=np.zeros(k, np.int64), S=np.zeros(k, np.int64), T=np.zeros(k, np.float64),
               EF=np.zeros(k, np.float64), flag=np.zeros(k, np.uint8), t=np.zeros(k, np.int64))
    nodes_buf = nodes if k else np.zeros(1, np.int32)
    rc = _load().ef_oracle_vertex(n, _p(rp), _p(ci), k, _p(nodes_buf), threads, _p(out["N"]), _p(out["S"]),
                                  _p(out["T"]), _p(out["EF"]), _p(out["flag"]), _p(out["t"]))
    if rc != 0:
        raise RuntimeError(f"ef_oracle_vertex failed ({rc})")
    return out


def _hist(fn, g, s, col_idx=None):
    rp, ci, n = _csr(g, col_idx)
    deg = np.diff(rp)
    cap = int(3 * (deg.max() if n else 0) + 1)
    d = np.zeros(cap, np.int32)
    c = np.zeros(cap, np.int64)
    k = getattr(_load(), fn)(n, _p(rp), _p(ci), int(s), cap, _p(d), _p(c))
    if k < 0:
        raise RuntimeError(f"{fn} failed ({k})")
    return {int(a): int(b) for a, b in zip(d[:k], c[:k])}


def vertex_hist(g, s, col_idx=None) -> dict:
    """H_s as {degree: count} from the vertex-centric enumeration."""
    return _hist("ef_oracle_vertex_hist", g, s, col_idx)


def alg1_hist(g, s, col_idx=None) -> dict:
    """H_s as {degree: count} from Algorithm 1's Phases 1-2."""
    return _hist("ef_oracle_alg1_hist", g, s, col_idx)


def triangles(g, col_idx=None) -> np.ndarray:
    """t[v] = number of adjacent pairs of neighbours of v (plain definition)."""
    rp, ci, n = _csr(g, col_idx)
    t = np.zeros(max(n, 1), np.int64)
    rc = _load().ef_oracle_triangles(n, _p(rp), _p(ci), _p(t))
    if rc != 0:
        raise RuntimeError(f"ef_oracle_triangles failed ({rc})")
    return t[:n]


def num_threads() -> int:
    """Threads the OpenMP build uses by default (1 when built without OpenMP)."""
    return int(_load().ef_oracle_num_threads())

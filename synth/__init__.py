"""Seeded synthetic graphs shaped like the paper's workloads (Section 5.1, Table 1).

This module only builds inputs: symmetric, sorted, simple CSR graphs with int32
indices (nnz = 2|E|).  It holds none of the Expected-Force arithmetic, and it
imports neither the CUDA library nor the CPU oracle, so both can be fed from it.

Large generators are C (``graphgen.c``, compiled to ``libgraphgen.so`` by
``build_lib()``); the small closed-form families used as pins (complete graphs,
stars, paths, cycles, bipartite graphs, hypercubes, Petersen) are numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None

# Seeds of the five standard workloads: 20230606 + workload index.
SEED_BASE = 20230606


def build_lib(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_lib()
        lib = ctypes.CDLL(_LIB)
        P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
        I64P = ctypes.POINTER(ctypes.c_int64)
        lib.gg_erdos_renyi.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, P32, P32, I64P]
        lib.gg_barabasi_albert.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P32, P32, I64P]
        lib.gg_powerlaw_cm.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_uint64, P32, P32, I64P]
        lib.gg_watts_strogatz.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                          P32, P32, I64P]
        lib.gg_ws_batch.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, I64P, P32, P32, I64P]
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, P32, P32, I64P]
        lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      P32, P32, I64P]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        for f in ("gg_erdos_renyi", "gg_barabasi_albert", "gg_powerlaw_cm", "gg_watts_strogatz",
                  "gg_ws_batch", "gg_rmat", "gg_from_edges"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Symmetric CSR of an undirected simple graph (host numpy arrays)."""
    row_ptr: np.ndarray   # int32[n+1]
    col_idx: np.ndarray   # int32[nnz], nnz = 2|E|, rows sorted ascending
    name: str = ""
    graph_off: np.ndarray | None = None   # int64[G+1] for disjoint-union batches

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def wedges(self) -> int:
        """W = sum_v C(D_v, 2): the number of clusters Algorithm 1 enumerates."""
        d = self.degrees
        return int((d * (d - 1) // 2).sum())


def _call(fn, n_hint, *args) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    rp = ctypes.POINTER(ctypes.c_int32)()
    col = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rc = getattr(lib, fn)(*args, ctypes.byref(rp), ctypes.byref(col), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"{fn} failed with code {rc}")
    n = n_hint
    row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    col_idx = np.ctypeslib.as_array(col, shape=(max(int(nnz.value), 1),))[: int(nnz.value)].copy()
    lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(col, ctypes.c_void_p))
    return row_ptr, col_idx


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    rp, ci = _call("gg_erdos_renyi", n, n, p, seed)
    return Graph(rp, ci, f"er_n{n}_p{p}")


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    rp, ci = _call("gg_barabasi_albert", n, n, m, seed)
    return Graph(rp, ci, f"ba_n{n}_m{m}")


def powerlaw_cm(n: int, gamma: float, dmin: int, dmax: int, seed: int) -> Graph:
    rp, ci = _call("gg_powerlaw_cm", n, n, gamma, dmin, dmax, seed)
    return Graph(rp, ci, f"plcm_n{n}_g{gamma}_d{dmin}-{dmax}")


def watts_strogatz(n: int, k: int, p: float, seed: int) -> Graph:
    rp, ci = _call("gg_watts_strogatz", n, n, k, p, seed)
    return Graph(rp, ci, f"ws_n{n}_k{k}_p{p}")


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19) -> Graph:
    n = 1 << scale
    rp, ci = _call("gg_rmat", n, scale, edge_factor, a, b, c, seed)
    return Graph(rp, ci, f"rmat_s{scale}_ef{edge_factor}")


def ws_batch(G: int, nlo: int, nhi: int, klo: int, khi: int, p: float, seed: int) -> Graph:
    lib = _load()
    off = np.zeros(G + 1, dtype=np.int64)
    rp = ctypes.POINTER(ctypes.c_int32)()
    col = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64(0)
    rc = lib.gg_ws_batch(G, nlo, nhi, klo, khi, p, seed,
                         off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         ctypes.byref(rp), ctypes.byref(col), ctypes.byref(nnz))
    if rc != 0:
        raise RuntimeError(f"gg_ws_batch failed with code {rc}")
    n = int(off[-1])
    row_ptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    col_idx = np.ctypeslib.as_array(col, shape=(max(int(nnz.value), 1),))[: int(nnz.value)].copy()
    lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(col, ctypes.c_void_p))
    return Graph(row_ptr, col_idx, f"ws_batch_G{G}", graph_off=off)


def from_edges(n: int, edges) -> Graph:
    """CSR from an iterable of undirected (u, v) pairs; loops dropped, duplicates merged."""
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges, dtype=np.int32).reshape(-1, 2)
    u = np.ascontiguousarray(e[:, 0])
    v = np.ascontiguousarray(e[:, 1])
    rp, ci = _call("gg_from_edges", n, n, len(u), u.ctypes.data, v.ctypes.data)
    return Graph(rp, ci, f"edges_n{n}")


# ---------------------------------------------------------------- families

def complete(n: int) -> Graph:
    """K_n, built directly as CSR (row v = all other nodes, ascending)."""
    if n <= 1:
        return Graph(np.zeros(n + 1, np.int32), np.zeros(0, np.int32), f"K{n}")
    cols = np.tile(np.arange(n, dtype=np.int32), n).reshape(n, n)
    mask = ~np.eye(n, dtype=bool)
    col_idx = cols[mask].astype(np.int32)
    row_ptr = (np.arange(n + 1, dtype=np.int64) * (n - 1)).astype(np.int32)
    return Graph(row_ptr, col_idx, f"K{n}")


def star(k: int) -> Graph:
    """K_{1,k}: centre 0, leaves 1..k."""
    return from_edges(k + 1, [(0, i) for i in range(1, k + 1)])


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def complete_bipartite(r: int, s: int) -> Graph:
    """K_{r,s}: nodes 0..r-1 on one side, r..r+s-1 on the other; built directly as CSR."""
    left = np.tile(np.arange(r, r + s, dtype=np.int32), r)
    right = np.tile(np.arange(0, r, dtype=np.int32), s)
    col_idx = np.concatenate([left, right]).astype(np.int32)
    deg = np.concatenate([np.full(r, s, np.int64), np.full(s, r, np.int64)])
    row_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    return Graph(row_ptr, col_idx, f"K{r},{s}")


def hypercube(k: int) -> Graph:
    n = 1 << k
    return from_edges(n, [(v, v ^ (1 << b)) for v in range(n) for b in range(k) if v < v ^ (1 << b)])


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return from_edges(10, outer + spokes + inner)


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Graph with node v renamed perm[v]."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    e = np.stack([perm[src], perm[g.col_idx]], axis=1)
    e = e[e[:, 0] < e[:, 1]]
    return from_edges(g.n, e)


def disjoint_union(gs) -> Graph:
    off = 0
    edges = []
    offs = [0]
    for g in gs:
        src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
        e = np.stack([src + off, g.col_idx.astype(np.int64) + off], axis=1)
        edges.append(e[e[:, 0] < e[:, 1]])
        off += g.n
        offs.append(off)
    e = np.concatenate(edges) if edges else np.zeros((0, 2), np.int64)
    out = from_edges(off, e)
    out.graph_off = np.asarray(offs, dtype=np.int64)
    return out


# ------------------------------------------------------- standard workloads
# The five workloads: (1) ER G(2000, 0.004); (2) BA n=1e6, m=5; (3) power-law
# configuration model n=4e6, gamma=2.3, degrees in [3, 20000]; (4) 4096 WS
# graphs, n in [200, 20000], k even in [4, 12], p=0.1; (5) BA n=1.6e7, m=4.
# "3b" is workload 3 with minimum degree 6: about 4.4e7 undirected edges
# (8.7e7 CSR entries), the 44M-edge graph read as undirected edges.

def workload(idx, scale: float = 1.0) -> Graph:
    """Standard workload `idx` (1..5, or "3b"); `scale` < 1 shrinks node counts for tests."""
    if idx == "3b":
        return powerlaw_cm(max(10, int(4_000_000 * scale)), 2.3, 6, 20000 if scale >= 1 else
                           max(7, int(20000 * scale ** 0.5)), SEED_BASE + 6)
    seed = SEED_BASE + idx
    if idx == 1:
        return erdos_renyi(max(3, int(2000 * scale)), 0.004, seed)
    if idx == 2:
        return barabasi_albert(max(6, int(1_000_000 * scale)), 5, seed)
    if idx == 3:
        return powerlaw_cm(max(10, int(4_000_000 * scale)), 2.3, 3, 20000 if scale >= 1 else
                           max(4, int(20000 * scale ** 0.5)), seed)
    if idx == 4:
        G = max(1, int(4096 * scale))
        return ws_batch(G, 200, 20000 if scale >= 1 else max(200, int(20000 * scale ** 0.5)), 4, 12, 0.1, seed)
    if idx == 5:
        return barabasi_albert(max(5, int(16_000_000 * scale)), 4, seed)
    raise ValueError(idx)

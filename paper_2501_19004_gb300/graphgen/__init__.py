"""Seeded synthetic inputs for the Louvain method (SBM, R-MAT, grid).

The graphs follow the workload classes the paper evaluates on (Table 2:
web/social graphs with skewed degrees, low-degree road/k-mer graphs) and the
planted-partition case where the communities are known.  Every generator is
a pure function of its arguments: counter-based SplitMix64 in C, identical for
any thread count.  No part of the Louvain method lives here; the CUDA path and
the CPU oracle both consume these graphs.

A graph is returned as a :class:`CSR` of numpy arrays: ``offsets`` (int64,
n+1), ``cols`` (int32, nnz) and ``weights`` (int32, nnz, or ``None`` for unit
weights).  Both directions of every undirected edge are stored, self-loops are
dropped and duplicates merged, rows are sorted.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` in place (gcc, OpenMP) if it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i64, i32, u64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.gg_rmat.restype = vp
            lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64, ctypes.c_int, ctypes.c_int]
            lib.gg_sbm.restype = vp
            lib.gg_sbm.argtypes = [i64, i64, dbl, dbl, u64, ctypes.c_int]
            lib.gg_grid.restype = vp
            lib.gg_grid.argtypes = [i64, dbl, u64, ctypes.c_int, ctypes.c_int]
            lib.gg_from_pairs.restype = vp
            lib.gg_from_pairs.argtypes = [i64, i64, vp, vp]
            lib.gg_size.restype = None
            lib.gg_size.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32)]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [vp, vp, vp, vp]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [vp]
            lib.gg_sbm_union.restype = vp
            lib.gg_sbm_union.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            lib.gg_splitmix64.restype = u64
            lib.gg_splitmix64.argtypes = [u64, u64]
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class CSR:
    offsets: np.ndarray            # int64 [n+1]
    cols: np.ndarray               # int32 [nnz]
    weights: Optional[np.ndarray]  # int32 [nnz] or None (unit)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.cols.shape[0])

    def weights_or_ones(self) -> np.ndarray:
        return self.weights if self.weights is not None else np.ones(self.nnz, dtype=np.int32)

    def total_weight(self) -> int:
        """2m: the sum of all stored entries."""
        return int(self.weights.astype(np.int64).sum()) if self.weights is not None else self.nnz


def _take(handle, name: str) -> CSR:
    lib = _load()
    if not handle:
        raise MemoryError(f"graph generator failed for {name} (bad arguments or out of host memory)")
    try:
        n, nnz, weighted = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        lib.gg_size(handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(weighted))
        off = np.empty(n.value + 1, dtype=np.int64)
        col = np.empty(nnz.value, dtype=np.int32)
        w = np.empty(nnz.value, dtype=np.int32) if weighted.value else None
        lib.gg_copy(handle, off.ctypes.data, col.ctypes.data, w.ctypes.data if w is not None else None)
    finally:
        lib.gg_free(handle)
    return CSR(off, col, w, name)


def splitmix64(seed: int, idx: int) -> int:
    return int(_load().gg_splitmix64(seed & (2**64 - 1), idx & (2**64 - 1)))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 7, weight_range=(1, 1)) -> CSR:
    """R-MAT graph: 2^scale vertices, edge_factor * 2^scale samples."""
    h = _load().gg_rmat(scale, edge_factor, a, b, c, seed, weight_range[0], weight_range[1])
    return _take(h, f"rmat{scale}-ef{edge_factor}-s{seed}")


def sbm(n: int, block: int, p_in: float, p_out: float, seed: int, direct: Optional[bool] = None) -> CSR:
    """Planted-partition SBM with consecutive blocks of ``block`` vertices."""
    if direct is None:
        direct = n <= 4000
    h = _load().gg_sbm(n, block, p_in, p_out, seed, 1 if direct else 0)
    return _take(h, f"sbm{n}-b{block}-s{seed}")


def grid(side: int, long_frac: float = 0.02, seed: int = 11, weight_range=(1, 8)) -> CSR:
    """side x side 4-neighbour grid plus long_frac * grid-edges random pairs."""
    h = _load().gg_grid(side, long_frac, seed, weight_range[0], weight_range[1])
    return _take(h, f"grid{side}-s{seed}")


def from_pairs(n: int, u, v, weights=None, name: str = "pairs") -> CSR:
    """Symmetric CSR from an undirected pair list.  With ``weights`` (one per
    pair; duplicates must agree) the entries carry them, else unit weights."""
    u = np.ascontiguousarray(u, dtype=np.int64)
    v = np.ascontiguousarray(v, dtype=np.int64)
    g = _take(_load().gg_from_pairs(n, u.shape[0], u.ctypes.data, v.ctypes.data), name)
    if weights is not None:
        lut = {}
        for a, b, w in zip(u.tolist(), v.tolist(), list(weights)):
            lut[(min(a, b), max(a, b))] = int(w)
        ws = np.empty(g.nnz, dtype=np.int32)
        for i in range(g.n):
            for k in range(g.offsets[i], g.offsets[i + 1]):
                j = int(g.cols[k])
                ws[k] = lut[(min(i, j), max(i, j))]
        g.weights = ws
    return g


def ring_of_cliques(r: int, k: int) -> CSR:
    """r cliques K_k joined in a ring by one edge between consecutive cliques
    (vertex k*q+k-1 to vertex k*(q+1) mod r*k)."""
    us, vs = [], []
    for q in range(r):
        base = q * k
        for a in range(k):
            for b in range(a + 1, k):
                us.append(base + a)
                vs.append(base + b)
        us.append(base + k - 1)
        vs.append((base + k) % (r * k))
    return from_pairs(r * k, us, vs, name=f"ring{r}x{k}")


def batched_sbm_params(g: int):
    """Per-graph parameters of the batched planted-partition workload:
    n log-uniform in [200, 200000], mean degree uniform in [8, 32], mixing
    ratio mu uniform in [0.1, 0.4], blocks of 50; seed g."""
    u1 = (splitmix64(0xBA7C4ED, 3 * g) >> 11) / 2.0**53
    u2 = (splitmix64(0xBA7C4ED, 3 * g + 1) >> 11) / 2.0**53
    u3 = (splitmix64(0xBA7C4ED, 3 * g + 2) >> 11) / 2.0**53
    n = int(round(math.exp(math.log(200) + u1 * (math.log(200000) - math.log(200)))))
    dbar = 8.0 + 24.0 * u2
    mu = 0.1 + 0.3 * u3
    block = 50
    p_in = min(1.0, (1.0 - mu) * dbar / (block - 1))
    p_out = mu * dbar / max(1, n - block)
    return n, block, p_in, p_out


def batched_sbm(g: int) -> CSR:
    n, block, p_in, p_out = batched_sbm_params(g)
    c = sbm(n, block, p_in, p_out, seed=g, direct=False)
    c.name = f"bsbm{g}"
    return c


def concat(graphs) -> "tuple[CSR, np.ndarray]":
    """Union of several graphs (the input of a batched run): graph g's vertices
    become [vo[g], vo[g+1]) and its columns are shifted by vo[g].  Returns
    (union CSR, vo int64 [G+1]).  The union is weighted if any graph is."""
    graphs = list(graphs)
    G = len(graphs)
    vo = np.zeros(G + 1, dtype=np.int64)
    eo = np.zeros(G + 1, dtype=np.int64)
    for k, g in enumerate(graphs):
        vo[k + 1] = vo[k] + g.n
        eo[k + 1] = eo[k] + g.nnz
    off = np.empty(int(vo[G]) + 1, dtype=np.int64)
    col = np.empty(int(eo[G]), dtype=np.int32)
    weighted = any(g.weights is not None for g in graphs)
    w = np.empty(int(eo[G]), dtype=np.int32) if weighted else None
    for k, g in enumerate(graphs):
        a, b = int(vo[k]), int(vo[k + 1])
        off[a:b] = g.offsets[:-1] + eo[k]
        col[eo[k]:eo[k + 1]] = g.cols + np.int32(vo[k])
        if weighted:
            w[eo[k]:eo[k + 1]] = g.weights if g.weights is not None else 1
    off[int(vo[G])] = eo[G]
    return CSR(off, col, w, f"union{G}"), vo


def batched_sbm_union(G: int, first: int = 0):
    """Union of batched_sbm(first) .. batched_sbm(first + G - 1), generated in
    parallel; equals concat() of the single graphs.  Returns (CSR, vo)."""
    lib = _load()
    prm = [batched_sbm_params(g) for g in range(first, first + G)]
    n = np.array([p[0] for p in prm], dtype=np.int64)
    blk = np.array([p[1] for p in prm], dtype=np.int64)
    pin = np.array([p[2] for p in prm], dtype=np.float64)
    pout = np.array([p[3] for p in prm], dtype=np.float64)
    seed = np.arange(first, first + G, dtype=np.uint64)
    vo = np.zeros(G + 1, dtype=np.int64)
    h = lib.gg_sbm_union(G, n.ctypes.data, blk.ctypes.data, pin.ctypes.data, pout.ctypes.data, seed.ctypes.data,
                         vo.ctypes.data)
    c = _take(h, f"bsbm-union{first}+{G}")
    return c, vo


def num_threads() -> int:
    return int(_load().gg_num_threads())

"""CPU oracle for the Louvain method (arXiv 2501.19004).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library's
product path never does.  It shares no code with the CUDA path.

The arithmetic lives in ``louvain_oracle.c`` (plain C, exact 128-bit integer
sums, OpenMP only over independent decisions); this module compiles it with
gcc and wraps it with ctypes.  Each wrapper names the passage of the paper it
follows.

Parity status per function (what pins it, in tests/test_oracle_pins.py):
  modularity           Eq. 1 -- pinned (networkx, brute force, closed forms)
  delta_modularity     Eq. 2 -- pinned (exact rational Q(after) - Q(before))
  decide               Alg. 2/5 body -- pinned (brute-force argmax over moves)
  aggregate            Alg. 3/6 -- pinned (brute-force super-graph, Q invariance)
  bucket / fmix32      schedule hash -- pinned (MurmurHash3 published vectors,
                       bucket balance)
  louvain              Alg. 1/4 whole run -- pinned by invariants, closed forms
                       (ring of cliques, disjoint cliques), brute-force optimum
                       bound, planted-partition recovery
  refine               Leiden refinement (Traag et al. 2019; Sec. 5.2, Sec. 6)
                       -- pinned by brute-force merge choices, connectivity
                       and containment of the refined communities, the
                       well-connectedness condition, and aggregation
                       invariance; louvain(refine=True) by the whole-run pins
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "louvain_oracle.c")
_LIB = os.path.join(_HERE, "liblouvain_oracle.so")
_lock = threading.Lock()
_lib = None

ITER_FIELDS = 4
PASS_FIELDS = 6


def build(force: bool = False) -> str:
    """Compile ``liblouvain_oracle.so`` in place with gcc if it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class OrConfig(ctypes.Structure):
    _fields_ = [
        ("max_passes", ctypes.c_int32),
        ("max_iterations", ctypes.c_int32),
        ("tolerance", ctypes.c_double),
        ("tolerance_drop", ctypes.c_double),
        ("aggregation_tolerance", ctypes.c_double),
        ("pickless_period", ctypes.c_int32),
        ("buckets", ctypes.c_int32),
        ("schedule_seed", ctypes.c_uint64),
        ("check_invariants", ctypes.c_int32),
        ("num_threads", ctypes.c_int32),
        ("refine", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i64, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
            lib.or_louvain.restype = ctypes.c_int
            lib.or_louvain.argtypes = [i64, vp, vp, vp, ctypes.POINTER(OrConfig), vp, vp, vp, vp,
                                       ctypes.POINTER(ctypes.c_double)]
            lib.or_modularity.restype = ctypes.c_int
            lib.or_modularity.argtypes = [i64, vp, vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
            lib.or_delta_modularity.restype = ctypes.c_int
            lib.or_delta_modularity.argtypes = [i64, vp, vp, vp, vp, i64, i32, vp]
            lib.or_decide.restype = ctypes.c_int
            lib.or_decide.argtypes = [i64, vp, vp, vp, vp, i64, i32, vp]
            lib.or_aggregate.restype = ctypes.c_int
            lib.or_aggregate.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp, vp]
            lib.or_refine.restype = ctypes.c_int
            lib.or_refine.argtypes = [i64, vp, vp, vp, vp, i32, u64, i32, vp]
            lib.or_fmix32.restype = u32
            lib.or_fmix32.argtypes = [u32]
            lib.or_bucket.restype = u32
            lib.or_bucket.argtypes = [i64, i32, i32, u64, i32]
            lib.or_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _i128(hi: int, lo: int) -> int:
    return (int(hi) << 64) + (int(lo) & (2**64 - 1))


def _graph_args(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.int32)
    return off, col, w


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class Config:
    """Run parameters; defaults are the paper's (Sec. 4.1, Sec. 4.3)."""
    max_passes: int = 10
    max_iterations: int = 20
    tolerance: float = 0.01
    tolerance_drop: float = 10.0
    aggregation_tolerance: float = 0.8
    pickless_period: int = 4
    buckets: int = 4
    schedule_seed: int = 0
    check_invariants: bool = False
    num_threads: int = 0
    refine: bool = False  # Leiden: refine P before aggregating (or_louvain's refine)

    def c(self) -> OrConfig:
        return OrConfig(self.max_passes, self.max_iterations, self.tolerance, self.tolerance_drop,
                        self.aggregation_tolerance, self.pickless_period, self.buckets,
                        self.schedule_seed & (2**64 - 1), int(self.check_invariants), self.num_threads,
                        int(self.refine))


@dataclass
class Result:
    membership: np.ndarray
    modularity: float
    q_num: int
    q_den: int
    passes: int
    communities: int
    two_m: int
    exit_reason: int
    iter_stats: np.ndarray = field(repr=False)   # [passes, iterations, 4]
    pass_stats: np.ndarray = field(repr=False)   # [passes, 6]

    def iterations(self):
        """Per pass: list of (evaluated, moves, gain) for the iterations run."""
        out = []
        for p in range(self.passes):
            li = int(self.pass_stats[p, 2])
            out.append([(int(r[0]), int(r[1]), _i128(r[2], r[3])) for r in self.iter_stats[p, :li]])
        return out


def louvain(g, cfg: Optional[Config] = None) -> Result:
    """The whole method: Algorithm 1 / 4 with Algorithms 2/5 and 3/6, under
    the deterministic bucket schedule."""
    cfg = cfg or Config()
    lib = _load()
    off, col, w = _graph_args(g)
    n = off.shape[0] - 1
    memb = np.empty(max(n, 1), dtype=np.int32)
    it = np.zeros((max(cfg.max_passes, 1), cfg.max_iterations, ITER_FIELDS), dtype=np.int64)
    ps = np.zeros((max(cfg.max_passes, 1), PASS_FIELDS), dtype=np.int64)
    summ = np.zeros(8, dtype=np.int64)
    q = ctypes.c_double()
    cc = cfg.c()
    st = lib.or_louvain(n, _ptr(off), _ptr(col), _ptr(w), ctypes.byref(cc), _ptr(memb), _ptr(it), _ptr(ps),
                        _ptr(summ), ctypes.byref(q))
    if st != 0:
        raise RuntimeError(f"oracle louvain failed with status {st}")
    return Result(memb[:n], q.value, _i128(summ[2], summ[3]), _i128(summ[4], summ[5]), int(summ[0]),
                  int(summ[1]), int(summ[6]), int(summ[7]), it, ps)


def modularity(g, membership) -> tuple[float, int, int]:
    """Eq. 1: returns (Q, exact numerator, exact denominator) with
    Q = (2m*S_in - sum_c Sigma_c^2) / (2m)^2."""
    lib = _load()
    off, col, w = _graph_args(g)
    m = np.ascontiguousarray(membership, dtype=np.int32)
    num = np.zeros(2, dtype=np.int64)
    den = np.zeros(2, dtype=np.int64)
    q = ctypes.c_double()
    st = lib.or_modularity(off.shape[0] - 1, _ptr(off), _ptr(col), _ptr(w), _ptr(m), _ptr(num), _ptr(den),
                           ctypes.byref(q))
    if st != 0:
        raise RuntimeError(f"oracle modularity failed with status {st}")
    return q.value, _i128(num[0], num[1]), _i128(den[0], den[1])


def delta_modularity_scaled(g, membership, i: int, c: int) -> int:
    """Eq. 2 scaled by 2m^2: s(c) - s(d) for moving i from membership[i] to c."""
    lib = _load()
    off, col, w = _graph_args(g)
    m = np.ascontiguousarray(membership, dtype=np.int32)
    out = np.zeros(2, dtype=np.int64)
    st = lib.or_delta_modularity(off.shape[0] - 1, _ptr(off), _ptr(col), _ptr(w), _ptr(m), i, c, _ptr(out))
    if st != 0:
        raise RuntimeError(f"oracle delta_modularity failed with status {st}")
    return _i128(out[0], out[1])


def decide(g, membership, i: int, pickless: bool = False) -> tuple[bool, int, int]:
    """One local-moving decision for vertex i (Algorithm 5 body):
    returns (moves, target, 2m^2 * dQ of the move)."""
    lib = _load()
    off, col, w = _graph_args(g)
    m = np.ascontiguousarray(membership, dtype=np.int32)
    out = np.zeros(4, dtype=np.int64)
    st = lib.or_decide(off.shape[0] - 1, _ptr(off), _ptr(col), _ptr(w), _ptr(m), i, int(pickless), _ptr(out))
    if st != 0:
        raise RuntimeError(f"oracle decide failed with status {st}")
    return bool(out[0]), int(out[1]), _i128(out[2], out[3])


def aggregate(g, membership, ncomm: int):
    """Algorithm 3 / 6: super-vertex graph of a dense membership.
    Returns (offsets int64, cols int32, weights int64), rows sorted."""
    lib = _load()
    off, col, w = _graph_args(g)
    n = off.shape[0] - 1
    m = np.ascontiguousarray(membership, dtype=np.int32)
    nnz = ctypes.c_int64()
    st = lib.or_aggregate(n, _ptr(off), _ptr(col), _ptr(w), _ptr(m), ncomm, ctypes.byref(nnz), None, None, None)
    if st != 0:
        raise RuntimeError(f"oracle aggregate failed with status {st}")
    o = np.empty(ncomm + 1, dtype=np.int64)
    c = np.empty(max(nnz.value, 1), dtype=np.int32)
    ww = np.empty(max(nnz.value, 1), dtype=np.int64)
    st = lib.or_aggregate(n, _ptr(off), _ptr(col), _ptr(w), _ptr(m), ncomm, ctypes.byref(nnz), _ptr(o), _ptr(c),
                          _ptr(ww))
    if st != 0:
        raise RuntimeError(f"oracle aggregate failed with status {st}")
    return o, c[:nnz.value], ww[:nnz.value]


def refine(g, bound, pass_: int = 0, seed: int = 0, buckets: int = 16) -> np.ndarray:
    """The Leiden refinement of partition `bound` (ids in [0, n)) on g, one
    sweep over `buckets` buckets (a whole run with B buckets refines over 4B):
    refined ids, each the vertex id of one member (leiden_refine in
    louvain_oracle.c)."""
    lib = _load()
    off, col, w = _graph_args(g)
    n = off.shape[0] - 1
    b = np.ascontiguousarray(bound, dtype=np.int32)
    out = np.empty(max(n, 1), dtype=np.int32)
    st = lib.or_refine(n, _ptr(off), _ptr(col), _ptr(w), _ptr(b), pass_, seed & (2**64 - 1), buckets, _ptr(out))
    if st != 0:
        raise RuntimeError(f"oracle refine failed with status {st}")
    return out[:n]


def fmix32(h: int) -> int:
    return int(_load().or_fmix32(h & 0xFFFFFFFF))


def bucket(i: int, pass_: int, iteration: int, seed: int, buckets: int) -> int:
    return int(_load().or_bucket(i, pass_, iteration, seed & (2**64 - 1), buckets))


def num_threads() -> int:
    return int(_load().or_num_threads())

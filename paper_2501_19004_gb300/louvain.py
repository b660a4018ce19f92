"""Python binding of the C ABI in ``include/louvain.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
``liblouvain_gb300.so``.  If the library is missing this module raises; there
is no fallback.  Functions keep the ABI's names; :class:`Louvain` wraps a
context.

Graphs are :class:`paper_2501_19004_gb300.graphgen.CSR` objects (host numpy
arrays) or :class:`DeviceCSR` (torch CUDA tensors).  PyTorch provides device
memory and the current stream only.
"""
from __future__ import annotations

import contextlib
import ctypes
import json
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

STATUS = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_HASH_OVERFLOW", 5: "E_TIMEOUT",
          6: "E_OVERFLOW", 7: "E_STATE"}
MODE_PLAIN, MODE_LEARNED = 0, 1
KERNELS = ["select", "move_thread", "move_warp", "move_mid", "move_block", "move_hub", "apply", "pass_init",
           "comm_count", "comm_scatter", "merge_thread", "merge_warp", "merge_mid", "merge_block", "merge_big",
           "dendrogram", "modularity", "renumber", "move_hub_eval", "merge_big_emit", "mlp_select", "move_group",
           "move_wide", "merge_xl", "merge_group", "move_half"]


def kernel_mask(*names) -> int:
    """profile_mask bits for the named kernel groups."""
    m = 0
    for nm in names:
        m |= 1 << KERNELS.index(nm)
    return m
ITER_FIELDS, PASS_FIELDS = 4, 6


class LouvainError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LouvainGraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("cols", ctypes.c_void_p), ("weights", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class LouvainConfig(ctypes.Structure):
    _fields_ = [("max_passes", ctypes.c_int32), ("max_iterations", ctypes.c_int32),
                ("tolerance", ctypes.c_double), ("tolerance_drop", ctypes.c_double),
                ("aggregation_tolerance", ctypes.c_double), ("pickless_period", ctypes.c_int32),
                ("buckets", ctypes.c_int32), ("schedule_seed", ctypes.c_uint64), ("mode", ctypes.c_int32),
                ("model", ctypes.c_void_p), ("skip_threshold", ctypes.c_float),
                ("record_pass_modularity", ctypes.c_int32), ("check_symmetry", ctypes.c_int32),
                ("profile_mask", ctypes.c_uint32), ("trace_capacity", ctypes.c_int64), ("trace_rate", ctypes.c_float),
                ("learned_fallback", ctypes.c_int32), ("learned_skip_clears", ctypes.c_int32),
                ("table_window", ctypes.c_int64), ("asynchronous", ctypes.c_int32),
                ("learned_min_degree", ctypes.c_int32), ("refine", ctypes.c_int32)]


_lib = None


def load(path: Optional[str] = None):
    """Load the CUDA library (built by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: run paper_2501_19004_gb300.build.build() "
                           "(or __graft_entry__.build()) on a machine with nvcc")
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    lib.louvain_config_default.restype = None
    lib.louvain_config_default.argtypes = [P(LouvainConfig)]
    lib.louvain_create.restype = ctypes.c_int
    lib.louvain_create.argtypes = [P(LouvainGraph), P(LouvainConfig), vp, P(vp)]
    lib.louvain_run.restype = ctypes.c_int
    lib.louvain_run.argtypes = [vp]
    lib.louvain_run_passes.restype = ctypes.c_int
    lib.louvain_run_passes.argtypes = [vp, i32, P(i32)]
    lib.louvain_resume.restype = ctypes.c_int
    lib.louvain_resume.argtypes = [vp, i32, P(i32)]
    lib.louvain_save_state.restype = ctypes.c_int
    lib.louvain_save_state.argtypes = [vp, vp, ctypes.c_size_t, P(ctypes.c_size_t)]
    lib.louvain_load_state.restype = ctypes.c_int
    lib.louvain_load_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.louvain_modularity.restype = ctypes.c_int
    lib.louvain_modularity.argtypes = [vp, P(ctypes.c_double), vp, vp]
    lib.louvain_memberships.restype = ctypes.c_int
    lib.louvain_memberships.argtypes = [vp, vp, i32]
    lib.louvain_records.restype = ctypes.c_int
    lib.louvain_records.argtypes = [vp, vp, vp, vp]
    lib.louvain_stats.restype = ctypes.c_int
    lib.louvain_stats.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.louvain_set_profile.restype = ctypes.c_int
    lib.louvain_set_profile.argtypes = [vp, ctypes.c_uint32]
    lib.louvain_destroy.restype = None
    lib.louvain_destroy.argtypes = [vp]
    lib.louvain_last_error.restype = ctypes.c_char_p
    lib.louvain_last_error.argtypes = [vp]
    lib.louvain_modularity_of.restype = ctypes.c_int
    lib.louvain_modularity_of.argtypes = [P(LouvainGraph), vp, vp, P(ctypes.c_double), vp, vp]
    lib.louvain_traces.restype = ctypes.c_int
    lib.louvain_traces.argtypes = [vp, vp, vp, i64, P(i64), i32]
    lib.louvain_mlp_forward.restype = ctypes.c_int
    lib.louvain_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
    lib.louvain_mlp_gradient.restype = ctypes.c_int
    lib.louvain_mlp_gradient.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    lib.louvain_mlp_train.restype = ctypes.c_int
    lib.louvain_mlp_train.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_uint64, vp, vp]
    lib.louvain_modularity_noalloc.restype = ctypes.c_int
    lib.louvain_modularity_noalloc.argtypes = [P(LouvainGraph), vp, vp, P(ctypes.c_double), vp, vp]
    lib.louvain_create_batched.restype = ctypes.c_int
    lib.louvain_create_batched.argtypes = [P(LouvainGraph), vp, i64, P(LouvainConfig), vp, P(vp)]
    lib.louvain_batch_results.restype = ctypes.c_int
    lib.louvain_batch_results.argtypes = [vp, vp, vp, vp]
    lib.louvain_schedule_words.restype = i32
    lib.louvain_schedule_words.argtypes = []
    lib.louvain_get_schedule.restype = ctypes.c_int
    lib.louvain_get_schedule.argtypes = [vp, vp, i32]
    lib.louvain_set_schedule.restype = ctypes.c_int
    lib.louvain_set_schedule.argtypes = [vp, vp, i32]
    lib.louvain_autotune.restype = ctypes.c_int
    lib.louvain_autotune.argtypes = [vp, i32, ctypes.c_char_p, ctypes.c_size_t]
    lib.louvain_model_size.restype = i64
    lib.louvain_model_size.argtypes = []
    lib.louvain_version.restype = ctypes.c_char_p
    lib.louvain_version.argtypes = []
    if path is None:
        _lib = lib
    return lib


def _check(st: int, ctx=None):
    if st != 0:
        msg = load().louvain_last_error(ctx).decode(errors="replace")
        raise LouvainError(st, msg)


@dataclass
class Config:
    """Run parameters (defaults as in ``louvain_config_default``)."""
    max_passes: int = 10
    max_iterations: int = 20
    tolerance: float = 0.01
    tolerance_drop: float = 10.0
    aggregation_tolerance: float = 0.8
    pickless_period: int = 4
    buckets: int = 4
    schedule_seed: int = 0
    mode: int = MODE_PLAIN
    model: Optional[np.ndarray] = None
    skip_threshold: float = 0.5
    record_pass_modularity: bool = False
    check_symmetry: bool = False
    profile_mask: int = 0
    trace_capacity: int = 0
    trace_rate: float = 1.0
    learned_fallback: int = 0
    learned_skip_clears: int = 0
    table_window: int = 0
    asynchronous: bool = False
    learned_min_degree: int = 0
    refine: bool = False  # the Leiden form: refine P before aggregating it

    def c(self) -> LouvainConfig:
        self._model_keep = None
        mp = None
        if self.model is not None:
            self._model_keep = np.ascontiguousarray(self.model, dtype=np.float32)
            mp = self._model_keep.ctypes.data
        return LouvainConfig(self.max_passes, self.max_iterations, self.tolerance, self.tolerance_drop,
                             self.aggregation_tolerance, self.pickless_period, self.buckets,
                             self.schedule_seed & (2**64 - 1), self.mode, mp, self.skip_threshold,
                             int(self.record_pass_modularity), int(self.check_symmetry), self.profile_mask,
                             self.trace_capacity, self.trace_rate, self.learned_fallback,
                             self.learned_skip_clears, self.table_window, int(self.asynchronous),
                             self.learned_min_degree, int(self.refine))


@dataclass
class DeviceCSR:
    """A CSR held in torch CUDA tensors (int64 offsets, int32 cols/weights)."""
    offsets: "object"
    cols: "object"
    weights: "object" = None

    @property
    def n(self):
        return int(self.offsets.shape[0] - 1)

    @property
    def nnz(self):
        return int(self.cols.shape[0])

    @staticmethod
    def from_host(g, device="cuda"):
        import torch
        return DeviceCSR(torch.from_numpy(np.ascontiguousarray(g.offsets)).to(device),
                         torch.from_numpy(np.ascontiguousarray(g.cols)).to(device),
                         None if g.weights is None else torch.from_numpy(np.ascontiguousarray(g.weights)).to(device))


def _graph_struct(g):
    """(LouvainGraph, keep-alive list) for a host CSR or a DeviceCSR."""
    if isinstance(g, DeviceCSR):
        import torch
        for t, dt in ((g.offsets, torch.int64), (g.cols, torch.int32)):
            if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
                raise ValueError("DeviceCSR needs contiguous CUDA tensors: int64 offsets, int32 cols/weights")
        if g.weights is not None and (g.weights.dtype != torch.int32 or not g.weights.is_cuda):
            raise ValueError("DeviceCSR weights must be int32 CUDA tensors")
        gs = LouvainGraph(g.n, g.nnz, g.offsets.data_ptr(), g.cols.data_ptr(),
                          None if g.weights is None else g.weights.data_ptr(), 1)
        return gs, [g]
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.int32)
    gs = LouvainGraph(off.shape[0] - 1, col.shape[0], off.ctypes.data, col.ctypes.data,
                      None if w is None else w.ctypes.data, 0)
    return gs, [off, col, w]


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(None)


# ------------------------------------------------------------- ABI mirror
def louvain_config_default() -> LouvainConfig:
    c = LouvainConfig()
    load().louvain_config_default(ctypes.byref(c))
    return c


def louvain_create(graph, cfg: Optional[Config] = None, stream=None) -> ctypes.c_void_p:
    cfg = cfg or Config()
    gs, keep = _graph_struct(graph)
    cc = cfg.c()
    ctx = ctypes.c_void_p()
    st = load().louvain_create(ctypes.byref(gs), ctypes.byref(cc), stream if stream is not None else _current_stream(),
                               ctypes.byref(ctx))
    del keep
    _check(st, None)
    return ctx


def louvain_run(ctx):
    _check(load().louvain_run(ctx), ctx)


def louvain_run_passes(ctx, max_new_passes: int) -> bool:
    """Start a run; True if it stopped between two passes after
    ``max_new_passes`` passes (0 = run to the end)."""
    sus = ctypes.c_int32()
    _check(load().louvain_run_passes(ctx, int(max_new_passes), ctypes.byref(sus)), ctx)
    return bool(sus.value)


def louvain_resume(ctx, max_new_passes: int = 0) -> bool:
    """Continue a suspended run; True if it stopped again."""
    sus = ctypes.c_int32()
    _check(load().louvain_resume(ctx, int(max_new_passes), ctypes.byref(sus)), ctx)
    return bool(sus.value)


def louvain_save_state(ctx) -> np.ndarray:
    """Checkpoint of a suspended run as a uint8 array (host)."""
    size = ctypes.c_size_t()
    _check(load().louvain_save_state(ctx, None, 0, ctypes.byref(size)), ctx)
    buf = np.zeros((size.value + 7) // 8, dtype=np.int64).view(np.uint8)[:size.value]
    _check(load().louvain_save_state(ctx, buf.ctypes.data, size.value, ctypes.byref(size)), ctx)
    return buf


def louvain_load_state(ctx, buf) -> None:
    """Restore a checkpoint (bytes or a uint8 array) into ``ctx``."""
    if isinstance(buf, np.ndarray):
        raw = np.ascontiguousarray(buf).view(np.uint8).reshape(-1)
    else:
        raw = np.frombuffer(bytes(buf), dtype=np.uint8)
    if raw.ctypes.data % 8:
        raw = np.frombuffer(raw.tobytes(), dtype=np.uint8)  # fresh bytes objects are 8-byte aligned
    _check(load().louvain_load_state(ctx, raw.ctypes.data, raw.nbytes), ctx)


def louvain_modularity(ctx):
    q = ctypes.c_double()
    num = np.zeros(2, dtype=np.int64)
    den = np.zeros(2, dtype=np.int64)
    _check(load().louvain_modularity(ctx, ctypes.byref(q), num.ctypes.data, den.ctypes.data), ctx)
    return q.value, _i128(num), _i128(den)


def louvain_memberships(ctx, out=None, n=None):
    """Memberships into `out` (numpy int32 host array or int32 CUDA tensor);
    allocates a numpy array of length n when out is None."""
    if out is None:
        out = np.empty(n, dtype=np.int32)
    if isinstance(out, np.ndarray):
        assert out.dtype == np.int32 and out.flags.c_contiguous
        _check(load().louvain_memberships(ctx, out.ctypes.data, 0), ctx)
    else:
        _check(load().louvain_memberships(ctx, out.data_ptr(), 1), ctx)
    return out


def louvain_records(ctx, max_passes, max_iterations):
    it = np.zeros((max(max_passes, 1), max_iterations, ITER_FIELDS), dtype=np.int64)
    ps = np.zeros((max(max_passes, 1), PASS_FIELDS), dtype=np.int64)
    summ = np.zeros(8, dtype=np.int64)
    _check(load().louvain_records(ctx, it.ctypes.data, ps.ctypes.data, summ.ctypes.data), ctx)
    return it, ps, summ


def louvain_stats(ctx) -> dict:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().louvain_stats(ctx, buf, len(buf)), ctx)
    return json.loads(buf.value.decode())


def louvain_set_profile(ctx, mask: int):
    _check(load().louvain_set_profile(ctx, mask), ctx)


def louvain_destroy(ctx):
    load().louvain_destroy(ctx)


def louvain_modularity_of(graph, membership, stream=None):
    """Modularity (Eq. 1) of `membership` on `graph`, computed on the device.
    Returns (Q, exact numerator, exact denominator)."""
    gs, keep = _graph_struct(graph)
    if isinstance(graph, DeviceCSR):
        mp = membership.data_ptr()
    else:
        membership = np.ascontiguousarray(membership, dtype=np.int32)
        mp = membership.ctypes.data
    q = ctypes.c_double()
    num = np.zeros(2, dtype=np.int64)
    den = np.zeros(2, dtype=np.int64)
    st = load().louvain_modularity_of(ctypes.byref(gs), mp, stream if stream is not None else _current_stream(),
                                      ctypes.byref(q), num.ctypes.data, den.ctypes.data)
    del keep
    _check(st, None)
    return q.value, _i128(num), _i128(den)


def louvain_traces(ctx, cap: int, canonical: bool = True):
    """(features [count][8], labels [count]) recorded by the last run (numpy).
    The device appends samples in whatever order its threads finish; with
    `canonical` they are sorted (by label, then the features) so that the
    same run always yields the same training set in the same order."""
    feats = np.zeros((max(cap, 1), 8), dtype=np.float32)
    labels = np.zeros(max(cap, 1), dtype=np.float32)
    cnt = ctypes.c_int64()
    _check(load().louvain_traces(ctx, feats.ctypes.data, labels.ctypes.data, cap, ctypes.byref(cnt), 0), ctx)
    X, Y = feats[:cnt.value], labels[:cnt.value]
    if canonical and X.shape[0]:
        order = np.lexsort(tuple(X[:, k] for k in range(7, -1, -1)) + (Y,))
        X, Y = np.ascontiguousarray(X[order]), np.ascontiguousarray(Y[order])
    return X, Y


def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


def louvain_mlp_forward(params, X):
    """Logits of feature rows X (torch CUDA float32 [n][8]); params torch CUDA float32."""
    import torch
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(load().louvain_mlp_forward(_dev(params), _dev(X), X.shape[0], _dev(out), _current_stream()))
    return out


def louvain_mlp_gradient(params, X, Y):
    """(gradient, mean loss) of the BCE loss (torch CUDA tensors)."""
    import torch
    grad = torch.zeros(params.shape[0], dtype=torch.float32, device=X.device)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    _check(load().louvain_mlp_gradient(_dev(params), _dev(X), _dev(Y), X.shape[0], _dev(grad), _dev(loss),
                                       _current_stream()))
    return grad, float(loss.item())


def louvain_mlp_train(params, X, Y, epochs=10, batch=4096, lr=3e-3, seed=0):
    """Adam training in place of params (torch CUDA); returns per-epoch losses."""
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(load().louvain_mlp_train(_dev(params), _dev(X), _dev(Y), X.shape[0], epochs, batch, lr, seed,
                                    losses.ctypes.data, _current_stream()))
    return losses[:epochs]


def louvain_modularity_noalloc(graph, membership, stream=None):
    """louvain_modularity_of for a DeviceCSR and a CUDA membership tensor,
    with no allocation inside the library (fixed scratch; see louvain.h).
    Returns (status, Q, exact numerator, exact denominator)."""
    gs, keep = _graph_struct(graph)
    q = ctypes.c_double()
    num = np.zeros(2, dtype=np.int64)
    den = np.zeros(2, dtype=np.int64)
    st = load().louvain_modularity_noalloc(ctypes.byref(gs), ctypes.c_void_p(membership.data_ptr()),
                                           stream if stream is not None else _current_stream(), ctypes.byref(q),
                                           num.ctypes.data, den.ctypes.data)
    del keep
    return st, q.value, _i128(num), _i128(den)


def louvain_create_batched(graph, vertex_offsets, cfg: Optional[Config] = None, stream=None) -> ctypes.c_void_p:
    """Context for a batch: `graph` is the union, graph g owning the vertices
    [vertex_offsets[g], vertex_offsets[g+1])."""
    cfg = cfg or Config()
    gs, keep = _graph_struct(graph)
    vo = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
    cc = cfg.c()
    ctx = ctypes.c_void_p()
    st = load().louvain_create_batched(ctypes.byref(gs), vo.ctypes.data, vo.shape[0] - 1, ctypes.byref(cc),
                                       stream if stream is not None else _current_stream(), ctypes.byref(ctx))
    del keep
    _check(st, None)
    return ctx


def louvain_batch_results(ctx, num_graphs: int, max_passes: int):
    """(results [G][8], q [G], pass_records [G][max_passes][3]) of the last batched run."""
    res = np.zeros((num_graphs, 8), dtype=np.int64)
    q = np.zeros(num_graphs, dtype=np.float64)
    pr = np.zeros((num_graphs, max(max_passes, 1), 3), dtype=np.int64)
    _check(load().louvain_batch_results(ctx, res.ctypes.data, q.ctypes.data, pr.ctypes.data), ctx)
    return res, q, pr


SCHEDULE_FIELDS = ["group_max", "half_max", "warp_max",
                   "move_thread", "move_warp", "move_mid", "move_block", "move_hub", "move_group", "move_wide",
                   "unused_bin7", "move_half",
                   "merge_thread", "merge_warp", "merge_mid", "merge_block", "merge_big", "merge_xl", "merge_group",
                   "graphs", "concurrent"]


def louvain_schedule_words() -> int:
    """Number of int32 words of a launch schedule."""
    return int(load().louvain_schedule_words())


def louvain_last_error(ctx=None) -> str:
    """Description of the last error on ctx (or of the last failed create)."""
    return load().louvain_last_error(ctx).decode(errors="replace")


def louvain_get_schedule(ctx) -> dict:
    n = int(load().louvain_schedule_words())
    w = np.zeros(n, dtype=np.int32)
    _check(load().louvain_get_schedule(ctx, w.ctypes.data, n), ctx)
    return dict(zip(SCHEDULE_FIELDS, (int(v) for v in w)))


def louvain_set_schedule(ctx, sched: dict):
    """Set schedule fields (missing ones keep their current values)."""
    cur = louvain_get_schedule(ctx)
    cur.update(sched)
    w = np.array([cur[k] for k in SCHEDULE_FIELDS], dtype=np.int32)
    _check(load().louvain_set_schedule(ctx, w.ctypes.data, w.shape[0]), ctx)


def louvain_autotune(ctx, max_runs: int = 24) -> dict:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().louvain_autotune(ctx, max_runs, buf, len(buf)), ctx)
    return json.loads(buf.value.decode())


def louvain_model_size() -> int:
    return int(load().louvain_model_size())


@contextlib.contextmanager
def using_library(path: str):
    """Within the block, every call of this module goes to the library at
    `path` (a build of the same sources with other compile-time options,
    e.g. a probe bound for failure tests), then back to the default one."""
    global _lib
    saved = _lib
    _lib = load(path)
    try:
        yield _lib
    finally:
        _lib = saved


def louvain_version() -> str:
    return load().louvain_version().decode()


def _i128(a) -> int:
    return (int(a[0]) << 64) + (int(a[1]) & (2**64 - 1))


# ------------------------------------------------------------- convenience
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
    iter_stats: np.ndarray
    pass_stats: np.ndarray

    def iterations(self):
        out = []
        for p in range(self.passes):
            li = int(self.pass_stats[p, 2])
            out.append([(int(r[0]), int(r[1]), _i128(r[2:4])) for r in self.iter_stats[p, :li]])
        return out


class Louvain:
    """One graph on the device plus all workspace; ``run()`` can be repeated."""

    def __init__(self, graph, cfg: Optional[Config] = None, stream=None):
        self.cfg = cfg or Config()
        self.n = graph.n
        self.ctx = louvain_create(graph, self.cfg, stream)

    def run(self):
        louvain_run(self.ctx)
        return self

    def run_passes(self, max_new_passes: int) -> bool:
        """Start a run that stops between two passes after ``max_new_passes``
        passes; True if it stopped (False: finished)."""
        return louvain_run_passes(self.ctx, max_new_passes)

    def resume(self, max_new_passes: int = 0) -> bool:
        """Continue a stopped run (0 = to the end); True if it stopped again."""
        return louvain_resume(self.ctx, max_new_passes)

    def save_state(self) -> np.ndarray:
        """Checkpoint of the stopped run (uint8 array in host memory)."""
        return louvain_save_state(self.ctx)

    def load_state(self, buf):
        """Restore a checkpoint taken on the same graph and settings; resume()
        then continues the run."""
        louvain_load_state(self.ctx, buf)
        return self

    def result(self) -> Result:
        q, num, den = louvain_modularity(self.ctx)
        memb = louvain_memberships(self.ctx, n=self.n)
        it, ps, summ = louvain_records(self.ctx, self.cfg.max_passes, self.cfg.max_iterations)
        return Result(memb, q, num, den, int(summ[0]), int(summ[1]), int(summ[6]), int(summ[7]), it, ps)

    def stats(self) -> dict:
        return louvain_stats(self.ctx)

    def set_profile(self, mask: int):
        louvain_set_profile(self.ctx, mask)

    def schedule(self) -> dict:
        return louvain_get_schedule(self.ctx)

    def set_schedule(self, sched: dict):
        louvain_set_schedule(self.ctx, sched)

    def autotune(self, max_runs: int = 24) -> dict:
        return louvain_autotune(self.ctx, max_runs)

    def close(self):
        if self.ctx:
            louvain_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(graph, cfg: Optional[Config] = None) -> Result:
    with Louvain(graph, cfg) as lv:
        return lv.run().result()


@dataclass
class BatchResult:
    """Per-graph results of a batched run; memberships are local dense ids."""
    membership: np.ndarray      # [n] of the union
    vertex_offsets: np.ndarray  # [G+1]
    modularity: np.ndarray      # [G]
    summary: np.ndarray         # [G][8]: passes, communities, Qnum hi/lo, Qden hi/lo, 2m, exit reason
    pass_records: np.ndarray    # [G][max_passes][3]: n', l_i, |Gamma|

    def graph(self, g: int):
        """(membership, modularity, exact numerator, exact denominator, passes, communities, exit reason)."""
        a, b = int(self.vertex_offsets[g]), int(self.vertex_offsets[g + 1])
        r = self.summary[g]
        return (self.membership[a:b], float(self.modularity[g]), _i128(r[2:4]), _i128(r[4:6]), int(r[0]),
                int(r[1]), int(r[7]))


class LouvainBatch:
    """Many graphs in one context (louvain_create_batched); ``run()`` can be repeated."""

    def __init__(self, graph, vertex_offsets, cfg: Optional[Config] = None, stream=None):
        self.cfg = cfg or Config()
        self.n = graph.n
        self.vo = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
        self.G = self.vo.shape[0] - 1
        self.ctx = louvain_create_batched(graph, self.vo, self.cfg, stream)

    def run(self):
        louvain_run(self.ctx)
        return self

    def result(self) -> BatchResult:
        memb = louvain_memberships(self.ctx, n=self.n)
        res, q, pr = louvain_batch_results(self.ctx, self.G, self.cfg.max_passes)
        return BatchResult(memb, self.vo, q, res, pr)

    def stats(self) -> dict:
        return louvain_stats(self.ctx)

    def set_profile(self, mask: int):
        louvain_set_profile(self.ctx, mask)

    def schedule(self) -> dict:
        return louvain_get_schedule(self.ctx)

    def set_schedule(self, sched: dict):
        louvain_set_schedule(self.ctx, sched)

    def autotune(self, max_runs: int = 24) -> dict:
        return louvain_autotune(self.ctx, max_runs)

    def close(self):
        if self.ctx:
            louvain_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Python binding of libtc (include/tc.h): exact triangle counting on one GPU.

Thin ctypes marshalling over the C ABI.  PyTorch supplies device memory and
the current CUDA stream; every step of the computation runs in the library's
own CUDA kernels.  There is no CPU fallback: if ``libtc.so`` has not been
built (``python -m paper_1706_05151_gb300.build``) or no GPU is present, the
calls raise.

The functions mirror the C entry points:
    orient            tc_orient          Eq. (1), Definition 1, Figure 2 preprocessing
    count             tc_count           Figure 2 counting loop (Theorems 1-2)
    count_local       tc_count_local     Section 11 (T_v) and C_v (Preliminaries)
    list_triangles    tc_list_count + tc_list_write   Section 10
    sparsify_count    tc_sparsify_count  Section 9.1
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtc.so")

TC_OP_ORIENT, TC_OP_COUNT, TC_OP_LIST, TC_OP_SPARSIFY, TC_OP_BATCH, TC_OP_PARTITION = 0, 1, 2, 3, 4, 5
# cost functions of the paper's load-balancing schemes (Table "lbscheme"), as tc_cost
COST_VERTICES, COST_DEGREE, COST_DHAT, COST_DEG_DHAT, COST_DHAT_SQ, COST_WORK = 0, 1, 2, 3, 4, 5
STATUS = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_INVALID_GRAPH", 3: "TC_ERR_WORKSPACE",
          4: "TC_ERR_CAPACITY", 5: "TC_ERR_CUDA", 6: "TC_ERR_UNSUPPORTED", 7: "TC_ERR_TIMEOUT",
          8: "TC_ERR_REJECTED", 9: "TC_ERR_NOT_READY"}

# every symbol include/tc.h declares
EXPORTS = ["tc_ctx_create", "tc_ctx_destroy", "tc_ctx_set_async", "tc_ctx_status", "tc_status_string",
           "tc_last_error", "tc_ctx_sm_count", "tc_version", "tc_workspace_size", "tc_orient", "tc_count",
           "tc_count_local", "tc_list_count", "tc_list_write", "tc_list", "tc_analyze", "tc_sparsify_count",
           "tc_batch", "tc_serve_create", "tc_serve_destroy", "tc_serve_last_error", "tc_serve_add_graph",
           "tc_serve_remove_graph", "tc_serve_submit", "tc_serve_poll", "tc_serve_wait", "tc_serve_release",
           "tc_serve_stats",
           "tc_ctx_set_tuning", "tc_ctx_set_hub_min", "tc_ctx_set_profiling", "tc_ctx_stage_count", "tc_ctx_stage", "tc_ctx_reset_stats", "tc_ctx_launches",
           "tc_count_static", "tc_capture_begin", "tc_capture_end", "tc_exec_launch", "tc_exec_kernels",
           "tc_exec_destroy", "tc_partition", "tc_count_range", "tc_orient_by",
           "tc_sparsify_count_part", "tc_count_streamed_workspace_size", "tc_count_streamed",
           "tc_ctx_set_kernel_shape", "tc_orient_host"]


class TcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class TcResult(ctypes.Structure):
    """Mirror of the C struct tc_result."""
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_int32), ("graph_id", ctypes.c_int64),
                ("n", ctypes.c_int32), ("triangles", ctypes.c_uint64), ("tv", ctypes.c_void_p),
                ("cc", ctypes.c_void_p), ("tri", ctypes.c_void_p), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class TcServeConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("admit_timeout_ms", ctypes.c_int64), ("grid_div", ctypes.c_int32),
                ("tile_max", ctypes.c_int32), ("high_slots", ctypes.c_int32), ("small_edges", ctypes.c_int64)]


class TcServeStats(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("running", ctypes.c_int64), ("pool_used", ctypes.c_size_t),
                ("pool_capacity", ctypes.c_size_t), ("edges_done", ctypes.c_int64)]


class TcGraph(ctypes.Structure):
    """Mirror of the C struct tc_graph."""
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("cols", ctypes.c_void_p), ("deg", ctypes.c_void_p), ("dhat", ctypes.c_void_p)]


_lib = None
_lib_lock = threading.Lock()
vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t


def load_library(path: str = LIB_PATH):
    """Load libtc.so (raises if it is missing: the library has no fallback path)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run `python -m paper_1706_05151_gb300.build` "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        G = ctypes.POINTER(TcGraph)
        sigs = {
            "tc_ctx_create": (i32, [ctypes.c_int, ctypes.POINTER(vp)]),
            "tc_ctx_destroy": (None, [vp]),
            "tc_ctx_set_async": (i32, [vp, ctypes.c_int]),
            "tc_ctx_status": (i32, [vp, vp]),
            "tc_status_string": (ctypes.c_char_p, [i32]),
            "tc_last_error": (ctypes.c_char_p, [vp]),
            "tc_ctx_sm_count": (ctypes.c_int, [vp]),
            "tc_version": (ctypes.c_char_p, []),
            "tc_workspace_size": (i32, [ctypes.c_int, i32, i64, ctypes.POINTER(sz)]),
            "tc_orient": (i32, [vp, i32, i64, vp, vp, vp, vp, vp, vp, sz, vp]),
            "tc_count": (i32, [vp, G, vp, vp, sz, vp]),
            "tc_count_local": (i32, [vp, G, vp, vp, vp, vp, sz, vp]),
            "tc_list_count": (i32, [vp, G, vp, vp, sz, vp]),
            "tc_list_write": (i32, [vp, G, vp, i64, vp, sz, vp]),
            "tc_list": (i32, [vp, G, vp, i64, ctypes.POINTER(i64), vp, sz, vp]),
            "tc_analyze": (i32, [vp, G, vp, vp, vp, vp, i64, ctypes.POINTER(i64), vp, sz, vp]),
            "tc_batch": (i32, [vp, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
            "tc_orient_by": (i32, [vp, i32, i64, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
            "tc_orient_host": (i32, [vp, i32, i64, vp, vp, vp, vp, vp, vp, vp, sz, vp]),
            "tc_sparsify_count_part": (i32, [vp, G, ctypes.c_double, u64, i32, i32, i32, vp, vp, vp, sz, vp]),
            "tc_partition": (i32, [vp, G, i32, ctypes.c_int, vp, vp, vp, sz, vp]),
            "tc_count_range": (i32, [vp, G, i32, i32, vp, vp, vp, sz, vp]),
            "tc_count_streamed_workspace_size": (i32, [i32, i64, sz, ctypes.POINTER(sz)]),
            "tc_count_streamed": (i32, [vp, i32, i64, vp, vp, vp, vp, sz, vp, sz, vp]),
            "tc_capture_begin": (i32, [vp, vp]),
            "tc_capture_end": (i32, [vp, vp, ctypes.POINTER(vp)]),
            "tc_exec_launch": (i32, [vp, vp]),
            "tc_exec_kernels": (i64, [vp]),
            "tc_exec_destroy": (None, [vp]),
            "tc_sparsify_count": (i32, [vp, G, ctypes.c_double, u64, vp, vp, vp, sz, vp]),
            "tc_serve_create": (i32, [ctypes.c_int, ctypes.POINTER(TcServeConfig), vp, sz, ctypes.POINTER(vp)]),
            "tc_serve_destroy": (None, [vp]),
            "tc_serve_last_error": (ctypes.c_char_p, [vp]),
            "tc_serve_add_graph": (i32, [vp, i32, i64, vp, ctypes.POINTER(i64)]),
            "tc_serve_remove_graph": (i32, [vp, i64]),
            "tc_serve_submit": (i32, [vp, i64, ctypes.c_int, ctypes.POINTER(i64)]),
            "tc_serve_poll": (i32, [vp, i64, ctypes.POINTER(TcResult)]),
            "tc_serve_wait": (i32, [vp, i64, i64, ctypes.POINTER(TcResult)]),
            "tc_serve_release": (i32, [vp, i64]),
            "tc_serve_stats": (i32, [vp, ctypes.POINTER(TcServeStats)]),
            "tc_ctx_set_hub_min": (i32, [vp, i32]),
            "tc_ctx_set_tuning": (i32, [vp, i32, i32]),
            "tc_ctx_set_kernel_shape": (i32, [vp, i32, i32, i32, i32]),
            "tc_ctx_set_profiling": (i32, [vp, ctypes.c_int]),
            "tc_ctx_stage_count": (ctypes.c_int, [vp]),
            "tc_ctx_stage": (i32, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
            "tc_ctx_reset_stats": (i32, [vp]),
            "tc_ctx_launches": (i64, [vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device: torch.device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Context:
    """A tc_ctx bound to one CUDA device, with a reusable device workspace."""

    def __init__(self, device: int | torch.device = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libtc needs a CUDA GPU; none is available (there is no CPU fallback)")
        self.lib = load_library()
        self.device = torch.device("cuda", device if isinstance(device, int) else device.index or 0)
        h = vp()
        st = self.lib.tc_ctx_create(self.device.index, ctypes.byref(h))
        if st != 0:
            raise TcError(st, "tc_ctx_create failed")
        self.handle = h
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st != 0:
            raise TcError(st, self.lib.tc_last_error(self.handle).decode())

    @property
    def sm_count(self) -> int:
        return int(self.lib.tc_ctx_sm_count(self.handle))

    def set_async(self, on: bool):
        self.check(self.lib.tc_ctx_set_async(self.handle, 1 if on else 0))

    def status(self):
        self.check(self.lib.tc_ctx_status(self.handle, _stream(self.device)))

    def set_tuning(self, tile_max: int = 0, grid_div: int = 1):
        """tc_ctx_set_tuning: tile/block threshold on |N_v| and the share of the GPU per launch."""
        self.check(self.lib.tc_ctx_set_tuning(self.handle, int(tile_max), int(grid_div)))

    def set_kernel_shape(self, tile_ids: int = 0, tile_windows: int = 0, hash_batch: int = 0, hash_windows: int = 0):
        """tc_ctx_set_kernel_shape: tile kernel (256, 8) / (256, 4) / (128, 8); hash kernels' batch
        32 / 16 and windows in flight 4 / 8 (zeros: the defaults)."""
        self.check(self.lib.tc_ctx_set_kernel_shape(self.handle, int(tile_ids), int(tile_windows), int(hash_batch),
                                                    int(hash_windows)))

    def set_hub_min(self, hub_min: int = 0):
        """tc_ctx_set_hub_min: lists of >= hub_min ids take their longer-list in-edges (0 default, -1 off)."""
        self.check(self.lib.tc_ctx_set_hub_min(self.handle, hub_min))

    def set_profiling(self, on: bool):
        self.check(self.lib.tc_ctx_set_profiling(self.handle, 1 if on else 0))

    def reset_stats(self):
        self.check(self.lib.tc_ctx_reset_stats(self.handle))

    @property
    def launches(self) -> int:
        """Kernels this context launched since creation or the last reset_stats()."""
        return int(self.lib.tc_ctx_launches(self.handle))

    def stages(self) -> dict:
        """{stage name: (total ms, timed calls)} of the profiled kernel groups."""
        out = {}
        for i in range(int(self.lib.tc_ctx_stage_count(self.handle))):
            name, ms, calls = ctypes.c_char_p(), ctypes.c_double(), i64()
            self.check(self.lib.tc_ctx_stage(self.handle, i, ctypes.byref(name), ctypes.byref(ms),
                                             ctypes.byref(calls)))
            out[name.value.decode()] = (float(ms.value), int(calls.value))
        return out

    def workspace_size(self, op: int, n: int, m: int) -> int:
        b = sz(0)
        self.check(self.lib.tc_workspace_size(op, n, m, ctypes.byref(b)))
        return int(b.value)

    def workspace(self, op: int, n: int, m: int) -> torch.Tensor:
        need = self.workspace_size(op, n, m)
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def release_workspace(self):
        """Drop the cached workspace (it is reallocated by the next call that needs one)."""
        self._ws = None


_default_ctx: dict[int, Context] = {}


def default_context(device: int = 0) -> Context:
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


@dataclass
class Graph:
    """An oriented graph in device memory (the C struct tc_graph)."""
    n: int
    m: int
    offsets: torch.Tensor  # int64[n+1]
    cols: torch.Tensor     # int32[m]
    deg: torch.Tensor | None = None   # int32[n]
    dhat: torch.Tensor | None = None  # int32[n]

    def struct(self) -> TcGraph:
        return TcGraph(self.n, self.m, self.offsets.data_ptr(), self.cols.data_ptr() if self.m else None,
                       self.deg.data_ptr() if self.deg is not None else None,
                       self.dhat.data_ptr() if self.dhat is not None else None)


def orient(edges: torch.Tensor, n: int, ctx: Context | None = None, keys: torch.Tensor | None = None) -> Graph:
    """tc_orient: edges int32[m, 2] on the GPU (each undirected edge once) -> oriented CSR.
    With keys (int64[n] on the GPU), tc_orient_by: v before u iff (keys[v], v) < (keys[u], u)."""
    ctx = ctx or default_context()
    dev = ctx.device
    if edges.device != dev or edges.dtype != torch.int32 or edges.dim() != 2 or edges.shape[1] != 2:
        raise ValueError("edges must be an int32 [m, 2] tensor on the context's device")
    edges = edges.contiguous()
    m = int(edges.shape[0])
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    cols = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    deg = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    dhat = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ws = ctx.workspace(TC_OP_ORIENT, n, m)
    if keys is None:
        ctx.check(ctx.lib.tc_orient(ctx.handle, n, m, _ptr(edges) if m else None, _ptr(offsets), _ptr(cols),
                                    _ptr(deg), _ptr(dhat), _ptr(ws), ws.numel(), _stream(dev)))
    else:
        if keys.device != dev or keys.dtype != torch.int64 or keys.shape != (n,):
            raise ValueError("keys must be an int64 [n] tensor on the context's device")
        keys = keys.contiguous()
        ctx.check(ctx.lib.tc_orient_by(ctx.handle, n, m, _ptr(edges) if m else None, _ptr(keys), _ptr(offsets),
                                       _ptr(cols), _ptr(deg), _ptr(dhat), _ptr(ws), ws.numel(), _stream(dev)))
    return Graph(n, m, offsets, cols[:m], deg[:n], dhat[:n])


def orient_host(edges_host: torch.Tensor, n: int, ctx: Context | None = None,
                edges_dev: torch.Tensor | None = None) -> tuple[Graph, torch.Tensor]:
    """tc_orient_host: edges int32[m, 2] in page-locked host memory -> (oriented CSR, the device copy).

    The copy goes up in chunks on the context's copy stream while the degree pass
    counts the chunks already there.  edges_dev (int32[m, 2] on the device) is
    reused when given, else allocated."""
    ctx = ctx or default_context()
    dev = ctx.device
    if edges_host.device.type != "cpu" or edges_host.dtype != torch.int32 or edges_host.dim() != 2 \
            or edges_host.shape[1] != 2 or not edges_host.is_contiguous():
        raise ValueError("edges_host must be a contiguous int32 [m, 2] tensor in host memory")
    m = int(edges_host.shape[0])
    if edges_dev is None:
        edges_dev = torch.empty((max(m, 1), 2), dtype=torch.int32, device=dev)
    elif edges_dev.device != dev or edges_dev.dtype != torch.int32 or edges_dev.numel() < 2 * m \
            or not edges_dev.is_contiguous():
        raise ValueError("edges_dev must be a contiguous int32 tensor of at least [m, 2] on the context's device")
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    cols = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    deg = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    dhat = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ws = ctx.workspace(TC_OP_ORIENT, n, m)
    ctx.check(ctx.lib.tc_orient_host(ctx.handle, n, m, edges_host.data_ptr() if m else None,
                                     _ptr(edges_dev) if m else None, _ptr(offsets), _ptr(cols), _ptr(deg),
                                     _ptr(dhat), _ptr(ws), ws.numel(), _stream(dev)))
    return Graph(n, m, offsets, cols[:m], deg[:n], dhat[:n]), edges_dev[:m]


def count(g: Graph, ctx: Context | None = None, out: torch.Tensor | None = None) -> int:
    """tc_count: the exact triangle count T."""
    ctx = ctx or default_context()
    total = out if out is not None else torch.empty(1, dtype=torch.int64, device=ctx.device)
    ws = ctx.workspace(TC_OP_COUNT, g.n, g.m)
    ctx.check(ctx.lib.tc_count(ctx.handle, ctypes.byref(g.struct()), _ptr(total), _ptr(ws), ws.numel(),
                               _stream(ctx.device)))
    return int(total.item()) if out is None else total


def count_local(g: Graph, clustering: bool = True, ctx: Context | None = None):
    """tc_count_local: (T, T_v int64[n], C_v float64[n] or None)."""
    ctx = ctx or default_context()
    total = torch.empty(1, dtype=torch.int64, device=ctx.device)
    tv = torch.empty(max(g.n, 1), dtype=torch.int64, device=ctx.device)
    cc = torch.empty(max(g.n, 1), dtype=torch.float64, device=ctx.device) if clustering else None
    ws = ctx.workspace(TC_OP_COUNT, g.n, g.m)
    ctx.check(ctx.lib.tc_count_local(ctx.handle, ctypes.byref(g.struct()), _ptr(total), _ptr(tv), _ptr(cc),
                                     _ptr(ws), ws.numel(), _stream(ctx.device)))
    return int(total.item()), tv[: g.n], (cc[: g.n] if cc is not None else None)


def list_triangles(g: Graph, ctx: Context | None = None) -> torch.Tensor:
    """tc_list_count then tc_list_write: int32[T, 3] triples (v, u, w), v < u < w in the order."""
    ctx = ctx or default_context()
    total = torch.empty(1, dtype=torch.int64, device=ctx.device)
    ws = ctx.workspace(TC_OP_LIST, g.n, g.m)
    gs = g.struct()
    ctx.check(ctx.lib.tc_list_count(ctx.handle, ctypes.byref(gs), _ptr(total), _ptr(ws), ws.numel(),
                                    _stream(ctx.device)))
    T = int(total.item())
    tri = torch.empty((max(T, 1), 3), dtype=torch.int32, device=ctx.device)
    ctx.check(ctx.lib.tc_list_write(ctx.handle, ctypes.byref(gs), _ptr(tri), T, _ptr(ws), ws.numel(),
                                    _stream(ctx.device)))
    return tri[:T]


def list_triangles_into(g: Graph, tri: torch.Tensor, ctx: Context | None = None) -> int:
    """tc_list: both passes into a caller buffer int32[cap, 3]; returns T (raises TC_ERR_CAPACITY)."""
    ctx = ctx or default_context()
    ws = ctx.workspace(TC_OP_LIST, g.n, g.m)
    cnt = i64(0)
    ctx.check(ctx.lib.tc_list(ctx.handle, ctypes.byref(g.struct()), _ptr(tri), int(tri.shape[0]),
                              ctypes.byref(cnt), _ptr(ws), ws.numel(), _stream(ctx.device)))
    return int(cnt.value)


def analyze(g: Graph, clustering: bool = True, tri: torch.Tensor | None = None, ctx: Context | None = None):
    """tc_analyze: (T, T_v int64[n], C_v float64[n] or None, triples int32[T, 3]).

    `tri` is an optional int32[cap, 3] output buffer; if it is too small (or
    absent) the call is repeated once with a buffer of exactly T rows.
    """
    ctx = ctx or default_context()
    total = torch.empty(1, dtype=torch.int64, device=ctx.device)
    tv = torch.empty(max(g.n, 1), dtype=torch.int64, device=ctx.device)
    cc = torch.empty(max(g.n, 1), dtype=torch.float64, device=ctx.device) if clustering else None
    ws = ctx.workspace(TC_OP_LIST, g.n, g.m)
    gs = g.struct()
    if tri is None:
        tri = torch.empty((1, 3), dtype=torch.int32, device=ctx.device)
    cnt = i64(0)

    def call(buf):
        return ctx.lib.tc_analyze(ctx.handle, ctypes.byref(gs), _ptr(total), _ptr(tv), _ptr(cc), _ptr(buf),
                                  int(buf.shape[0]), ctypes.byref(cnt), _ptr(ws), ws.numel(), _stream(ctx.device))
    st = call(tri)
    if st == 4:
        tri = torch.empty((max(int(cnt.value), 1), 3), dtype=torch.int32, device=ctx.device)
        st = call(tri)
    ctx.check(st)
    T = int(cnt.value)
    return T, tv[: g.n], (cc[: g.n] if cc is not None else None), tri[:T]


def sparsify_count(g: Graph, q: float, seed: int, ctx: Context | None = None):
    """tc_sparsify_count: (T' of the kept graph, kept edges, estimate T'/q^3)."""
    ctx = ctx or default_context()
    kept_tri = torch.empty(1, dtype=torch.int64, device=ctx.device)
    kept_edges = torch.empty(1, dtype=torch.int64, device=ctx.device)
    ws = ctx.workspace(TC_OP_SPARSIFY, g.n, g.m)
    ctx.check(ctx.lib.tc_sparsify_count(ctx.handle, ctypes.byref(g.struct()), float(q), int(seed),
                                        _ptr(kept_tri), _ptr(kept_edges), _ptr(ws), ws.numel(),
                                        _stream(ctx.device)))
    t = int(kept_tri.item())
    est = float(t) / (q * q * q) if q > 0 else float("nan")
    return t, int(kept_edges.item()), est


def sparsify_count_part(g: Graph, q: float, seed: int, part: int, v_begin: int, v_end: int,
                        kept: torch.Tensor, ctx: Context | None = None) -> int:
    """tc_sparsify_count_part: ADD to kept (int64[1]) the triangles with apex in [v_begin, v_end)
    that survive this part's own coins; returns the number of edges those coins keep."""
    ctx = ctx or default_context()
    kept_edges = torch.zeros(1, dtype=torch.int64, device=ctx.device)
    ws = ctx.workspace(TC_OP_SPARSIFY, g.n, g.m)
    ctx.check(ctx.lib.tc_sparsify_count_part(ctx.handle, ctypes.byref(g.struct()), float(q), int(seed), int(part),
                                             int(v_begin), int(v_end), _ptr(kept), _ptr(kept_edges), _ptr(ws),
                                             ws.numel(), _stream(ctx.device)))
    return int(kept_edges.item())


def partition(g: Graph, parts: int, cost: int = COST_WORK, ctx: Context | None = None):
    """tc_partition: (bounds int64[parts+1], per-part cost uint64[parts] as int64) on the device."""
    ctx = ctx or default_context()
    bounds = torch.empty(parts + 1, dtype=torch.int64, device=ctx.device)
    costs = torch.empty(parts, dtype=torch.int64, device=ctx.device)
    ws = ctx.workspace(TC_OP_PARTITION, g.n, g.m)
    ctx.check(ctx.lib.tc_partition(ctx.handle, ctypes.byref(g.struct()), parts, cost, _ptr(bounds), _ptr(costs),
                                   _ptr(ws), ws.numel(), _stream(ctx.device)))
    return bounds, costs


def count_range(g: Graph, v_begin: int, v_end: int, total: torch.Tensor, tv: torch.Tensor | None = None,
                ctx: Context | None = None):
    """tc_count_range: ADD the triangles whose apex is in [v_begin, v_end) to total (int64[1])
    and, if given, each vertex's share to tv (int64[n])."""
    ctx = ctx or default_context()
    ws = ctx.workspace(TC_OP_COUNT, g.n, g.m)
    ctx.check(ctx.lib.tc_count_range(ctx.handle, ctypes.byref(g.struct()), int(v_begin), int(v_end), _ptr(total),
                                     _ptr(tv), _ptr(ws), ws.numel(), _stream(ctx.device)))


def count_streamed(offsets_host: torch.Tensor, cols_host: torch.Tensor, list_bytes: int, local: bool = False,
                   ctx: Context | None = None):
    """tc_count_streamed: T (and T_v if local) of an oriented CSR held in host memory
    (offsets int64[n+1], cols int32[m]; page-locked for overlapped copies), counted
    through a device list buffer of list_bytes.  Returns (T, tv or None)."""
    ctx = ctx or default_context()
    if offsets_host.is_cuda or cols_host.is_cuda:
        raise ValueError("count_streamed takes the CSR in host memory")
    off = offsets_host.contiguous()
    cols = cols_host.contiguous()
    assert off.dtype == torch.int64 and cols.dtype == torch.int32
    n, m = off.numel() - 1, cols.numel()
    need = sz(0)
    ctx.check(ctx.lib.tc_count_streamed_workspace_size(n, m, int(list_bytes), ctypes.byref(need)))
    ws = torch.empty(max(int(need.value), 256), dtype=torch.uint8, device=ctx.device)
    total = torch.empty(1, dtype=torch.int64, device=ctx.device)
    tv = torch.empty(max(n, 1), dtype=torch.int64, device=ctx.device) if local else None
    ctx.check(ctx.lib.tc_count_streamed(ctx.handle, n, m, vp(off.data_ptr()), vp(cols.data_ptr() if m else 0),
                                        _ptr(total), _ptr(tv), int(list_bytes), _ptr(ws), ws.numel(),
                                        _stream(ctx.device)))
    T = int(total.item())
    return T, (tv[:n] if local else None)


@dataclass
class Batch:
    """Inputs of tc_batch on the device: the graphs side by side."""
    G: int
    N: int
    E: int
    vbase: torch.Tensor   # int64[G+1]
    ebase: torch.Tensor   # int64[G+1]
    edges: torch.Tensor   # int32[E, 2], local ids


def make_batch(graphs, device) -> Batch:
    """Concatenate [(n_g, edges_g int32[m_g, 2] with local ids), ...] into tc_batch inputs."""
    import numpy as np
    ns = np.array([int(n) for n, _ in graphs], dtype=np.int64)
    ms = np.array([len(e) for _, e in graphs], dtype=np.int64)
    vbase = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    ebase = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    edges = np.concatenate([np.asarray(e, dtype=np.int32).reshape(-1, 2) for _, e in graphs]) if len(graphs) \
        else np.zeros((0, 2), np.int32)
    return Batch(len(graphs), int(vbase[-1]), int(ebase[-1]), torch.from_numpy(vbase).to(device),
                 torch.from_numpy(ebase).to(device), torch.from_numpy(np.ascontiguousarray(edges)).to(device))


def batch(b: Batch, local: bool = True, ctx: Context | None = None):
    """tc_batch: (totals int64[G], tv int64[N] or None, the oriented union as a Graph)."""
    ctx = ctx or default_context()
    dev = ctx.device
    N, E = b.N, b.E
    offsets = torch.empty(N + 1, dtype=torch.int64, device=dev)
    cols = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
    deg = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    dhat = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    totals = torch.empty(b.G, dtype=torch.int64, device=dev)
    tv = torch.empty(max(N, 1), dtype=torch.int64, device=dev) if local else None
    ws = ctx.workspace(TC_OP_BATCH, N, E)
    ctx.check(ctx.lib.tc_batch(ctx.handle, b.G, N, E, _ptr(b.vbase), _ptr(b.ebase), _ptr(b.edges) if E else None,
                               _ptr(offsets), _ptr(cols), _ptr(deg), _ptr(dhat), _ptr(totals), _ptr(tv),
                               _ptr(ws), ws.numel(), _stream(dev)))
    return totals, (tv[:N] if tv is not None else None), Graph(N, E, offsets, cols[:E], deg[:N], dhat[:N])


class CapturedBatch:
    """tc_batch recorded once as a CUDA graph (tc_capture_begin / tc_capture_end)
    and replayed with one launch per call.

    Every buffer the sequence touches -- outputs and a workspace of its own -- is
    allocated here, before the capture, and kept alive by this object.  A replay
    re-runs the recorded kernels on b's device buffers: refill b.edges (and
    b.vbase, b.ebase, for graphs of the same G, N and E) in place between replays.
    """

    def __init__(self, b: Batch, local: bool = True, ctx: Context | None = None):
        self.ctx = ctx = ctx or default_context()
        dev = ctx.device
        self.b = b
        N, E = b.N, b.E
        self.offsets = torch.empty(N + 1, dtype=torch.int64, device=dev)
        self.cols = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
        self.deg = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
        self.dhat = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
        self.totals = torch.empty(b.G, dtype=torch.int64, device=dev)
        self.tv = torch.empty(max(N, 1), dtype=torch.int64, device=dev) if local else None
        self.ws = torch.empty(max(ctx.workspace_size(TC_OP_BATCH, N, E), 1), dtype=torch.uint8, device=dev)
        self.handle = None
        stream = torch.cuda.Stream(dev)
        stream.wait_stream(torch.cuda.current_stream(dev))
        lib, h = ctx.lib, ctx.handle
        sp = ctypes.c_void_p(stream.cuda_stream)
        ctx.check(lib.tc_capture_begin(h, sp))
        st = lib.tc_batch(h, b.G, N, E, _ptr(b.vbase), _ptr(b.ebase), _ptr(b.edges) if E else None,
                          _ptr(self.offsets), _ptr(self.cols), _ptr(self.deg), _ptr(self.dhat), _ptr(self.totals),
                          _ptr(self.tv), _ptr(self.ws), self.ws.numel(), sp)
        x = vp()
        st_end = lib.tc_capture_end(h, sp, ctypes.byref(x))
        ctx.check(st if st != 0 else st_end)
        self.handle = x
        self.kernels = int(lib.tc_exec_kernels(x))

    def replay(self, stream: torch.cuda.Stream | None = None):
        """Enqueue one replay on `stream` (default: the current stream)."""
        s = stream or torch.cuda.current_stream(self.ctx.device)
        self.ctx.check(self.ctx.lib.tc_exec_launch(self.handle, ctypes.c_void_p(s.cuda_stream)))

    def result(self):
        """(totals int64[G], tv int64[N] or None, the oriented union as a Graph) of the last replay."""
        N, E = self.b.N, self.b.E
        return (self.totals, self.tv[:N] if self.tv is not None else None,
                Graph(N, E, self.offsets, self.cols[:E], self.deg[:N], self.dhat[:N]))

    def close(self):
        if self.handle is not None:
            self.ctx.lib.tc_exec_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """A zero-copy view of device memory for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


COUNT, LOCAL, LIST = 0, 1, 2


@dataclass
class ServeResult:
    ticket: int
    status: int
    kind: int
    graph_id: int
    triangles: int
    queue_ms: float
    latency_ms: float
    tv: torch.Tensor | None = None
    cc: torch.Tensor | None = None
    tri: torch.Tensor | None = None


class Server:
    """tc_serve_*: a continuous-batching request server over resident graphs.

    The device pool (pool_bytes of HBM) is allocated here with PyTorch and
    handed to the server, which takes every device byte it uses from it.
    """

    def __init__(self, pool_bytes: int, slots: int = 8, device: int = 0, admit_timeout_ms: int = 10000,
                 grid_div: int = 0, tile_max: int = 0, high_slots: int = 0, small_edges: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libtc needs a CUDA GPU; none is available (there is no CPU fallback)")
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        h = vp()
        cfg = TcServeConfig(slots, admit_timeout_ms, grid_div, tile_max, high_slots, small_edges)
        st = self.lib.tc_serve_create(device, ctypes.byref(cfg), _ptr(self.pool), self.pool.numel(), ctypes.byref(h))
        if st != 0:
            raise TcError(st, "tc_serve_create failed")
        self.handle = h
        self.edges_of = {}

    def _check(self, st: int):
        if st != 0:
            raise TcError(st, self.lib.tc_serve_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tc_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_graph(self, n: int, edges) -> int:
        import numpy as np
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        gid = i64(0)
        self._check(self.lib.tc_serve_add_graph(self.handle, int(n), len(e), e.ctypes.data_as(vp) if len(e) else None,
                                                ctypes.byref(gid)))
        self.edges_of[int(gid.value)] = len(e)
        return int(gid.value)

    def remove_graph(self, graph_id: int):
        self._check(self.lib.tc_serve_remove_graph(self.handle, int(graph_id)))

    def submit(self, graph_id: int, kind: int) -> int:
        t = i64(0)
        self._check(self.lib.tc_serve_submit(self.handle, int(graph_id), int(kind), ctypes.byref(t)))
        return int(t.value)

    def _result(self, ticket: int, r: TcResult, copy: bool) -> ServeResult:
        out = ServeResult(ticket, r.status, r.kind, r.graph_id, int(r.triangles), r.queue_ms, r.latency_ms)
        if copy and r.status == 0:
            if r.tv:
                out.tv = torch.as_tensor(_DeviceArray(r.tv, (r.n,), "<i8"), device=self.device).clone()
                out.cc = torch.as_tensor(_DeviceArray(r.cc, (r.n,), "<f8"), device=self.device).clone()
            if r.tri and r.triangles:
                out.tri = torch.as_tensor(_DeviceArray(r.tri, (int(r.triangles), 3), "<i4"),
                                          device=self.device).clone()
            elif r.kind == LIST:
                out.tri = torch.empty((0, 3), dtype=torch.int32, device=self.device)
            # the clones are queued on PyTorch's stream: they must have read the
            # server's memory before the ticket (and that memory) is released
            torch.cuda.current_stream(self.device).synchronize()
        return out

    def wait(self, ticket: int, timeout_ms: int = 60000, copy: bool = True, release: bool = True) -> ServeResult:
        r = TcResult()
        st = self.lib.tc_serve_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(r))
        if st == 7:
            raise TcError(st, "request still running")
        res = self._result(ticket, r, copy)
        if release:
            self._check(self.lib.tc_serve_release(self.handle, int(ticket)))
        return res

    def poll(self, ticket: int):
        r = TcResult()
        st = self.lib.tc_serve_poll(self.handle, int(ticket), ctypes.byref(r))
        return st, (self._result(ticket, r, False) if st != 9 else None)

    def release(self, ticket: int):
        self._check(self.lib.tc_serve_release(self.handle, int(ticket)))

    def stats(self) -> dict:
        s = TcServeStats()
        self._check(self.lib.tc_serve_stats(self.handle, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in TcServeStats._fields_}


def graph_from_csr(offsets: torch.Tensor, cols: torch.Tensor, deg=None, dhat=None) -> Graph:
    """Wrap an existing oriented CSR (device tensors) as a Graph."""
    n = int(offsets.numel()) - 1
    return Graph(n, int(cols.numel()), offsets, cols, deg, dhat)

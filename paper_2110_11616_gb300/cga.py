"""Thin Python binding of libcga (include/cga.h): argument marshalling only.

Every step of the hot path runs in the CUDA kernels of libcga.so; this module
passes torch device pointers, the current CUDA stream and a torch-backed
allocator through the C ABI.  There is no CPU fallback: if libcga.so is missing
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcga.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_NONFINITE = -2
ERR_GRID_MISMATCH = -3
ERR_OOM = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_INTERNAL = -7
ERR_CAPACITY = -8
NOALLOC_MAX_QUERIES = 1 << 20
MAX_POINTS = (1 << 30) - 1
PLANES = {"xy": 0, "xz": 1, "yz": 2}

# Every symbol include/cga.h declares.
EXPORTS = (
    "cga_grid_from_box", "cga_build", "cga_merge", "cga_project", "cga_nn_query",
    "cga_decode", "cga_info", "cga_view", "cga2d_info", "cga2d_view", "cga_download",
    "cga2d_download", "cga_free", "cga2d_free", "cga_strerror", "cga_kernel_launches",
    "cga_build_batch", "cga_merge_batch", "cga_project_batch", "cga_nn_query_batch",
    "cga_pipeline_create", "cga_pipeline_run", "cga_pipeline_run_graph", "cga_pipeline_view",
    "cga_pipeline_view_xy", "cga_pipeline_free", "cga_nn_query_noalloc",
    "cga_server_create", "cga_server_submit", "cga_server_poll", "cga_server_drain",
    "cga_server_free", "cga_now_ns", "cga_nn_sort_queries", "cga_nn_query_ordered",
    "cga_nn_prepare", "cga_nn_prepare_levels", "cga_nn_autotune", "cga_nn_autotune_for",
    "cga_tuning_set", "cga_tuning_get", "cga_autotune", "cga_pipeline_autotune",
    "cga_build_values", "cga_merge_values", "cga_values", "cga_perspective",
    "cga_radius_count", "cga_radius_fill", "cga_knn",
    "cga_kmeans", "cga_motion_vectors", "cga_reconstruct", "cga_nn_query_voxels", "cga_lookup",
    "cga_garrays_x", "cga_garrays_lookup", "cga_residual",
    "cga_selftest_wait_timeout",
)


class CgaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = _lib_strerror(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_uint32), ("scale", ctypes.c_float),
                ("offset", ctypes.c_float * 3)]

    def __repr__(self):
        return f"Grid(bits={self.bits}, scale={self.scale}, offset={tuple(self.offset)})"


class Allocator(ctypes.Structure):
    _fields_ = [
        ("ctx", ctypes.c_void_p),
        ("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.c_void_p)),
        ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)),
    ]


class Sizes(ctypes.Structure):
    _fields_ = [("h", ctypes.c_uint64), ("g", ctypes.c_uint64), ("u", ctypes.c_uint64),
                ("bytes", ctypes.c_uint64), ("capacity", ctypes.c_uint64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libcga.so; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libcga.so not found at {path}: build it with "
                           "__graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.cga_grid_from_box.argtypes = [P, ctypes.c_float, U32, ctypes.POINTER(Grid)]
    lib.cga_build.argtypes = [P, U64, ctypes.POINTER(Grid), P, P, P, PP]
    lib.cga_merge.argtypes = [P, P, P, P, PP]
    lib.cga_project.argtypes = [P, I, P, P, PP]
    lib.cga_nn_query.argtypes = [P, P, U64, P, P, P]
    lib.cga_decode.argtypes = [P, P, P]
    lib.cga_info.argtypes = [P, ctypes.POINTER(Sizes)]
    lib.cga2d_info.argtypes = [P, ctypes.POINTER(U64), ctypes.POINTER(U64)]
    lib.cga_download.argtypes = [P, P, P, P, P, P]
    lib.cga2d_download.argtypes = [P, P, P, P]
    lib.cga_free.argtypes = [P]
    lib.cga_free.restype = None
    lib.cga2d_free.argtypes = [P]
    lib.cga2d_free.restype = None
    lib.cga_kernel_launches.argtypes = []
    lib.cga_kernel_launches.restype = ctypes.c_uint64
    lib.cga_strerror.argtypes = [I]
    lib.cga_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _lib_strerror(code):
    try:
        return load().cga_strerror(code).decode()
    except Exception:  # library missing: still describe the code
        return f"error {code}"


def _check(rc, what=""):
    if rc != OK:
        raise CgaError(rc, what)


# ------------------------------------------------------------------ allocator
def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libcga needs a CUDA GPU; none is available")
    return torch


@ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
def _torch_alloc(ctx, nbytes, stream):
    try:
        import torch
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
    except Exception:
        return None


@ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
def _torch_free(ctx, ptr, stream):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:  # interpreter shutdown: the process is exiting anyway
        pass


TORCH_ALLOCATOR = Allocator(None, _torch_alloc, _torch_free)


def _alloc_arg(allocator):
    if allocator == "torch":
        return ctypes.byref(TORCH_ALLOCATOR)
    if allocator is None:
        return None
    return ctypes.byref(allocator)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------- grid
def grid_from_box(lo, extent: float, bits: int) -> Grid:
    lo_a = np.ascontiguousarray(np.asarray(lo, np.float32).reshape(3))
    g = Grid()
    _check(load().cga_grid_from_box(lo_a.ctypes.data_as(ctypes.c_void_p), float(extent), int(bits),
                                    ctypes.byref(g)), "cga_grid_from_box")
    return g


def make_grid(bits: int, scale: float, offset) -> Grid:
    g = Grid()
    g.bits = bits
    g.scale = scale
    for a in range(3):
        g.offset[a] = offset[a]
    return g


# -------------------------------------------------------------------- handles
class Cga:
    """Owning wrapper of a cga_t*; frees it (stream-ordered) when collected."""

    def __init__(self, ptr, grid: Grid, keep=()):
        self.ptr = ptr
        self.grid = grid
        self._keep = keep

    def info(self) -> dict:
        s = Sizes()
        _check(load().cga_info(self.ptr, ctypes.byref(s)), "cga_info")
        return {"h": s.h, "g": s.g, "u": s.u, "bytes": s.bytes, "capacity": s.capacity}

    def status(self) -> int:
        s = Sizes()
        return load().cga_info(self.ptr, ctypes.byref(s))

    def download(self) -> dict:
        s = Sizes()
        rc = load().cga_info(self.ptr, ctypes.byref(s))
        _check(rc, "cga_info")
        out = {"X_index": np.zeros(s.h, np.uint16), "X_pointer": np.zeros(s.h + 1, np.uint32),
               "Y_index": np.zeros(s.g, np.uint16), "Y_pointer": np.zeros(s.g + 1, np.uint32),
               "Z_index": np.zeros(s.u, np.uint16)}
        args = [out[k].ctypes.data_as(ctypes.c_void_p) for k in
                ("X_index", "X_pointer", "Y_index", "Y_pointer", "Z_index")]
        _check(load().cga_download(self.ptr, *args), "cga_download")
        return out

    def free(self):
        if self.ptr:
            load().cga_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Cga2d:
    def __init__(self, ptr, bits: int, plane: int):
        self.ptr = ptr
        self.bits = bits
        self.plane = plane

    def info(self) -> dict:
        h, g = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().cga2d_info(self.ptr, ctypes.byref(h), ctypes.byref(g)), "cga2d_info")
        return {"h": h.value, "g": g.value}

    def download(self) -> dict:
        i = self.info()
        out = {"U_index": np.zeros(i["h"], np.uint16), "U_pointer": np.zeros(i["h"] + 1, np.uint32),
               "V_index": np.zeros(i["g"], np.uint16)}
        args = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("U_index", "U_pointer", "V_index")]
        _check(load().cga2d_download(self.ptr, *args), "cga2d_download")
        return out

    def free(self):
        if self.ptr:
            load().cga2d_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _dev_f32(t, what):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{what}: expected a contiguous float32 CUDA tensor")
    return t


# ----------------------------------------------------------------- operations
def cga_build(points, grid: Grid, xform=None, stream=None, allocator="torch") -> Cga:
    """points: (n, 3) float32 CUDA tensor; xform: None or 12 floats (R row-major, t)."""
    _dev_f32(points, "cga_build")
    n = points.numel() // 3
    x = None
    if xform is not None:
        x = np.ascontiguousarray(np.asarray(xform, np.float32).reshape(12))
    out = ctypes.c_void_p()
    _check(load().cga_build(ctypes.c_void_p(points.data_ptr()), n, ctypes.byref(grid),
                            None if x is None else x.ctypes.data_as(ctypes.c_void_p),
                            _alloc_arg(allocator), _stream(stream), ctypes.byref(out)),
           "cga_build")
    return Cga(out, grid)


def cga_merge(a: Cga, b: Cga, stream=None, allocator="torch") -> Cga:
    out = ctypes.c_void_p()
    _check(load().cga_merge(a.ptr, b.ptr, _alloc_arg(allocator), _stream(stream),
                            ctypes.byref(out)), "cga_merge")
    return Cga(out, a.grid)


def cga_project(a: Cga, plane, stream=None, allocator="torch") -> Cga2d:
    p = PLANES[plane] if isinstance(plane, str) else int(plane)
    out = ctypes.c_void_p()
    _check(load().cga_project(a.ptr, p, _alloc_arg(allocator), _stream(stream),
                              ctypes.byref(out)), "cga_project")
    return Cga2d(out, a.grid.bits, p)


def cga_nn_query(a: Cga, queries, idx=None, dist2=None, stream=None):
    """queries: (m, 3) float32 CUDA tensor.  Returns (idx int32 tensor holding
    uint32 values, dist2 int64 tensor holding uint64 values)."""
    torch = _torch()
    _dev_f32(queries, "cga_nn_query")
    m = queries.numel() // 3
    if idx is None:
        idx = torch.empty(m, dtype=torch.int32, device=queries.device)
    if dist2 is None:
        dist2 = torch.empty(m, dtype=torch.int64, device=queries.device)
    _check(load().cga_nn_query(a.ptr, ctypes.c_void_p(queries.data_ptr()), m,
                               ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(dist2.data_ptr()),
                               _stream(stream)), "cga_nn_query")
    return idx, dist2


def cga_decode(a: Cga, out=None, stream=None):
    """(u, 3) int32 CUDA tensor of (x, y, z) voxels in CGA order.  With `out`
    given (>= 3u int32 entries) no size query (and no host wait) happens."""
    torch = _torch()
    if out is None:
        u = a.info()["u"]
        out = torch.empty((u, 3), dtype=torch.int32, device="cuda")
        if u == 0:
            return out
    _check(load().cga_decode(a.ptr, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "cga_decode")
    return out


def kernel_launches() -> int:
    return int(load().cga_kernel_launches())


# -------------------------------------------------------------------- batches
class Cloud(ctypes.Structure):
    _fields_ = [("d_xyz", ctypes.c_void_p), ("n", ctypes.c_uint64), ("grid", Grid),
                ("h_xform12", ctypes.c_void_p)]


class Queries(ctypes.Structure):
    _fields_ = [("d_q", ctypes.c_void_p), ("m", ctypes.c_uint64), ("d_idx", ctypes.c_void_p),
                ("d_dist2", ctypes.c_void_p)]


class PipelineItem(ctypes.Structure):
    _fields_ = [("d_xyz", ctypes.c_void_p), ("n", ctypes.c_uint64), ("grid", Grid),
                ("xform12", ctypes.c_float * 12), ("d_q", ctypes.c_void_p), ("m", ctypes.c_uint64),
                ("d_idx", ctypes.c_void_p), ("d_dist2", ctypes.c_void_p)]


def _setup_batch(lib):
    if getattr(lib, "_batch_ready", False):
        return
    P, U32, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int
    lib.cga_build_batch.argtypes = [P, U32, P, P, P]
    lib.cga_merge_batch.argtypes = [P, P, U32, P, P, P]
    lib.cga_project_batch.argtypes = [P, P, U32, P, P, P]
    lib.cga_nn_query_batch.argtypes = [P, P, U32, P, P]
    lib.cga_pipeline_create.argtypes = [P, U32, P, P, ctypes.POINTER(ctypes.c_void_p)]
    lib.cga_pipeline_run.argtypes = [P, P]
    lib.cga_pipeline_run_graph.argtypes = [P, P]
    lib.cga_pipeline_view.argtypes = [P, U32, I, ctypes.POINTER(ctypes.c_void_p)]
    lib.cga_pipeline_view_xy.argtypes = [P, U32, ctypes.POINTER(ctypes.c_void_p)]
    lib.cga_pipeline_free.argtypes = [P]
    lib.cga_pipeline_free.restype = None
    lib._batch_ready = True


def _ptr_array(handles):
    arr = (ctypes.c_void_p * max(len(handles), 1))()
    for i, h in enumerate(handles):
        arr[i] = h.ptr if isinstance(h, (Cga, Cga2d)) else h
    return arr


def cga_build_batch(points_list, grids, xforms=None, stream=None, allocator="torch"):
    """One launch set for many clouds.  points_list: float32 CUDA tensors (n_i, 3);
    grids: one Grid or a list; xforms: None or a list of None / 12 floats."""
    lib = load()
    _setup_batch(lib)
    k = len(points_list)
    grids = grids if isinstance(grids, (list, tuple)) else [grids] * k
    xforms = xforms if xforms is not None else [None] * k
    clouds = (Cloud * max(k, 1))()
    keep = []
    for i, (pts, g, x) in enumerate(zip(points_list, grids, xforms)):
        _dev_f32(pts, "cga_build_batch")
        clouds[i].d_xyz = pts.data_ptr()
        clouds[i].n = pts.numel() // 3
        clouds[i].grid = g
        if x is not None:
            xa = np.ascontiguousarray(np.asarray(x, np.float32).reshape(12))
            keep.append(xa)
            clouds[i].h_xform12 = xa.ctypes.data
    out = (ctypes.c_void_p * max(k, 1))()
    _check(lib.cga_build_batch(clouds, k, _alloc_arg(allocator), _stream(stream), out),
           "cga_build_batch")
    return [Cga(ctypes.c_void_p(out[i]), grids[i]) for i in range(k)]


def cga_merge_batch(a_list, b_list, stream=None, allocator="torch"):
    lib = load()
    _setup_batch(lib)
    k = len(a_list)
    out = (ctypes.c_void_p * max(k, 1))()
    _check(lib.cga_merge_batch(_ptr_array(a_list), _ptr_array(b_list), k, _alloc_arg(allocator),
                               _stream(stream), out), "cga_merge_batch")
    return [Cga(ctypes.c_void_p(out[i]), a_list[i].grid) for i in range(k)]


def cga_project_batch(a_list, planes, stream=None, allocator="torch"):
    lib = load()
    _setup_batch(lib)
    k = len(a_list)
    pl = [PLANES[p] if isinstance(p, str) else int(p) for p in
          (planes if isinstance(planes, (list, tuple)) else [planes] * k)]
    parr = (ctypes.c_int * max(k, 1))(*pl)
    out = (ctypes.c_void_p * max(k, 1))()
    _check(lib.cga_project_batch(_ptr_array(a_list), parr, k, _alloc_arg(allocator),
                                 _stream(stream), out), "cga_project_batch")
    return [Cga2d(ctypes.c_void_p(out[i]), a_list[i].grid.bits, pl[i]) for i in range(k)]


def cga_nn_query_batch(a_list, queries_list, stream=None, allocator="torch"):
    """Returns [(idx int32, dist2 int64)] per item."""
    torch = _torch()
    lib = load()
    _setup_batch(lib)
    k = len(a_list)
    qs = (Queries * max(k, 1))()
    res = []
    for i, q in enumerate(queries_list):
        _dev_f32(q, "cga_nn_query_batch")
        m = q.numel() // 3
        idx = torch.empty(m, dtype=torch.int32, device=q.device)
        d2 = torch.empty(m, dtype=torch.int64, device=q.device)
        qs[i].d_q, qs[i].m, qs[i].d_idx, qs[i].d_dist2 = q.data_ptr(), m, idx.data_ptr(), d2.data_ptr()
        res.append((idx, d2))
    _check(lib.cga_nn_query_batch(_ptr_array(a_list), qs, k, _alloc_arg(allocator),
                                  _stream(stream)), "cga_nn_query_batch")
    return res


class _View(Cga):
    """Non-owning handle of a pipeline result (freeing it is a no-op)."""

    def free(self):
        self.ptr = None


class _View2d(Cga2d):
    def free(self):
        self.ptr = None


def _pipeline_items(points_list, grids, xforms, queries_list):
    """cga_pipeline_item array plus the NN output tensors of every item."""
    torch = _torch()
    k = len(points_list)
    grids = grids if isinstance(grids, (list, tuple)) else [grids] * k
    items = (PipelineItem * k)()
    idxs, d2s = [], []
    for i in range(k):
        pts, q = points_list[i], queries_list[i]
        _dev_f32(pts, "Pipeline")
        it = items[i]
        it.d_xyz, it.n, it.grid = pts.data_ptr(), pts.numel() // 3, grids[i]
        x = np.asarray(xforms[i], np.float32).reshape(12)
        for j in range(12):
            it.xform12[j] = float(x[j])
        m = 0 if q is None else q.numel() // 3
        idx = torch.empty(m, dtype=torch.int32, device="cuda")
        d2 = torch.empty(m, dtype=torch.int64, device="cuda")
        if m:
            _dev_f32(q, "Pipeline")
            it.d_q, it.m, it.d_idx, it.d_dist2 = q.data_ptr(), m, idx.data_ptr(), d2.data_ptr()
        idxs.append(idx)
        d2s.append(d2)
    return items, list(grids), idxs, d2s


def pipeline_autotune(points_list, grids, xforms, queries_list, stream=None):
    """cga_pipeline_autotune: time the graph-replayed pipeline of these items
    under every launch shape and keep the fastest for their (largest bits,
    largest n).  Returns (shape, {"sort": {...}, "merge": {...}})."""
    lib = load()
    P = ctypes.c_void_p
    lib.cga_pipeline_autotune.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(Tuning), P, P]
    items, grids, _, _ = _pipeline_items(points_list, grids, xforms, queries_list)
    t = Tuning()
    times = (ctypes.c_float * (len(SORT_CANDIDATES) + len(MERGE_CANDIDATES)))()
    _check(lib.cga_pipeline_autotune(items, len(items), ctypes.byref(t), times, _stream(stream)),
           "cga_pipeline_autotune")
    key = (max(g.bits for g in grids), _bucket(max(it.n for it in items)))
    _tuned[key] = t.as_dict()
    k = len(SORT_CANDIDATES)
    return t.as_dict(), {"sort": {c: float(v) for c, v in zip(SORT_CANDIDATES, times[:k])},
                         "merge": {c: float(v) for c, v in zip(MERGE_CANDIDATES, times[k:])}}


class Pipeline:
    """Pre-planned batch: build + transformed twin + merge + xy projection + NN
    for many clouds, queued by run() or replayed from a CUDA graph by run_graph()."""

    def __init__(self, points_list, grids, xforms, queries_list, stream=None, allocator="torch"):
        lib = load()
        _setup_batch(lib)
        items, self.grids, self.idx, self.dist2 = _pipeline_items(points_list, grids, xforms,
                                                                  queries_list)
        self._keep = (points_list, queries_list)
        self.ptr = ctypes.c_void_p()
        _check(lib.cga_pipeline_create(items, len(items), _alloc_arg(allocator), _stream(stream),
                                       ctypes.byref(self.ptr)), "cga_pipeline_create")
        self.count = len(items)

    def run(self, stream=None):
        _check(load().cga_pipeline_run(self.ptr, _stream(stream)), "cga_pipeline_run")

    def run_graph(self, stream=None):
        _check(load().cga_pipeline_run_graph(self.ptr, _stream(stream)), "cga_pipeline_run_graph")

    def view(self, i: int, which: str) -> Cga:
        w = {"cloud": 0, "twin": 1, "merged": 2}[which]
        out = ctypes.c_void_p()
        _check(load().cga_pipeline_view(self.ptr, i, w, ctypes.byref(out)), "cga_pipeline_view")
        return _View(out, self.grids[i])

    def view_xy(self, i: int) -> Cga2d:
        out = ctypes.c_void_p()
        _check(load().cga_pipeline_view_xy(self.ptr, i, ctypes.byref(out)), "cga_pipeline_view_xy")
        return _View2d(out, self.grids[i].bits, 0)

    def free(self):
        if self.ptr:
            load().cga_pipeline_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- served loop
REQ_NN = 0
REQ_MERGE_PROJECT = 1


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("plane", ctypes.c_int32), ("d_q", ctypes.c_void_p), ("m", ctypes.c_uint64),
                ("d_idx", ctypes.c_void_p), ("d_dist2", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_uint64), ("t_start_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64), ("merged", ctypes.c_void_p),
                ("projected", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32)]


def now_ns() -> int:
    lib = load()
    lib.cga_now_ns.restype = ctypes.c_uint64
    return int(lib.cga_now_ns())


class Server:
    """Continuous-batching request loop over a pool of resident CGAs."""

    def __init__(self, pool, memory_budget: int, slots: int = 4, max_batch: int = 64,
                 allocator=None):
        lib = load()
        P = ctypes.c_void_p
        lib.cga_server_create.argtypes = [P, ctypes.c_uint32, P, P, ctypes.POINTER(P)]
        lib.cga_server_submit.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64)]
        lib.cga_server_poll.argtypes = [P, P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
        lib.cga_server_drain.argtypes = [P]
        lib.cga_server_free.argtypes = [P]
        lib.cga_server_free.restype = None
        self.pool = list(pool)
        cfg = ServerConfig(memory_budget, slots, max_batch)
        self.ptr = ctypes.c_void_p()
        _check(lib.cga_server_create(_ptr_array(self.pool), len(self.pool), ctypes.byref(cfg),
                                     _alloc_arg(allocator), ctypes.byref(self.ptr)),
               "cga_server_create")
        self._keep = {}

    def submit_nn(self, a: int, queries, idx, dist2, keep=None) -> int:
        r = Request(REQ_NN, a, 0, 0, queries.data_ptr(), queries.numel() // 3, idx.data_ptr(),
                    dist2.data_ptr())
        t = ctypes.c_uint64()
        _check(load().cga_server_submit(self.ptr, ctypes.byref(r), ctypes.byref(t)),
               "cga_server_submit")
        self._keep[t.value] = (queries, idx, dist2, keep)
        return t.value

    def submit_merge_project(self, a: int, b: int, plane="xy") -> int:
        p = PLANES[plane] if isinstance(plane, str) else int(plane)
        r = Request(REQ_MERGE_PROJECT, a, b, p, None, 0, None, None)
        t = ctypes.c_uint64()
        _check(load().cga_server_submit(self.ptr, ctypes.byref(r), ctypes.byref(t)),
               "cga_server_submit")
        return t.value

    def poll(self, max_n: int = 4096):
        arr = (Completion * max_n)()
        n = ctypes.c_uint32()
        _check(load().cga_server_poll(self.ptr, arr, max_n, ctypes.byref(n)), "cga_server_poll")
        out = []
        for i in range(n.value):
            c = arr[i]
            d = {"ticket": c.ticket, "status": c.status, "t_submit_ns": c.t_submit_ns,
                 "t_start_ns": c.t_start_ns, "t_done_ns": c.t_done_ns,
                 "merged": Cga(ctypes.c_void_p(c.merged), self.pool[0].grid) if c.merged else None,
                 "projected": Cga2d(ctypes.c_void_p(c.projected), 0, 0) if c.projected else None}
            self._keep.pop(c.ticket, None)
            out.append(d)
        return out

    def drain(self):
        _check(load().cga_server_drain(self.ptr), "cga_server_drain")

    def free(self):
        if self.ptr:
            load().cga_server_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cga_nn_sort_queries(a: Cga, queries, order=None, stream=None):
    """Sorted (morton << 32 | index) keys of the queries, as an int64 tensor."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_nn_sort_queries.argtypes = [P, P, ctypes.c_uint64, P, P]
    m = queries.numel() // 3
    if order is None:
        order = torch.empty(m, dtype=torch.int64, device=queries.device)
    _check(lib.cga_nn_sort_queries(a.ptr, P(queries.data_ptr()), m, P(order.data_ptr()),
                                   _stream(stream)), "cga_nn_sort_queries")
    return order


def cga_nn_query_ordered(a: Cga, queries, order, idx, dist2, stream=None):
    lib = load()
    P = ctypes.c_void_p
    lib.cga_nn_query_ordered.argtypes = [P, P, ctypes.c_uint64, P, P, P, P]
    m = queries.numel() // 3
    _check(lib.cga_nn_query_ordered(a.ptr, P(queries.data_ptr()), m,
                                    None if order is None else P(order.data_ptr()),
                                    P(idx.data_ptr()), P(dist2.data_ptr()), _stream(stream)),
           "cga_nn_query_ordered")
    return idx, dist2


NN_MAX_LEVELS = 2
NN_TREE = 0xFFFFFFFF  # shifts (NN_TREE,): the occupancy tree instead of coarse levels
# cga_nn_autotune's candidates, in the order of its timings (coarse shifts)
NN_AUTOTUNE_CANDIDATES = ((), (2,), (3,), (4,), (5,), (2, 5), (3, 6), (3, 7), (4, 8), (NN_TREE,))


def cga_nn_prepare(a: Cga, shifts=(), stream=None):
    """Build the coarse levels (cells of 2^shift voxels, finest first) used by
    NN search; an int is one level, 0 or () none (x directory only),
    (NN_TREE,) or "tree" the occupancy tree."""
    if isinstance(shifts, str):
        if shifts != "tree":
            raise ValueError(f"cga_nn_prepare: unknown strategy {shifts!r}")
        shifts = (NN_TREE,)
    if isinstance(shifts, int):
        shifts = () if shifts == 0 else (shifts,)
    shifts = tuple(int(v) for v in shifts)
    lib = load()
    lib.cga_nn_prepare_levels.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32),
                                          ctypes.c_uint32, ctypes.c_void_p]
    arr = (ctypes.c_uint32 * max(1, len(shifts)))(*shifts)
    _check(lib.cga_nn_prepare_levels(a.ptr, arr, len(shifts), _stream(stream)),
           "cga_nn_prepare_levels")
    return a


def cga_nn_autotune(a: Cga, sample_queries, stream=None, queries_per_prepare: int = 0):
    """Measure the NN strategies on a query sample; keep the fastest on `a`.
    With queries_per_prepare > 0 (a CGA prepared once per that many queries)
    a strategy's cost is its preparation time plus the sample's search time
    scaled to that many queries (cga_nn_autotune_for).  Returns (shifts,
    {shifts: ms}) with shifts a tuple of coarse shifts."""
    lib = load()
    P = ctypes.c_void_p
    lib.cga_nn_autotune_for.argtypes = [P, P, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint32), P, P]
    _dev_f32(sample_queries, "cga_nn_autotune")
    chosen = (ctypes.c_uint32 * NN_MAX_LEVELS)()
    times = (ctypes.c_float * len(NN_AUTOTUNE_CANDIDATES))()
    _check(lib.cga_nn_autotune_for(a.ptr, P(sample_queries.data_ptr()),
                                   sample_queries.numel() // 3, int(queries_per_prepare),
                                   chosen, times, _stream(stream)), "cga_nn_autotune")
    shifts = tuple(int(v) for v in chosen if v != 0)
    return shifts, {c: float(t) for c, t in zip(NN_AUTOTUNE_CANDIDATES, times) if t >= 0}


# ------------------------------------------------------------ radius search
def cga_radius(a: Cga, queries, r2: int, stream=None):
    """Every stored voxel within squared distance r2 of each query: (offsets (m+1)
    int64, idx int32 holding uint32, dist2 int64), query j's at [offsets[j],
    offsets[j+1]) in ascending CGA index.  Waits once for the total."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_radius_count.argtypes = [P, P, ctypes.c_uint64, ctypes.c_uint64, P, P]
    lib.cga_radius_fill.argtypes = [P, P, ctypes.c_uint64, ctypes.c_uint64, P, P, P, P]
    _dev_f32(queries, "cga_radius")
    m = queries.numel() // 3
    offsets = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    _check(lib.cga_radius_count(a.ptr, P(queries.data_ptr()), m, int(r2), P(offsets.data_ptr()),
                                _stream(stream)), "cga_radius_count")
    total = int(offsets[m].item())
    idx = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    d2 = torch.empty(max(total, 1), dtype=torch.int64, device="cuda")
    _check(lib.cga_radius_fill(a.ptr, P(queries.data_ptr()), m, int(r2), P(offsets.data_ptr()),
                               P(idx.data_ptr()), P(d2.data_ptr()), _stream(stream)),
           "cga_radius_fill")
    return offsets, idx[:total], d2[:total]


def cga_knn(a: Cga, queries, k: int, stream=None):
    """The k nearest stored voxels of each query: (idx (m, k) int32 holding uint32,
    dist2 (m, k) int64 holding uint64), ascending by (distance^2, key)."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_knn.argtypes = [P, P, ctypes.c_uint64, ctypes.c_uint32, P, P, P]
    _dev_f32(queries, "cga_knn")
    m = queries.numel() // 3
    idx = torch.empty((m, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((m, k), dtype=torch.int64, device="cuda")
    _check(lib.cga_knn(a.ptr, P(queries.data_ptr()), m, k, P(idx.data_ptr()), P(d2.data_ptr()),
                       _stream(stream)), "cga_knn")
    return idx, d2


# ------------------------------------------------------ perspective projection
def cga_perspective(a: Cga, eye, cos_t: float, sin_t: float, D: float, W: int, H: int,
                    stream=None):
    """Perspective z-buffer image of a (Eq. 5-6): (index (H, W) int32 tensor holding
    uint32 values, depth (H, W) float32 tensor)."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_perspective.argtypes = [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_uint32, ctypes.c_uint32, P, P, P]
    e = np.ascontiguousarray(np.asarray(eye, np.float32).reshape(3))
    idx = torch.empty((H, W), dtype=torch.int32, device="cuda")
    dep = torch.empty((H, W), dtype=torch.float32, device="cuda")
    _check(lib.cga_perspective(a.ptr, e.ctypes.data_as(P), float(cos_t), float(sin_t), float(D),
                               W, H, P(idx.data_ptr()), P(dep.data_ptr()), _stream(stream)),
           "cga_perspective")
    return idx, dep


# ------------------------------------------------------------- value array
VALUE_POLICIES = {"average": 0, "first": 1}
MERGE_POLICIES = {"base": 0, "average": 1}


class _DeviceBytes:
    """A borrowed device byte range as a CUDA array (for torch.as_tensor)."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "|u1",
                                         "data": (ptr, False), "version": 3, "strides": None}


def cga_values(a: Cga):
    """A copy of a's Value array as a (u, channels) uint8 CUDA tensor, or None."""
    torch = _torch()
    lib = load()
    lib.cga_values.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                               ctypes.POINTER(ctypes.c_uint32)]
    ptr, ch = ctypes.c_void_p(), ctypes.c_uint32()
    _check(lib.cga_values(a.ptr, ctypes.byref(ptr), ctypes.byref(ch)), "cga_values")
    if not ptr.value or ch.value == 0:
        return None
    u = a.info()["u"]
    if u == 0:
        return torch.zeros((0, ch.value), dtype=torch.uint8, device="cuda")
    return torch.as_tensor(_DeviceBytes(ptr.value, (u, ch.value)), device="cuda").clone()


def cga_build_values(points, attrs, grid: Grid, xform=None, policy="average", stream=None,
                     allocator="torch") -> Cga:
    """cga_build plus per-voxel uint8 attributes: attrs is an (n, channels)
    uint8 CUDA tensor aligned with points."""
    lib = load()
    P = ctypes.c_void_p
    lib.cga_build_values.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.POINTER(Grid), P, ctypes.c_int, P, P,
                                     ctypes.POINTER(ctypes.c_void_p)]
    _dev_f32(points, "cga_build_values")
    n = points.numel() // 3
    if not attrs.is_cuda or attrs.dtype != _torch().uint8 or not attrs.is_contiguous():
        raise ValueError("cga_build_values: attrs must be a contiguous uint8 CUDA tensor")
    ch = attrs.numel() // max(n, 1) if n else (attrs.shape[-1] if attrs.dim() > 1 else 1)
    if n and attrs.numel() != n * ch:
        raise ValueError("cga_build_values: one attribute row per point")
    x = None
    if xform is not None:
        x = np.ascontiguousarray(np.asarray(xform, np.float32).reshape(12))
    out = ctypes.c_void_p()
    _check(lib.cga_build_values(P(points.data_ptr()), P(attrs.data_ptr()), ch, n,
                                ctypes.byref(grid),
                                x.ctypes.data_as(P) if x is not None else None,
                                VALUE_POLICIES[policy], _alloc_arg(allocator), _stream(stream),
                                ctypes.byref(out)), "cga_build_values")
    return Cga(out, grid)


def cga_merge_values(a: Cga, b: Cga, policy="base", stream=None, allocator="torch") -> Cga:
    """cga_merge plus the Value array (a is the base)."""
    lib = load()
    P = ctypes.c_void_p
    lib.cga_merge_values.argtypes = [P, P, ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_void_p)]
    out = ctypes.c_void_p()
    _check(lib.cga_merge_values(a.ptr, b.ptr, MERGE_POLICIES[policy], _alloc_arg(allocator),
                                _stream(stream), ctypes.byref(out)), "cga_merge_values")
    return Cga(out, a.grid)


# -------------------------------------------------------- launch-shape tuning
class Tuning(ctypes.Structure):
    _fields_ = [("radix_bits", ctypes.c_uint32), ("sort_threads", ctypes.c_uint32),
                ("merge_half", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {"radix_bits": self.radix_bits, "sort_threads": self.sort_threads,
                "merge_half": self.merge_half}


# cga_autotune's candidates, in the order of its timings
SORT_CANDIDATES = ((8, 256), (8, 512), (9, 512))  # (radix_bits, sort_threads)
MERGE_CANDIDATES = (512, 1024, 2048)               # merge_half
DEFAULT_TUNING = {"radix_bits": 8, "sort_threads": 512, "merge_half": 2048}
_tuned: dict = {}  # (bits, bit length of n) -> shape set through this module


def _bucket(n: int) -> int:
    return int(n).bit_length()


def tuning_get(bits: int, n: int) -> dict:
    """The launch shape a sort or merge with (grid bits, n elements) uses now."""
    lib = load()
    lib.cga_tuning_get.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(Tuning)]
    t = Tuning()
    _check(lib.cga_tuning_get(bits, n, ctypes.byref(t)), "cga_tuning_get")
    return t.as_dict()


def tuning_set(bits: int, n: int, shape=None):
    """Set the table entry for (bits, n's bit length); None restores the default."""
    lib = load()
    lib.cga_tuning_set.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(Tuning)]
    if shape is None:
        _check(lib.cga_tuning_set(bits, n, None), "cga_tuning_set")
        _tuned.pop((bits, _bucket(n)), None)
        return
    t = Tuning(shape["radix_bits"], shape["sort_threads"], shape["merge_half"])
    _check(lib.cga_tuning_set(bits, n, ctypes.byref(t)), "cga_tuning_set")
    _tuned[(bits, _bucket(n))] = t.as_dict()


def cga_autotune(points, grid: Grid, stream=None):
    """Time every sort and merge launch shape on this cloud; keep the fastest
    for (grid.bits, len(points)).  Returns (shape, {"sort": {...}, "merge": {...}})."""
    lib = load()
    P = ctypes.c_void_p
    lib.cga_autotune.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Grid), ctypes.POINTER(Tuning),
                                 P, P]
    _dev_f32(points, "cga_autotune")
    n = points.numel() // 3
    t = Tuning()
    times = (ctypes.c_float * (len(SORT_CANDIDATES) + len(MERGE_CANDIDATES)))()
    _check(lib.cga_autotune(P(points.data_ptr()), n, ctypes.byref(grid), ctypes.byref(t), times,
                            _stream(stream)), "cga_autotune")
    _tuned[(grid.bits, _bucket(n))] = t.as_dict()
    k = len(SORT_CANDIDATES)
    return t.as_dict(), {"sort": {c: float(v) for c, v in zip(SORT_CANDIDATES, times[:k])},
                         "merge": {c: float(v) for c, v in zip(MERGE_CANDIDATES, times[k:])}}


def tuning_cache_save(path: str, device: str | None = None):
    """Write the shapes set through this module to a JSON cache, under the
    current device's name (entries of other devices already in the file stay)."""
    import json
    device = device or _torch().cuda.get_device_name()
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[device] = [{"bits": b, "n_bit_length": nb, **shape}
                    for (b, nb), shape in sorted(_tuned.items())]
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def tuning_cache_load(path: str, device: str | None = None) -> int:
    """Apply the cached shapes of the current device; returns how many."""
    import json
    device = device or _torch().cuda.get_device_name()
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        entries = json.load(f).get(device, [])
    for e in entries:
        nb = int(e["n_bit_length"])
        tuning_set(int(e["bits"]), (1 << (nb - 1)) if nb > 0 else 0,
                   {k: int(e[k]) for k in ("radix_bits", "sort_threads", "merge_half")})
    return len(entries)


def selftest_wait_timeout(stream=None) -> int:
    """Run the bounded-wait self-test; returns the status the device recorded."""
    lib = load()
    lib.cga_selftest_wait_timeout.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
    obs = ctypes.c_int(0)
    _check(lib.cga_selftest_wait_timeout(_stream(stream), ctypes.byref(obs)),
           "cga_selftest_wait_timeout")
    return obs.value


# ------------------------------------------- compression pieces and G-Arrays
KMEANS_MAX_ITER = 1024


def _dev_i32xyz(t, what):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32
            and t.is_contiguous() and t.numel() % 3 == 0):
        raise TypeError(f"{what}: expected a contiguous (m, 3) int32 CUDA tensor")
    return t


def cga_kmeans(a: Cga, max_iter: int = 64, stream=None, u=None):
    """k-means of a's voxels with 8 corner-seeded centres (Sec. V-D): (labels (u,)
    uint8, centres (8, 3) int64 in 1/256 voxel, counts (8,) int64, passes (1,) int32),
    all device tensors.  With u (a's voxel count) given nothing is synchronized."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_kmeans.argtypes = [P, ctypes.c_uint32, P, P, P, P, P]
    u = a.info()["u"] if u is None else int(u)
    lab = torch.empty(max(u, 1), dtype=torch.uint8, device="cuda")
    cen = torch.empty((8, 3), dtype=torch.int64, device="cuda")
    cnt = torch.empty(8, dtype=torch.int64, device="cuda")
    it = torch.empty(1, dtype=torch.int32, device="cuda")
    _check(lib.cga_kmeans(a.ptr, int(max_iter), P(lab.data_ptr()), P(cen.data_ptr()),
                          P(cnt.data_ptr()), P(it.data_ptr()), _stream(stream)), "cga_kmeans")
    return lab[:u], cen, cnt, it


def cga_motion_vectors(ref_centres, ref_counts, pred_centres, pred_counts, stream=None):
    """mv = ref - pred centre per cluster non-empty in both frames: (8, 3) int64."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_motion_vectors.argtypes = [P, P, P, P, P, P]
    for t in (ref_centres, ref_counts, pred_centres, pred_counts):
        if not (t.is_cuda and t.dtype == torch.int64 and t.is_contiguous()):
            raise TypeError("cga_motion_vectors: expected contiguous int64 CUDA tensors")
    mv = torch.empty((8, 3), dtype=torch.int64, device="cuda")
    _check(lib.cga_motion_vectors(P(ref_centres.data_ptr()), P(ref_counts.data_ptr()),
                                  P(pred_centres.data_ptr()), P(pred_counts.data_ptr()),
                                  P(mv.data_ptr()), _stream(stream)), "cga_motion_vectors")
    return mv


def cga_reconstruct(pred: Cga, labels, mv, stream=None, u=None):
    """pred's voxels moved by their cluster's vector rounded half up: (u, 3) int32."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_reconstruct.argtypes = [P, P, P, P, P]
    u = pred.info()["u"] if u is None else int(u)
    out = torch.empty((max(u, 1), 3), dtype=torch.int32, device="cuda")
    _check(lib.cga_reconstruct(pred.ptr, P(labels.data_ptr()), P(mv.data_ptr()),
                               P(out.data_ptr()), _stream(stream)), "cga_reconstruct")
    return out[:u]


def cga_nn_query_voxels(a: Cga, qv, stream=None):
    """Exact NN of integer query voxels: (idx (m,) int32 holding uint32, dist2 (m,) int64)."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_nn_query_voxels.argtypes = [P, P, ctypes.c_uint64, P, P, P]
    _dev_i32xyz(qv, "cga_nn_query_voxels")
    m = qv.numel() // 3
    idx = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    d2 = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    _check(lib.cga_nn_query_voxels(a.ptr, P(qv.data_ptr()), m, P(idx.data_ptr()),
                                   P(d2.data_ptr()), _stream(stream)), "cga_nn_query_voxels")
    return idx[:m], d2[:m]


def cga_lookup(a: Cga, qv, stream=None):
    """CGA index of each integer voxel (int32 holding uint32; UINT32_MAX when absent)."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_lookup.argtypes = [P, P, ctypes.c_uint64, P, P]
    _dev_i32xyz(qv, "cga_lookup")
    m = qv.numel() // 3
    idx = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    _check(lib.cga_lookup(a.ptr, P(qv.data_ptr()), m, P(idx.data_ptr()), _stream(stream)),
           "cga_lookup")
    return idx[:m]


def cga_garrays_x(a: Cga, stream=None):
    """The G-Arrays X pointer: 2^bits + 1 cells (int32 holding uint32)."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_garrays_x.argtypes = [P, P, P]
    out = torch.empty((1 << a.grid.bits) + 1, dtype=torch.int32, device="cuda")
    _check(lib.cga_garrays_x(a.ptr, P(out.data_ptr()), _stream(stream)), "cga_garrays_x")
    return out


def cga_garrays_lookup(a: Cga, xptr, qv, stream=None):
    """cga_lookup through the dense G-Arrays X pointer."""
    torch = _torch()
    lib = load()
    P = ctypes.c_void_p
    lib.cga_garrays_lookup.argtypes = [P, P, P, ctypes.c_uint64, P, P]
    _dev_i32xyz(qv, "cga_garrays_lookup")
    m = qv.numel() // 3
    idx = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    _check(lib.cga_garrays_lookup(a.ptr, P(xptr.data_ptr()), P(qv.data_ptr()), m,
                                  P(idx.data_ptr()), _stream(stream)), "cga_garrays_lookup")
    return idx[:m]


def cga_residual(pred_values, ref_values, idx, stream=None):
    """Residual frame (Sec. V-D): pred - ref[idx] per channel as an (u_pred, C) int16
    tensor (pred where idx has no reference point).  Values: (u, C) uint8 CUDA
    tensors; idx: (u_pred,) int32 CUDA tensor holding uint32."""
    import torch
    for t in (pred_values, ref_values, idx):
        if not isinstance(t, torch.Tensor):
            raise TypeError("cga_residual: expected torch tensors")
    # the kernel reads u_pred rows of pred and indexes ref with pred's row
    # width: both must be (rows, C) with the same C, and pred must have one
    # row per entry of idx
    ch = pred_values.shape[1] if pred_values.dim() > 1 else 1
    if (pred_values.dim() != 2 or ref_values.dim() != 2 or ref_values.shape[1] != ch
            or pred_values.shape[0] != idx.numel() or idx.dim() != 1):
        raise ValueError(f"cga_residual: pred_values {tuple(pred_values.shape)}, ref_values "
                         f"{tuple(ref_values.shape)} and idx {tuple(idx.shape)} must be (u_pred, C),"
                         f" (u_ref, C) and (u_pred,)")
    torch = _torch()
    for t in (pred_values, ref_values, idx):
        if not (t.is_cuda and t.is_contiguous()):
            raise TypeError("cga_residual: expected contiguous CUDA tensors")
    lib = load()
    P = ctypes.c_void_p
    lib.cga_residual.argtypes = [P, ctypes.c_uint64, P, ctypes.c_uint64, P, ctypes.c_uint32, P, P]
    u_pred = idx.numel()
    u_ref = ref_values.shape[0]
    out = torch.empty((max(u_pred, 1), ch), dtype=torch.int16, device="cuda")
    _check(lib.cga_residual(P(pred_values.data_ptr()), u_pred, P(ref_values.data_ptr()), u_ref,
                            P(idx.data_ptr()), ch, P(out.data_ptr()), _stream(stream)),
           "cga_residual")
    return out[:u_pred]

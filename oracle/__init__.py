"""ctypes wrapper around the C++ CPU oracle (``cga_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` load this module; the CUDA library and its
Python binding never do.  The oracle computes the plain definitions of the
paper's CGA operations (Sec. V arrays, Eq. 1 merge, Eq. 3 projection,
Eq. 7-8 nearest neighbour) with std::sort / std::unique / std::set_union and
exhaustive search.

Parity pinned: tests/test_oracle_*.py pin every function against hand fixtures
(tests/golden/), closed forms, invariants and independent numpy routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cga_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_NONFINITE = -2

U32_MAX = 0xFFFFFFFF
U64_MAX = 0xFFFFFFFFFFFFFFFF


def compile_oracle(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, no fused mul-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "cga_oracle.h"))
    ):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC",
             "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Cga(ctypes.Structure):
    _fields_ = [
        ("bits", ctypes.c_uint32),
        ("h", ctypes.c_uint64),
        ("g", ctypes.c_uint64),
        ("u", ctypes.c_uint64),
        ("X_index", ctypes.c_void_p),
        ("X_pointer", ctypes.c_void_p),
        ("Y_index", ctypes.c_void_p),
        ("Y_pointer", ctypes.c_void_p),
        ("Z_index", ctypes.c_void_p),
    ]


class _Cga2d(ctypes.Structure):
    _fields_ = [
        ("bits", ctypes.c_uint32),
        ("h", ctypes.c_uint64),
        ("g", ctypes.c_uint64),
        ("U_index", ctypes.c_void_p),
        ("U_pointer", ctypes.c_void_p),
        ("V_index", ctypes.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(compile_oracle())
        P = ctypes.c_void_p
        U32, U64, F = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float
        _lib.orc_grid_from_box.argtypes = [P, F, U32, P, P]
        _lib.orc_quantize.argtypes = [P, U64, U32, F, P, P, P]
        _lib.orc_from_sorted_keys.argtypes = [P, U64, U32, ctypes.POINTER(_Cga)]
        _lib.orc_build.argtypes = [P, U64, U32, F, P, P, ctypes.POINTER(_Cga)]
        _lib.orc_decode.argtypes = [ctypes.POINTER(_Cga), P]
        _lib.orc_decode_keys.argtypes = [ctypes.POINTER(_Cga), P]
        _lib.orc_lookup.argtypes = [ctypes.POINTER(_Cga), U32, U32, U32]
        _lib.orc_lookup.restype = ctypes.c_int64
        _lib.orc_merge.argtypes = [ctypes.POINTER(_Cga), ctypes.POINTER(_Cga),
                                   ctypes.POINTER(_Cga)]
        _lib.orc_project.argtypes = [ctypes.POINTER(_Cga), ctypes.c_int,
                                     ctypes.POINTER(_Cga2d)]
        _lib.orc_query_voxels.argtypes = [P, U64, F, P, P, P]
        _lib.orc_radius_count.argtypes = [ctypes.POINTER(_Cga), F, P, P, U64, U64, P]
        _lib.orc_radius_fill.argtypes = [ctypes.POINTER(_Cga), F, P, P, U64, U64, P, P, P]
        _lib.orc_knn.argtypes = [ctypes.POINTER(_Cga), F, P, P, U64, U32, P, P]
        _lib.orc_perspective.argtypes = [ctypes.POINTER(_Cga), P, F, F, F, U32, U32, P, P]
        _lib.orc_build_values.argtypes = [P, P, U32, U64, U32, F, P, P, ctypes.c_int,
                                          ctypes.POINTER(_Cga), P]
        _lib.orc_merge_values.argtypes = [ctypes.POINTER(_Cga), P, ctypes.POINTER(_Cga), P, U32,
                                          ctypes.c_int, ctypes.POINTER(_Cga), P]
        C = ctypes.POINTER(_Cga)
        _lib.orc_lookup_voxels.argtypes = [C, P, U64, P]
        _lib.orc_garrays_x.argtypes = [C, P]
        _lib.orc_garrays_lookup.argtypes = [C, P, P, U64, P]
        _lib.orc_nn_voxels.argtypes = [C, P, U64, P, P]
        _lib.orc_kmeans.argtypes = [C, U32, P, P, P, P]
        _lib.orc_motion_vectors.argtypes = [P, P, P, P, P]
        _lib.orc_reconstruct.argtypes = [C, P, P, P]
        _lib.orc_residual.argtypes = [P, U64, P, U64, P, U32, P]
        for fn in (_lib.orc_nn_brute, _lib.orc_nn_window):
            fn.argtypes = [ctypes.POINTER(_Cga), F, P, P, U64, P, P]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Grid:
    bits: int
    scale: float  # float32 value held in a Python float
    offset: tuple  # three float32 values

    def offset_array(self) -> np.ndarray:
        return np.asarray(self.offset, dtype=np.float32)


@dataclass
class Cga:
    """Host copy of the five geometry arrays of a CGA."""
    bits: int
    X_index: np.ndarray
    X_pointer: np.ndarray
    Y_index: np.ndarray
    Y_pointer: np.ndarray
    Z_index: np.ndarray

    @property
    def h(self):
        return len(self.X_index)

    @property
    def g(self):
        return len(self.Y_index)

    @property
    def u(self):
        return len(self.Z_index)

    def nbytes(self) -> int:
        return 2 * self.h + 4 * (self.h + 1) + 2 * self.g + 4 * (self.g + 1) + 2 * self.u

    def _struct(self):
        # keep contiguous arrays alive on the instance while the struct is used
        self._keep = [np.ascontiguousarray(a) for a in (
            self.X_index, self.X_pointer, self.Y_index, self.Y_pointer, self.Z_index)]
        k = self._keep
        return _Cga(self.bits, self.h, self.g, self.u,
                    _ptr(k[0]), _ptr(k[1]), _ptr(k[2]), _ptr(k[3]), _ptr(k[4]))


@dataclass
class Cga2d:
    bits: int
    U_index: np.ndarray
    U_pointer: np.ndarray
    V_index: np.ndarray


def _empty_out(bits: int, cap: int):
    arrs = (np.zeros(cap, np.uint16), np.zeros(cap + 1, np.uint32),
            np.zeros(cap, np.uint16), np.zeros(cap + 1, np.uint32),
            np.zeros(cap, np.uint16))
    s = _Cga(bits, 0, 0, 0, *(_ptr(a) for a in arrs))
    return s, arrs


def _from_struct(s: _Cga, arrs) -> Cga:
    h, g, u = s.h, s.g, s.u
    return Cga(s.bits, arrs[0][:h].copy(), arrs[1][:h + 1].copy(), arrs[2][:g].copy(),
               arrs[3][:g + 1].copy(), arrs[4][:u].copy())


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


def _check(rc):
    if rc != OK:
        raise OracleError(rc)


def grid_from_box(lo, extent: float, bits: int) -> Grid:
    lo = np.asarray(lo, dtype=np.float32)
    scale = np.zeros(1, np.float32)
    off = np.zeros(3, np.float32)
    _check(lib().orc_grid_from_box(_ptr(lo), float(np.float32(extent)), bits,
                                   _ptr(scale), _ptr(off)))
    return Grid(bits, float(scale[0]), tuple(float(v) for v in off))


def _f32xyz(xyz) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    return a


def _xform(xform):
    if xform is None:
        return None, None
    x = np.ascontiguousarray(np.asarray(xform, dtype=np.float32).reshape(12))
    return x, _ptr(x)


def quantize(xyz, grid: Grid, xform=None) -> np.ndarray:
    p = _f32xyz(xyz)
    keys = np.zeros(len(p), np.uint64)
    x, xp = _xform(xform)
    off = grid.offset_array()
    _check(lib().orc_quantize(_ptr(p), len(p), grid.bits, grid.scale, _ptr(off), xp,
                              _ptr(keys)))
    return keys


def from_sorted_keys(keys, bits: int) -> Cga:
    k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint64))
    s, arrs = _empty_out(bits, len(k))
    _check(lib().orc_from_sorted_keys(_ptr(k), len(k), bits, ctypes.byref(s)))
    return _from_struct(s, arrs)


def build(xyz, grid: Grid, xform=None) -> Cga:
    p = _f32xyz(xyz)
    s, arrs = _empty_out(grid.bits, len(p))
    x, xp = _xform(xform)
    off = grid.offset_array()
    _check(lib().orc_build(_ptr(p), len(p), grid.bits, grid.scale, _ptr(off), xp,
                           ctypes.byref(s)))
    return _from_struct(s, arrs)


def decode(a: Cga) -> np.ndarray:
    out = np.zeros((a.u, 3), np.uint32)
    s = a._struct()
    _check(lib().orc_decode(ctypes.byref(s), _ptr(out)))
    return out


def decode_keys(a: Cga) -> np.ndarray:
    out = np.zeros(a.u, np.uint64)
    s = a._struct()
    _check(lib().orc_decode_keys(ctypes.byref(s), _ptr(out)))
    return out


def lookup(a: Cga, x: int, y: int, z: int) -> int:
    s = a._struct()
    return int(lib().orc_lookup(ctypes.byref(s), x, y, z))


def merge(a: Cga, b: Cga) -> Cga:
    sa, sb = a._struct(), b._struct()
    s, arrs = _empty_out(a.bits, a.u + b.u)
    _check(lib().orc_merge(ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(s)))
    return _from_struct(s, arrs)


VALUE_POLICIES = {"average": 0, "first": 1}
MERGE_POLICIES = {"base": 0, "average": 1}


def _attrs(attr, n):
    a = np.asarray(attr, dtype=np.uint8)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    if a.shape[0] != n:
        raise ValueError("one attribute row per point")
    return np.ascontiguousarray(a)


def build_values(xyz, attr, grid: Grid, xform=None, policy="average"):
    """Build plus the Value array (Sec. V): returns (Cga, values (u, channels) uint8)."""
    p = _f32xyz(xyz)
    a = _attrs(attr, len(p))
    ch = a.shape[1]
    s, arrs = _empty_out(grid.bits, len(p))
    vals = np.zeros((max(len(p), 1), ch), np.uint8)
    x, xp = _xform(xform)
    off = grid.offset_array()
    _check(lib().orc_build_values(_ptr(p), _ptr(a), ch, len(p), grid.bits, grid.scale, _ptr(off),
                                  xp, VALUE_POLICIES[policy], ctypes.byref(s), _ptr(vals)))
    c = _from_struct(s, arrs)
    return c, vals[:c.u].copy()


def merge_values(a: Cga, va, b: Cga, vb, policy="base"):
    """Merge with the Value arrays of a (the base) and b: returns (Cga, values)."""
    va = np.ascontiguousarray(np.asarray(va, dtype=np.uint8))
    vb = np.ascontiguousarray(np.asarray(vb, dtype=np.uint8))
    ch = va.shape[1] if va.ndim > 1 else 1
    sa, sb = a._struct(), b._struct()
    s, arrs = _empty_out(a.bits, a.u + b.u)
    vals = np.zeros((max(a.u + b.u, 1), ch), np.uint8)
    _check(lib().orc_merge_values(ctypes.byref(sa), _ptr(va), ctypes.byref(sb), _ptr(vb), ch,
                                  MERGE_POLICIES[policy], ctypes.byref(s), _ptr(vals)))
    c = _from_struct(s, arrs)
    return c, vals[:c.u].copy()


def radius(a: Cga, grid: Grid, q, r2: int):
    """Radius search: (offsets (m+1,) uint64, idx uint32, dist2 uint64) with query j's
    voxels, ascending CGA index, at [offsets[j], offsets[j+1])."""
    qq = _f32xyz(q)
    off = grid.offset_array()
    s = a._struct()
    counts = np.zeros(max(len(qq), 1), np.uint64)
    _check(lib().orc_radius_count(ctypes.byref(s), grid.scale, _ptr(off), _ptr(qq), len(qq),
                                  int(r2), _ptr(counts)))
    offsets = np.zeros(len(qq) + 1, np.uint64)
    offsets[1:] = np.cumsum(counts[:len(qq)])
    total = int(offsets[-1])
    idx = np.zeros(max(total, 1), np.uint32)
    d2 = np.zeros(max(total, 1), np.uint64)
    _check(lib().orc_radius_fill(ctypes.byref(s), grid.scale, _ptr(off), _ptr(qq), len(qq),
                                 int(r2), _ptr(offsets), _ptr(idx), _ptr(d2)))
    return offsets, idx[:total], d2[:total]


def knn(a: Cga, grid: Grid, q, k: int):
    """k nearest stored voxels per query by (distance^2, key): (idx (m, k), dist2 (m, k))."""
    qq = _f32xyz(q)
    off = grid.offset_array()
    s = a._struct()
    idx = np.zeros(max(len(qq) * k, 1), np.uint32)
    d2 = np.zeros(max(len(qq) * k, 1), np.uint64)
    _check(lib().orc_knn(ctypes.byref(s), grid.scale, _ptr(off), _ptr(qq), len(qq), k,
                         _ptr(idx), _ptr(d2)))
    return idx[:len(qq) * k].reshape(len(qq), k), d2[:len(qq) * k].reshape(len(qq), k)


def perspective(a: Cga, eye, cos_t: float, sin_t: float, D: float, W: int, H: int):
    """Perspective z-buffer image (Eq. 5-6): (index (H, W) uint32, depth (H, W) float32)."""
    e = np.ascontiguousarray(np.asarray(eye, np.float32).reshape(3))
    idx = np.zeros(W * H, np.uint32)
    dep = np.zeros(W * H, np.float32)
    s = a._struct()
    _check(lib().orc_perspective(ctypes.byref(s), _ptr(e), float(np.float32(cos_t)),
                                 float(np.float32(sin_t)), float(np.float32(D)), W, H, _ptr(idx),
                                 _ptr(dep)))
    return idx.reshape(H, W), dep.reshape(H, W)


PLANES = {"xy": 0, "xz": 1, "yz": 2}


def project(a: Cga, plane) -> Cga2d:
    p = PLANES[plane] if isinstance(plane, str) else int(plane)
    sa = a._struct()
    cap = a.u
    arrs = (np.zeros(cap, np.uint16), np.zeros(cap + 1, np.uint32), np.zeros(cap, np.uint16))
    s = _Cga2d(a.bits, 0, 0, *(_ptr(x) for x in arrs))
    _check(lib().orc_project(ctypes.byref(sa), p, ctypes.byref(s)))
    return Cga2d(a.bits, arrs[0][:s.h].copy(), arrs[1][:s.h + 1].copy(), arrs[2][:s.g].copy())


def _nn(fn, a: Cga, grid: Grid, q):
    qa = _f32xyz(q)
    idx = np.zeros(len(qa), np.uint32)
    d2 = np.zeros(len(qa), np.uint64)
    s = a._struct()
    off = grid.offset_array()
    _check(fn(ctypes.byref(s), grid.scale, _ptr(off), _ptr(qa), len(qa), _ptr(idx), _ptr(d2)))
    return idx, d2


def query_voxels(grid: Grid, q):
    """(m, 3) int64 query voxels and an m-long validity mask (NN reading)."""
    qa = _f32xyz(q)
    out = np.zeros((len(qa), 3), np.int64)
    valid = np.zeros(len(qa), np.uint8)
    off = grid.offset_array()
    _check(lib().orc_query_voxels(_ptr(qa), len(qa), grid.scale, _ptr(off), _ptr(out),
                                  _ptr(valid)))
    return out, valid.astype(bool)


def nn_brute(a: Cga, grid: Grid, q):
    return _nn(lib().orc_nn_brute, a, grid, q)


def nn_window(a: Cga, grid: Grid, q):
    return _nn(lib().orc_nn_window, a, grid, q)


# ---- compression pieces (Sec. V-D) and the G-Arrays form (Sec. V) -----------
def _i32xyz(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(-1, 3))


def lookup_voxels(a: Cga, qv):
    """CGA index of each integer voxel (uint32), UINT32_MAX when absent."""
    q = _i32xyz(qv)
    out = np.zeros(max(len(q), 1), np.uint32)
    s = a._struct()
    _check(lib().orc_lookup_voxels(ctypes.byref(s), _ptr(q), len(q), _ptr(out)))
    return out[:len(q)]


def garrays_x(a: Cga):
    """The G-Arrays X_pointer: 2^bits + 1 cells, xptr[v] = columns with x < v."""
    out = np.zeros((1 << a.bits) + 1, np.uint32)
    s = a._struct()
    _check(lib().orc_garrays_x(ctypes.byref(s), _ptr(out)))
    return out


def garrays_lookup(a: Cga, xptr, qv):
    """The lookup through the G-Arrays X_pointer (same answer as lookup_voxels)."""
    q = _i32xyz(qv)
    xp = np.ascontiguousarray(np.asarray(xptr, np.uint32))
    out = np.zeros(max(len(q), 1), np.uint32)
    s = a._struct()
    _check(lib().orc_garrays_lookup(ctypes.byref(s), _ptr(xp), _ptr(q), len(q), _ptr(out)))
    return out[:len(q)]


def nn_voxels(a: Cga, qv):
    """Exact NN of integer query voxels: (idx uint32, dist2 uint64)."""
    q = _i32xyz(qv)
    idx = np.zeros(max(len(q), 1), np.uint32)
    d2 = np.zeros(max(len(q), 1), np.uint64)
    s = a._struct()
    _check(lib().orc_nn_voxels(ctypes.byref(s), _ptr(q), len(q), _ptr(idx), _ptr(d2)))
    return idx[:len(q)], d2[:len(q)]


def kmeans(a: Cga, max_iter: int):
    """k-means of the stored voxels, 8 corner-seeded centres (Sec. V-D):
    (labels (u,) uint8, centres (8, 3) int64 in 1/256 voxel, counts (8,) uint64, passes)."""
    lab = np.zeros(max(a.u, 1), np.uint8)
    cen = np.zeros(24, np.int64)
    cnt = np.zeros(8, np.uint64)
    it = np.zeros(1, np.uint32)
    s = a._struct()
    _check(lib().orc_kmeans(ctypes.byref(s), int(max_iter), _ptr(lab), _ptr(cen), _ptr(cnt),
                            _ptr(it)))
    return lab[:a.u], cen.reshape(8, 3), cnt, int(it[0])


def motion_vectors(ref_centres, ref_counts, pred_centres, pred_counts):
    """mv[c] = ref[c] - pred[c] (1/256 voxel), 0 where either cluster is empty."""
    rc = np.ascontiguousarray(np.asarray(ref_centres, np.int64).reshape(24))
    pc = np.ascontiguousarray(np.asarray(pred_centres, np.int64).reshape(24))
    rn = np.ascontiguousarray(np.asarray(ref_counts, np.uint64).reshape(8))
    pn = np.ascontiguousarray(np.asarray(pred_counts, np.uint64).reshape(8))
    mv = np.zeros(24, np.int64)
    _check(lib().orc_motion_vectors(_ptr(rc), _ptr(rn), _ptr(pc), _ptr(pn), _ptr(mv)))
    return mv.reshape(8, 3)


def reconstruct(a: Cga, labels, mv):
    """Each voxel moved by its cluster's motion vector rounded half up: (u, 3) int32."""
    lab = np.ascontiguousarray(np.asarray(labels, np.uint8))
    m = np.ascontiguousarray(np.asarray(mv, np.int64).reshape(24))
    out = np.zeros((max(a.u, 1), 3), np.int32)
    s = a._struct()
    _check(lib().orc_reconstruct(ctypes.byref(s), _ptr(lab), _ptr(m), _ptr(out)))
    return out[:a.u]


def residual(pred_values, ref_values, idx):
    """Residual frame (Sec. V-D): pred - ref[idx] per channel as int16 (pred where
    idx has no reference point)."""
    pv = np.ascontiguousarray(np.asarray(pred_values, np.uint8))
    rv = np.ascontiguousarray(np.asarray(ref_values, np.uint8))
    ch = pv.shape[1] if pv.ndim > 1 else 1
    ix = np.ascontiguousarray(np.asarray(idx, np.uint32))
    u_pred = len(ix)
    u_ref = len(rv) if rv.ndim > 1 else len(rv) // ch
    out = np.zeros((max(u_pred, 1), ch), np.int16)
    _check(lib().orc_residual(_ptr(pv), u_pred, _ptr(rv), u_ref, _ptr(ix), ch, _ptr(out)))
    return out[:u_pred]

"""C-ABI library: it loads, exports every symbol include/cga.h declares, and
its host-only logic (grid set-up, argument checks) behaves -- no GPU work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_11616_gb300 import build_ext, cga
    build_ext.build()
    return cga.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cga.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(cga[a-z_0-9]*)\s*\(", text, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_2110_11616_gb300 import cga
    assert sorted(cga.EXPORTS) == declared_functions()


def test_grid_from_box_matches_oracle(lib, orc):
    from paper_2110_11616_gb300 import cga
    for lo, ext, bits in [((0, 0, 0), 1.0, 10), ((-128, -128, -128), 256.0, 16),
                          ((0.1, -3.7, 2.25), 13.3, 12), ((5, 5, 5), 0.37, 1)]:
        g = cga.grid_from_box(lo, ext, bits)
        o = orc.grid_from_box(lo, ext, bits)
        assert g.bits == o.bits and np.float32(g.scale) == np.float32(o.scale)
        assert tuple(np.float32(v) for v in g.offset) == tuple(np.float32(v) for v in o.offset)


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2110_11616_gb300 import cga
    g = cga.Grid()
    out = ctypes.c_void_p()
    lo = (ctypes.c_float * 3)(0, 0, 0)
    assert lib.cga_grid_from_box(lo, 1.0, 0, ctypes.byref(g)) == cga.ERR_INVALID_ARG
    assert lib.cga_grid_from_box(lo, 1.0, 17, ctypes.byref(g)) == cga.ERR_INVALID_ARG
    assert lib.cga_grid_from_box(lo, -1.0, 8, ctypes.byref(g)) == cga.ERR_INVALID_ARG
    bad = cga.make_grid(0, 1.0, (0, 0, 0))
    assert lib.cga_build(None, 0, ctypes.byref(bad), None, None, None,
                         ctypes.byref(out)) == cga.ERR_INVALID_ARG
    nanscale = cga.make_grid(8, float("nan"), (0, 0, 0))
    assert lib.cga_build(None, 0, ctypes.byref(nanscale), None, None, None,
                         ctypes.byref(out)) == cga.ERR_INVALID_ARG
    ok = cga.make_grid(8, 1.0, (0, 0, 0))
    assert lib.cga_build(None, 5, ctypes.byref(ok), None, None, None,
                         ctypes.byref(out)) == cga.ERR_INVALID_ARG
    assert lib.cga_build(ctypes.c_void_p(16), cga.MAX_POINTS + 1, ctypes.byref(ok), None, None,
                         None, ctypes.byref(out)) == cga.ERR_INVALID_ARG
    assert lib.cga_build(None, 0, ctypes.byref(ok), None, None, None, None) == cga.ERR_INVALID_ARG
    assert lib.cga_merge(None, None, None, None, ctypes.byref(out)) == cga.ERR_INVALID_ARG
    assert lib.cga_project(None, 0, None, None, ctypes.byref(out)) == cga.ERR_INVALID_ARG
    assert lib.cga_nn_query(None, None, 1, None, None, None) == cga.ERR_INVALID_ARG
    assert lib.cga_decode(None, None, None) == cga.ERR_INVALID_ARG
    assert lib.cga_nn_prepare_levels(None, None, 0, None) == cga.ERR_INVALID_ARG
    assert lib.cga_nn_prepare(None, 0, None) == cga.ERR_INVALID_ARG
    assert out.value is None


def test_search_and_compression_arguments_rejected_on_host(lib):
    """Null handles and out-of-range sizes are refused before any device work."""
    from paper_2110_11616_gb300 import cga
    P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "cga_knn": [P, P, U64, U32, P, P, P],
        "cga_radius_count": [P, P, U64, U64, P, P],
        "cga_radius_fill": [P, P, U64, U64, P, P, P, P],
        "cga_kmeans": [P, U32, P, P, P, P, P],
        "cga_motion_vectors": [P, P, P, P, P, P],
        "cga_reconstruct": [P, P, P, P, P],
        "cga_nn_query_voxels": [P, P, U64, P, P, P],
        "cga_lookup": [P, P, U64, P, P],
        "cga_garrays_x": [P, P, P],
        "cga_garrays_lookup": [P, P, P, U64, P, P],
        "cga_residual": [P, U64, P, U64, P, U32, P, P],
    }
    for name, args in sig.items():
        getattr(lib, name).argtypes = args
    bad = cga.ERR_INVALID_ARG
    assert lib.cga_knn(None, None, 1, 8, None, None, None) == bad
    assert lib.cga_radius_count(None, None, 1, 4, None, None) == bad
    assert lib.cga_radius_fill(None, None, 1, 4, None, None, None, None) == bad
    assert lib.cga_kmeans(None, 10, None, None, None, None, None) == bad
    assert lib.cga_motion_vectors(None, None, None, None, None, None) == bad
    assert lib.cga_reconstruct(None, None, None, None, None) == bad
    assert lib.cga_nn_query_voxels(None, None, 1, None, None, None) == bad
    assert lib.cga_lookup(None, None, 1, None, None) == bad
    assert lib.cga_garrays_x(None, None, None) == bad
    assert lib.cga_garrays_lookup(None, None, None, 1, None, None) == bad
    assert lib.cga_residual(None, 1, None, 1, None, 3, None, None) == bad
    assert lib.cga_residual(None, 0, None, 0, None, 0, None, None) == bad  # channels 0


def test_strerror_names_every_code(lib):
    from paper_2110_11616_gb300 import cga
    seen = set()
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        s = lib.cga_strerror(code).decode()
        assert s and s != "unknown error"
        seen.add(s)
    assert len(seen) == 8
    assert lib.cga_strerror(-99).decode() == "unknown error"


def test_residual_wrapper_rejects_mismatched_shapes():
    """cga_residual's binding checks the row counts and channel widths it
    passes to the kernel (which cannot see them) before anything runs."""
    import torch

    from paper_2110_11616_gb300 import cga
    pred = torch.zeros((10, 3), dtype=torch.uint8)
    ref = torch.zeros((7, 3), dtype=torch.uint8)
    idx = torch.zeros(10, dtype=torch.int32)
    for p, r, i in [(pred, ref, idx[:9]),                                 # rows != idx
                    (pred, torch.zeros((7, 4), dtype=torch.uint8), idx),  # channel widths
                    (pred.reshape(-1), ref, idx),                         # not (rows, C)
                    (pred, ref, idx.reshape(2, 5))]:
        with pytest.raises(ValueError):
            cga.cga_residual(p, r, i)
    # shapes agree: host tensors are refused next (no GPU here: refused earlier)
    with pytest.raises((TypeError, RuntimeError)):
        cga.cga_residual(pred, ref, idx)

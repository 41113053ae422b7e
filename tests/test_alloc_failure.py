"""Allocator failure on the host: when the caller's allocator returns NULL
part-way through a call, the call returns CGA_ERR_OOM and hands back every
block it had already obtained (no leak).  The fake allocator returns fake
addresses, and the failing calls stop before any device work is queued, so
this runs without a GPU."""
import ctypes

import pytest

from paper_2110_11616_gb300 import build_ext, cga


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return cga.load()


class FakeAllocator:
    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()
        self.next = 1 << 40

        @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        def alloc(ctx, n, stream):
            self.calls += 1
            if self.calls >= self.fail_at:
                return None
            p = self.next
            self.next += (int(n) + 4095) & ~4095
            self.live.add(p)
            return p

        @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
        def free(ctx, p, stream):
            self.live.discard(p)

        self._a, self._f = alloc, free
        self.struct = cga.Allocator(None, alloc, free)


@pytest.mark.parametrize("fail_at", [1, 2])
def test_build_oom_releases_everything(lib, fail_at):
    fa = FakeAllocator(fail_at)
    g = cga.make_grid(10, 1024.0, (0.0, 0.0, 0.0))
    out = ctypes.c_void_p()
    rc = lib.cga_build(ctypes.c_void_p(1 << 20), 1000, ctypes.byref(g), None,
                       ctypes.byref(fa.struct), None, ctypes.byref(out))
    assert rc == cga.ERR_OOM
    assert out.value is None
    assert fa.live == set()
    assert fa.calls == fail_at


def test_allocator_with_missing_callback_is_rejected(lib):
    a = cga.Allocator()  # both callbacks NULL
    g = cga.make_grid(10, 1024.0, (0.0, 0.0, 0.0))
    out = ctypes.c_void_p()
    assert lib.cga_build(None, 0, ctypes.byref(g), None, ctypes.byref(a), None,
                         ctypes.byref(out)) == cga.ERR_INVALID_ARG

"""The oracle's window NN search (Sec. V-C, oracle/) called on query chunks
from a pool of threads, for the full-size parity checks: its ctypes calls
release the GIL, so the chunks run on every host core.  The oracle itself is
called unchanged; only the queries are split, and the answers joined back in
query order."""
import concurrent.futures as cf
import os

import numpy as np


def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def nn_window(orc, o_cga, og, q, threads=None):
    """orc.nn_window(o_cga, og, q), the queries split over `threads` threads."""
    q = np.ascontiguousarray(q, dtype=np.float32).reshape(-1, 3)
    t = threads or host_threads()
    n = len(q)
    if n == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint64)
    chunk = max(16, -(-n // (4 * t)))
    parts = [q[i:i + chunk] for i in range(0, n, chunk)]
    with cf.ThreadPoolExecutor(max_workers=t) as ex:
        res = list(ex.map(lambda p: orc.nn_window(o_cga, og, p), parts))
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])

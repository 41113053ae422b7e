"""Reader for the hand-derived fixtures in tests/golden/cga_fixtures.txt."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_DTYPES = {"index": np.uint16, "pointer": np.uint32}


def _points(text):
    rows = [r.split() for r in text.split(";") if r.strip()]
    return np.array([[int(v) for v in r] for r in rows], np.int64).reshape(-1, 3)


def load_cases(name="cga_fixtures.txt"):
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, _, rest = line.partition(" ")
            if head == "case":
                cur = {"name": rest.strip()}
            elif head == "end":
                cases[cur["name"]] = cur
                cur = None
            elif head == "bits":
                cur["bits"] = int(rest)
            elif head in ("points", "a", "b"):
                cur[head] = _points(rest)
            else:
                kind = "pointer" if head.endswith("pointer") else "index"
                cur[head] = np.array([int(v) for v in rest.split()], _DTYPES[kind])
    return cases


def voxels_to_float(vox):
    """Integer voxel coordinates as float32 points for the grid scale = 1,
    offset = 0, where floor(fma(p, 1, 0)) returns the voxel itself."""
    return np.asarray(vox, np.float64).astype(np.float32).reshape(-1, 3)

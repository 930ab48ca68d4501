"""Host-side logic of bench.py that needs no GPU: the count of grid cells the
kernel boxes cover (the grid part of the table kernel's minimum HBM bytes),
against brute-force enumeration of every box."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def brute_cells(uvw, info, conj_fold):
    npad, du = info["npad"], info["du"]
    wbar = np.asarray(info["wbar"])
    cells = set()
    for u, v, w in uvw:
        if conj_fold and w < 0:
            u, v, w = -u, -v, -w
        k = int(np.argmin(np.abs(w - wbar)))
        up, vp = u / du, v / du
        if not (-npad / 2 <= up < npad / 2 and -npad / 2 <= vp < npad / 2):
            continue
        J = info["jw"][k]
        q0u = int(np.floor(up)) - J // 2 + 1
        q0v = int(np.floor(vp)) - J // 2 + 1
        for b in range(J):
            for a in range(J):
                cells.add((k, (q0v + b) % npad, (q0u + a) % npad))
    return len(cells)


def test_covered_grid_cells_against_brute_force():
    rng = np.random.default_rng(5)
    npad, du = 64, 1.5
    n = 300
    uvw = np.column_stack([rng.uniform(-52, 52, n) * du, rng.uniform(-52, 52, n) * du,
                           rng.uniform(-40, 40, n)])
    uvw[:5, 0] = (npad / 2 - 0.5) * du      # boxes across the grid edge (circular)
    uvw[5:8, 1] = (npad / 2 + 2.0) * du     # outside the grid: dropped
    info = {"npad": npad, "du": du, "wbar": [3.0, 17.0, 33.0], "jw": [4, 6, 10]}
    for fold in (True, False):
        assert bench.covered_grid_cells(uvw, info, fold) == brute_cells(uvw, info, fold)

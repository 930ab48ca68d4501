"""Host-side logic of bench.py that needs no GPU: the count of grid cells the
kernel boxes cover (the grid part of the minimum HBM bytes), against
brute-force enumeration of every box; the DDE convolution's multiply-add
count, against enumeration of its terms."""
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


def test_dde_multiply_add_count_matches_enumeration():
    """The DDE roofline's work: the separable passes' complex multiply-adds,
    counted term by term (terms outside the box left out, as the kernels do)
    against the closed form bench.py uses."""
    for J in (2, 4, 8, 38):
        for jd in (1, 3, 5, 15):
            h = jd // 2
            Jc = J + 2 * h
            row = sum(1 for kb in range(J) for cu in range(Jc) for s in range(jd)
                      if 0 <= cu - 2 * h + s < J)
            col = sum(1 for cv in range(Jc) for cu in range(Jc)
                      for kb in range(max(0, cv - 2 * h), min(J - 1, cv) + 1))
            assert bench.dde_macs([1], [J], jd) == row + col
    assert bench.dde_macs([3, 2], [4, 8], 5) == 3 * bench.dde_macs([1], [4], 5) + \
        2 * bench.dde_macs([1], [8], 5)

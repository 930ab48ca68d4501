"""The plain FP64 operator on the tiny configuration exactly as specified:
128^2 image, 256^2 grid, FOV 20 deg, J = 4, one w-stack, 5,000 visibilities
with (u, v) uniform in a 60-wavelength disk and w uniform in [-40, 40],
complex128, 20 point sources at seed 0 (workloads.tiny()).

The FP64 GPU path (quadrature tolerance 1e-12) matches the FP64 oracle
(tolerance 1e-13) to 1e-10 relative L2 in degrid and grid; the FP32 path to
1e-5.  The method's own accuracy -- the gridded operator against the direct
measurement equation (Sec. 2) -- is reported beside it: the GPU's distance
from the direct equation equals the oracle's (5.1e-3 for J = 4, os = 2,
alpha = 1).  The oracle values come from tests/golden/tiny_fp64.npz, written
by tests/golden/make_tiny_fp64.py from oracle/ alone (3 minutes of oracle
time).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_fp64.npz")


@pytest.fixture(scope="module")
def tiny():
    g = dict(np.load(GOLDEN))
    wl = W.tiny()
    uvw = W.uvw_for(wl)
    assert len(uvw) == 5000
    assert np.allclose(np.abs(uvw).sum(axis=0), g["uvw_sums"], rtol=1e-12, atol=0)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    yv = W.random_vis(len(uvw), int(g["vis_seed"]))
    return wl, uvw, x, yv, g


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_tiny_config_matches_oracle(tiny, precision):
    wl, uvw, x, yv, g = tiny
    tol = 1e-12 if precision == "f64" else 1e-6
    plan = phi.Plan(torch.from_numpy(uvw), image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg),
                    oversample=wl.oversample, support=wl.support, n_stacks=wl.n_stacks,
                    conj_fold=int(wl.conj_fold), precision=precision, quad_rel_tol=tol,
                    quad_abs_tol=tol)
    info = plan.info()
    assert info["n_dropped"] == 0 and info["jw"] == [int(g["jw"])]
    rd = torch.float64 if precision == "f64" else torch.float32
    cd = torch.complex128 if precision == "f64" else torch.complex64
    y = plan.degrid(torch.from_numpy(x).cuda().to(rd)).cpu().numpy()
    img = plan.grid(torch.from_numpy(yv).cuda().to(cd)).cpu().numpy()
    gate = 1e-10 if precision == "f64" else 1e-5
    e_deg, e_grid = O.rel_l2(y, g["y_ref"]), O.rel_l2(img, g["img_ref"])
    assert e_deg < gate and e_grid < gate, (e_deg, e_grid)
    # the method's accuracy against the direct measurement equation: the
    # same as the oracle's (the operator is the same within the gate)
    e_method = O.rel_l2(y, g["y_direct"])
    e_method_oracle = O.rel_l2(g["y_ref"], g["y_direct"])
    print(f"tiny {precision}: degrid {e_deg:.2e}, grid {e_grid:.2e} vs the oracle; "
          f"{e_method:.3e} vs the direct equation (oracle {e_method_oracle:.3e})")
    assert abs(e_method - e_method_oracle) <= 2 * gate
    assert 1e-3 < e_method < 1e-2
    bad, _ = plan.stats()
    assert bad == 0
    plan.close()

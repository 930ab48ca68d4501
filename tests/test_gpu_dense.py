"""Full-density gridding and all-stack degridding on the MWA-like snapshot
(2048^2 image, 4096^2 grid, 8 stacks, fold on, FP32 with FP64 chirp phase)
against the FP64 oracle at quadrature tolerance 1e-12.

The oracle values come from tests/golden/mwa_dense_cells.npz, which
tests/golden/make_dense_cells.py writes from oracle/ alone (about 14 minutes
of oracle time, too long for a test).  For every stack it holds the busiest
grid cell of the full workload (960 to 2,552 contributions) and every kept
visibility whose tap box covers it; gridding those visibilities accumulates
that cell exactly as the full run does (Eq. stacked adjoint), in the FP32
atomics of the timed kernel.  Gate: relative L2 <= 1e-5 (the FP32 path's), on the
sub-observation built with the full plan's centres and supports, and on the
full plan in the bench's launch configuration.
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

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mwa_dense_cells.npz")
TOL32 = 1e-5


@pytest.fixture(scope="module")
def dense():
    g = dict(np.load(GOLDEN))
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    sel = g["dense_sel"]
    # the same baselines as the ones the oracle was run on
    assert np.allclose(np.abs(uvw[sel]).sum(axis=0), g["uvw_sums"], rtol=1e-12, atol=0)
    geo = O.geometry_from(wl, tol_rel=float(g["tol"]), tol_abs=float(g["tol"]))
    sub = np.ascontiguousarray(uvw[sel])
    op = O.make_plan(sub, geo, wl.n_stacks, wl.conj_fold, centres=g["centres"],
                     stack_jw=g["stack_jw"])
    # the oracle's image of the gridded values, stack by stack from its patches
    img_k = {}
    for k in range(wl.n_stacks):
        grid = np.zeros((geo.Npad, geo.Npad), np.complex128)
        J = int(g["stack_jw"][k])
        v0, u0 = (int(t) for t in g[f"dense_patch_origin_{k}"])
        rows = np.arange(v0, v0 + 2 * J - 1) % geo.Npad
        cols = np.arange(u0, u0 + 2 * J - 1) % geo.Npad
        grid[np.ix_(rows, cols)] = g[f"dense_patch_{k}"]
        img_k[k] = O.image_from_grids(op, {k: grid})
    y_in = W.random_vis(len(uvw), int(g["vis_seed"]))
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    kw = dict(image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg), oversample=wl.oversample,
              support=wl.support, n_stacks=wl.n_stacks, conj_fold=int(wl.conj_fold))
    return wl, uvw, g, op, img_k, y_in, x, kw


def per_stack_rel(a, b, stack, n):
    return [O.rel_l2(a[stack == k], b[stack == k]) for k in range(n)]


def test_dense_selection_reaches_full_density(dense):
    """Host check of the fixture: each stack's busiest cell receives as many
    contributions from the selected visibilities as the golden file states
    (960 to 2,552), i.e. its full-run count."""
    wl, uvw, g, op, _, _, _, _ = dense
    npad = op.geo.Npad
    for k in range(wl.n_stacks):
        s = op.stack == k
        J = int(g["stack_jw"][k])
        assert np.all(op.jw[s] == J) and not op.dropped[s].any()
        q0u = (np.floor(op.upix[s]).astype(np.int64) - J // 2 + 1) % npad
        q0v = (np.floor(op.vpix[s]).astype(np.int64) - J // 2 + 1) % npad
        cv, cu = (int(t) for t in g["dense_cell"][k])
        cover = (((cu - q0u) % npad) < J) & (((cv - q0v) % npad) < J)
        assert cover.all() and cover.sum() == int(g["dense_count"][k]) >= 900


def test_dense_sub_observation_matches_oracle(dense):
    """The selected visibilities as their own observation (fixed centres and
    supports of the full plan): degrid per stack and the gridded image."""
    wl, uvw, g, op, img_k, y_in, x, kw = dense
    sel = g["dense_sel"]
    plan = phi.Plan(torch.from_numpy(np.ascontiguousarray(uvw[sel])), centres=g["centres"],
                    stack_jw=g["stack_jw"], **kw)
    info = plan.info()
    assert list(info["jw"]) == [int(j) for j in g["stack_jw"]]
    assert list(info["counts"]) == [int(np.sum(op.stack == k)) for k in range(wl.n_stacks)]
    y = plan.degrid(torch.from_numpy(x).cuda().float()).cpu().numpy()
    assert O.rel_l2(y, g["dense_y_ref"]) < TOL32
    assert max(per_stack_rel(y, g["dense_y_ref"], op.stack, wl.n_stacks)) < TOL32
    img = plan.grid(torch.from_numpy(y_in[sel]).cuda().to(torch.complex64)).cpu().numpy()
    ref = sum(img_k.values())
    assert O.rel_l2(img, ref) < TOL32
    bad, _ = plan.stats()
    assert bad == 0
    plan.close()


def test_dense_cells_in_the_full_plan_match_oracle(dense):
    """The full plan (1.92M visibilities, the bench's launch configuration):
    gridding a visibility vector that is zero except on the selected
    visibilities, one stack at a time and all together; degridding the
    all-stack sample of 2,000 visibilities (250 per stack)."""
    wl, uvw, g, op, img_k, y_in, x, kw = dense
    plan = phi.Plan(torch.from_numpy(uvw), **kw)
    assert np.allclose(plan.info()["wbar"], g["centres"], rtol=1e-11, atol=1e-11)
    sel = g["dense_sel"]
    for k in list(range(wl.n_stacks)) + [None]:
        pick = sel if k is None else sel[op.stack == k]
        ym = np.zeros(len(uvw), np.complex64)
        ym[pick] = y_in[pick]
        img = plan.grid(torch.from_numpy(ym).cuda()).cpu().numpy()
        ref = sum(img_k.values()) if k is None else img_k[k]
        assert O.rel_l2(img, ref) < TOL32, k
    y = plan.degrid(torch.from_numpy(x).cuda().float()).cpu().numpy()
    s = g["sample_sel"]
    full = O.make_plan(uvw, op.geo, wl.n_stacks, wl.conj_fold)
    assert O.rel_l2(y[s], g["sample_y_ref"]) < TOL32
    assert max(per_stack_rel(y[s], g["sample_y_ref"], full.stack[s], wl.n_stacks)) < TOL32
    plan.close()

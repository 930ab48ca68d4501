"""Precision: FP32 (FP64 chirp phase) against the full-FP64 GPU path and the
FP64 oracle, on the precision-study workload (4096^2 image, 8192^2 grid,
17.5M visibilities, |w| <= 1500, 32 stacks, fold on) and on plans with given
centres (phi_plan_create_fixed)."""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_1903_06555_gb300 as phi
import workloads as W

pytestmark = pytest.mark.gpu


def test_fixed_centre_plan_matches_oracle_and_full_plan():
    geo = O.Geometry(128, 2.0, math.radians(20.0), 4.0, tol_rel=1e-13, tol_abs=1e-13)
    uvw = W.uvw_disk(1500, 60.0, 40.0, 31)
    x = W.point_sources(128, 20, 31)
    full = phi.Plan(torch.from_numpy(uvw), image_n=128, fov_rad=geo.fov, n_stacks=4, conj_fold=1,
                    precision="f64", quad_rel_tol=1e-12, quad_abs_tol=1e-12)
    info = full.info()
    y_full = full.degrid(torch.from_numpy(x).cuda()).cpu().numpy()
    sel = np.sort(np.random.default_rng(1).choice(1500, 300, replace=False))
    sub = phi.Plan(torch.from_numpy(np.ascontiguousarray(uvw[sel])), image_n=128, fov_rad=geo.fov,
                   n_stacks=4, conj_fold=1, precision="f64", quad_rel_tol=1e-12,
                   quad_abs_tol=1e-12, centres=info["wbar"], stack_jw=info["jw"])
    y_sub = sub.degrid(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(y_sub, y_full[sel])
    op = O.make_plan(uvw[sel], geo, 4, True, centres=info["wbar"], stack_jw=info["jw"])
    assert O.rel_l2(y_sub, O.degrid(op, x)) < 1e-10


@pytest.fixture(scope="module")
def precision_workload():
    wl = W.precision_study()
    uvw = W.uvw_for(wl)
    kw = dict(image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg), n_stacks=wl.n_stacks,
              conj_fold=int(wl.conj_fold))
    plan = phi.Plan(torch.from_numpy(uvw), **kw)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    y32 = plan.degrid(torch.from_numpy(x).cuda().float()).cpu().numpy()
    return wl, uvw, kw, plan.info(), x, y32


def test_precision_study_fp32_vs_fp64_and_oracle(precision_workload):
    """17.5M visibilities in FP32 at full size; a 20,000-visibility
    sub-observation with the same centres and supports (hence the same
    operator) in FP32 and FP64; the FP64 oracle on 120 of them from two
    stacks.  FP32 vs FP64 <= 1e-5, FP64 vs oracle <= 1e-10."""
    wl, uvw, kw, info, x, y32 = precision_workload
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(uvw), 20000, replace=False))
    sub = np.ascontiguousarray(uvw[sel])
    p32 = phi.Plan(torch.from_numpy(sub), centres=info["wbar"], stack_jw=info["jw"], **kw)
    p64 = phi.Plan(torch.from_numpy(sub), centres=info["wbar"], stack_jw=info["jw"],
                   precision="f64", quad_rel_tol=1e-12, quad_abs_tol=1e-12, **kw)
    s32 = p32.degrid(torch.from_numpy(x).cuda().float()).cpu().numpy()
    s64 = p64.degrid(torch.from_numpy(x).cuda()).cpu().numpy()
    # Same operator as the full plan, except for visibilities that sit within
    # Algorithm 1's last centre shift of a stack boundary: their nearest final
    # centre differs from the stack the last sweep gave them.
    wf, _ = O.fold(uvw)
    last, cen, _ = O.kmeans(wf[:, 2], wl.n_stacks)
    assert np.allclose(cen, info["wbar"], rtol=1e-11, atol=1e-11)
    nearest = np.argmin((cen[None, :] - wf[sel, 2:3]) ** 2, axis=1)
    moved = nearest != last[sel]
    same = s32 == y32[sel]
    assert np.all(same[~moved]) and moved.mean() < 0.02
    assert O.rel_l2(s32, s64) < 1e-5
    geo = O.geometry_from(wl, tol_rel=1e-13, tol_abs=1e-13)
    op = O.make_plan(sub, geo, wl.n_stacks, wl.conj_fold, centres=info["wbar"],
                     stack_jw=info["jw"])
    pick = np.concatenate([np.nonzero((op.stack == k) & ~op.dropped)[0][:60] for k in (3, 20)])
    ref = O.degrid(op, x, subset=pick)
    assert O.rel_l2(s64[pick], ref) < 1e-10
    assert O.rel_l2(s32[pick], ref) < 1e-5


def test_fp32_error_estimate_decides_like_fp64():
    """The adaptive quadrature's accept/refine decisions (Sec. 4 tolerance
    1e-6) taken from the FP32 error estimate equal those of the FP64 path.

    Both precisions start every chunk of taps from the same a-priori panel
    count (computed in FP32 from the same inputs) and double it while any
    tap's estimate exceeds max(abs_tol, rel_tol |K|); the FP64 path forms
    the estimate from FP64 node values, J0 and sums.  Equal tap-node totals
    over the same visibilities therefore mean that no chunk was refined by
    one precision and accepted by the other; the difference bounds how many
    were.  Either way the result stays within the tolerance: a refined chunk
    is only more accurate.  Workload: 4,000 kept
    visibilities of the MWA-like snapshot (all 8 stacks, J_w 26-36), degrid
    and grid, with the full plan's centres and supports."""
    g = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             "mwa_dense_cells.npz"))
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    sel = W.subsample(len(uvw), 4000, 17)
    sub = torch.from_numpy(np.ascontiguousarray(uvw[sel]))
    kw = dict(image_n=wl.image_n, fov_rad=math.radians(wl.fov_deg), n_stacks=wl.n_stacks,
              conj_fold=int(wl.conj_fold), centres=g["centres"], stack_jw=g["stack_jw"],
              quad_rel_tol=1e-6, quad_abs_tol=1e-6)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    y = W.random_vis(len(sel), 3)
    counts = {}
    for prec, rd, cd in (("f32", torch.float32, torch.complex64),
                         ("f64", torch.float64, torch.complex128)):
        plan = phi.Plan(sub, precision=prec, **kw)
        plan.degrid(torch.from_numpy(x).cuda().to(rd))
        plan.grid(torch.from_numpy(y).cuda().to(cd))
        counts[prec] = plan.stats_full()
        plan.close()
    print("FP32 (unconverged, taps, tap-nodes):", counts["f32"], " FP64:", counts["f64"])
    assert counts["f32"][1] == counts["f64"][1] > 0
    assert counts["f32"][0] == counts["f64"][0] == 0
    # The FP32 panel sums carry rounding of order 2^-24 sum_j |w_j h_j J_j|
    # (~6e-8 summed over the panels, against the 1e-6 tolerance), so a chunk
    # whose estimate lies within a few percent of the limit can be refined by
    # one precision only: measured 1.5e-4 of the tap-nodes on this workload
    # (64-tap chunks), FP32 the one refining more.  One differing decision
    # moves ~31 npan x 64 tap-nodes (~1e-5 of the total); the bound allows
    # about 100.
    assert abs(counts["f32"][2] - counts["f64"][2]) <= 1e-3 * counts["f64"][2]

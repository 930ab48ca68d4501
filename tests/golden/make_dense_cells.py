"""Write tests/golden/mwa_dense_cells.npz: FP64 oracle results for the
full-density gridding check and the all-stack degrid sample of the MWA-like
snapshot workload (2048^2 image, 4096^2 grid, 8 stacks, fold on).

Gridding (Eq. stacked adjoint) accumulates, into each cell of a stack's
padded grid, the taps of every visibility whose J_w x J_w box covers it.  In
the full workload the busiest cell of each stack receives 960 to 2,552 such
contributions.  For every stack this script finds that cell (ties: lowest
flat index) and selects every kept visibility of the stack whose box covers
it, so that in a sub-observation of the selected visibilities alone the cell
is accumulated exactly as in the full run.  With the full plan's centres and
per-stack supports (Algorithm 1 on all visibilities) the sub-observation's
operator is the full operator restricted to those visibilities.

Stored (all from oracle/ at quadrature tolerance 1e-12, relative and
absolute):
  centres, stack_jw       the full oracle plan's w-stack centres and supports
  dense_sel               selected visibility indices into the workload
  dense_cell, dense_count per stack: the busiest cell (v, u) and its count
  dense_y_ref             degrid of the workload image at dense_sel
  dense_patch_*           per stack, the oracle's grid of the random visibility
                          values W.random_vis(M, 9)[dense_sel] on the
                          (2 J_w - 1)^2 cells around the busiest cell (all its
                          nonzero cells; origin may be negative: indices wrap
                          mod Npad); the image follows by
                          oracle.image_from_grids
  sample_sel, sample_y_ref  250 random kept visibilities of every stack and
                          their degrid values
  uvw_sums                sums of |u|, |v|, |w| over dense_sel (the test
                          checks that it regenerates the same baselines)

Calls only oracle/ and workloads/.  Runs in about 15 minutes on 8 cores.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mwa_dense_cells.npz")
TOL = 1e-12
VIS_SEED = 9          # W.random_vis(M, VIS_SEED) are the gridded values
SAMPLE_PER_STACK = 250


def box_origin(plan, idx, npad):
    """First tap (q0u, q0v) of each visibility's box, mod npad:
    floor(u/du) - J_w/2 + 1 (J_w even)."""
    J = plan.jw[idx].astype(np.int64)
    q0u = (np.floor(plan.upix[idx]).astype(np.int64) - J // 2 + 1) % npad
    q0v = (np.floor(plan.vpix[idx]).astype(np.int64) - J // 2 + 1) % npad
    return q0u, q0v


def contributions(q0u, q0v, J, npad):
    """Per grid cell, the number of boxes (side J, origins q0) covering it."""
    cnt = np.zeros((npad, npad), np.int64)
    np.add.at(cnt, (q0v, q0u), 1)
    # cell c is covered by origins c - J + 1 .. c: a wrapped box sum
    ext = np.concatenate([cnt[npad - (J - 1):], cnt], axis=0)
    ext = np.concatenate([ext[:, npad - (J - 1):], ext], axis=1)
    cs = np.pad(np.cumsum(np.cumsum(ext, 0), 1), ((1, 0), (1, 0)))
    return cs[J:, J:] - cs[:-J, J:] - cs[J:, :-J] + cs[:-J, :-J]


def main():
    t0 = time.time()
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    M = len(uvw)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    yv = W.random_vis(M, VIS_SEED)
    geo = O.geometry_from(wl, tol_rel=TOL, tol_abs=TOL)
    npad = geo.Npad
    plan = O.make_plan(uvw, geo, wl.n_stacks, wl.conj_fold)
    kept = ~plan.dropped
    stack_jw = np.array([int(plan.jw[kept & (plan.stack == k)].max()) for k in range(wl.n_stacks)],
                        np.int32)
    sel_all, cells, counts = [], [], []
    for k in range(wl.n_stacks):
        idx = np.nonzero(kept & (plan.stack == k))[0]
        J = int(stack_jw[k])
        q0u, q0v = box_origin(plan, idx, npad)
        c = contributions(q0u, q0v, J, npad)
        cv, cu = np.unravel_index(int(np.argmax(c)), c.shape)
        cover = (((cu - q0u) % npad) < J) & (((cv - q0v) % npad) < J)
        assert int(cover.sum()) == int(c[cv, cu])
        sel_all.append(idx[cover])
        cells.append((cv, cu))
        counts.append(int(c[cv, cu]))
        print(f"stack {k}: J_w {J}, busiest cell (v, u) = ({cv}, {cu}) with {c[cv, cu]} "
              f"contributions", flush=True)
    dense = np.sort(np.concatenate(sel_all))
    stacks = list(range(wl.n_stacks))
    grids = O.stack_grids(plan, x, stacks)
    print(f"{dense.size} dense visibilities; degrid ...", flush=True)
    y_ref, _, bad1 = O.degrid_from_grids(plan, grids, dense, TOL, TOL)
    print(f"  {time.time() - t0:.0f} s; grid ...", flush=True)
    g, _, bad2 = O.grid_to_stacks(plan, yv[dense], dense, TOL, TOL)
    print(f"  {time.time() - t0:.0f} s; all-stack sample ...", flush=True)
    rng = np.random.default_rng(11)
    sample = np.sort(np.concatenate([
        rng.choice(np.nonzero(kept & (plan.stack == k))[0], SAMPLE_PER_STACK, replace=False)
        for k in stacks]))
    s_ref, _, bad3 = O.degrid_from_grids(plan, grids, sample, TOL, TOL)
    assert bad1 == bad2 == bad3 == 0
    out = dict(centres=plan.wbar, stack_jw=stack_jw, dense_sel=dense.astype(np.int64),
               dense_cell=np.array(cells, np.int64), dense_count=np.array(counts, np.int64),
               dense_y_ref=y_ref, sample_sel=sample.astype(np.int64), sample_y_ref=s_ref,
               uvw_sums=np.abs(uvw[dense]).sum(axis=0), tol=np.float64(TOL),
               vis_seed=np.int64(VIS_SEED))
    for k, gk in g.items():
        # every selected box covers the busiest cell, so all of the stack's
        # gridded cells lie in the (2 J_w - 1)^2 square around it (wrapped)
        J = int(stack_jw[k])
        v0, u0 = cells[k][0] - J + 1, cells[k][1] - J + 1
        rows = np.arange(v0, v0 + 2 * J - 1) % npad
        cols = np.arange(u0, u0 + 2 * J - 1) % npad
        patch = gk[np.ix_(rows, cols)]
        assert np.count_nonzero(patch) == np.count_nonzero(gk)
        out[f"dense_patch_{k}"] = patch
        out[f"dense_patch_origin_{k}"] = np.array([v0, u0], np.int64)
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT} ({os.path.getsize(OUT) / 1e6:.2f} MB) in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()

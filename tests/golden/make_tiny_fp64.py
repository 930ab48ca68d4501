"""Write tests/golden/tiny_fp64.npz: the FP64 oracle on the plain FP64
operator's tiny configuration (128^2 image, 256^2 grid, FOV 20 deg, J = 4,
one w-stack, 5,000 visibilities with (u, v) uniform in a 60-wavelength disk
and w uniform in [-40, 40], 20 point sources; workloads.tiny()).

Stored:
  y_ref     y = Phi x of the point-source image, oracle at quadrature
            tolerance 1e-13 (relative and absolute)
  img_ref   x = Re(Phi^H y) of the random visibilities W.random_vis(5000, 1),
            same tolerance
  y_direct  the direct measurement equation (Sec. 2) on the same image: the
            method's own accuracy is the distance of y_ref from it
  uvw_sums  sums of |u|, |v|, |w| (the test checks it regenerates them)

Calls only oracle/ and workloads/.  Runs in about 3 minutes on 8 cores.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_fp64.npz")
TOL = 1e-13
VIS_SEED = 1


def main():
    t0 = time.time()
    wl = W.tiny()
    uvw = W.uvw_for(wl)
    x = W.point_sources(wl.image_n, wl.n_sources, wl.seed)
    yv = W.random_vis(len(uvw), VIS_SEED)
    geo = O.geometry_from(wl, tol_rel=TOL, tol_abs=TOL)
    plan = O.make_plan(uvw, geo, wl.n_stacks, wl.conj_fold)
    y_ref = O.degrid(plan, x)
    img_ref = O.grid(plan, yv)
    y_direct = O.direct(x, uvw, geo)
    np.savez_compressed(OUT, y_ref=y_ref, img_ref=img_ref, y_direct=y_direct,
                        uvw_sums=np.abs(uvw).sum(axis=0), tol=np.float64(TOL),
                        vis_seed=np.int64(VIS_SEED), jw=np.int64(plan.jw.max()))
    print(f"wrote {OUT} ({os.path.getsize(OUT) / 1e3:.0f} kB) in {time.time() - t0:.0f} s; "
          f"method error vs the direct equation {O.rel_l2(y_ref, y_direct):.3e}")


if __name__ == "__main__":
    main()

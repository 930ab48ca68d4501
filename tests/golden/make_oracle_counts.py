"""Write tests/golden/mwa_oracle_evals.json: the oracle's integrand
evaluations per visibility at the paper's quadrature tolerance (1e-6
relative and absolute, Sec. 4) on the MWA-like snapshot workload, per w-stack.

The oracle integrates every tap separately by globally adaptive Gauss-Kronrod
bisection, so its evaluation count is the algorithmic work of the kernel
quadrature (tap-node integrand evaluations) independent of how the GPU shares
nodes between taps.  Calls only oracle/ and workloads/.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main(per_stack=60):
    wl = W.mwa_snapshot()
    uvw = W.uvw_for(wl)
    geo = O.geometry_from(wl, tol_rel=1e-6, tol_abs=1e-6)
    plan = O.make_plan(uvw, geo, wl.n_stacks, wl.conj_fold)
    rng = np.random.default_rng(7)
    out = {"source": "oracle integrand evaluations per visibility at tol 1e-6 (Sec. 4), "
                     "MWA-like snapshot workload; written by tests/golden/make_oracle_counts.py",
           "workload": wl.name, "stacks": []}
    t0 = time.time()
    for k in range(wl.n_stacks):
        idx = np.nonzero((plan.stack == k) & ~plan.dropped)[0]
        sel = rng.choice(idx, size=min(per_stack, idx.size), replace=False)
        evals = []
        for i in sel:
            J = int(plan.jw[i])
            q0u = np.floor(plan.upix[i]) - J // 2 + 1      # floor(u - J/2) + 1, exact for even J
            q0v = np.floor(plan.vpix[i]) - J // 2 + 1
            a = np.arange(J)
            du_ = plan.upix[i] - (q0u + a)
            dv_ = plan.vpix[i] - (q0v + a)
            rho = np.hypot(du_[None, :], dv_[:, None]).ravel()
            _, ev, bad = O.wkernel(rho, np.full(rho.size, plan.dw[i]), geo, return_stats=True)
            evals.append(ev)
        out["stacks"].append({"stack": k, "n_kept": int(idx.size), "jw": int(plan.jw[idx[0]]),
                              "sampled": int(sel.size),
                              "evals_per_vis": float(np.mean(evals))})
    tot = sum(s["n_kept"] for s in out["stacks"])
    out["evals_per_vis_mean"] = sum(s["n_kept"] * s["evals_per_vis"] for s in out["stacks"]) / tot
    out["n_kept"] = tot
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mwa_oracle_evals.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1), f"\n{time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()

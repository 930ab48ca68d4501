"""The allocation-free kernel evaluator, phi_wkernel_noalloc.

It serves callers that must not allocate device memory once running (their
GPU memory belongs to another allocator, or an allocation's implicit device
synchronisation would stall a real-time pipeline).  It keeps its scratch in
a fixed array inside the library instead of a plan.  This file runs last so
that a run stopping at the first failure has already run every other test;
it passes alone in a fresh process as well as after the rest.

Checked through the C ABI against phi_wkernel, the plan-based evaluator of
the same quadrature, on two calls in a row (the second must not see the
first's leftovers), at the tolerances of the other GPU kernel tests.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import paper_1903_06555_gb300 as phi
import workloads as W

pytestmark = pytest.mark.gpu


def _plan_and_params(precision):
    tol = 1e-12 if precision == "f64" else 1e-6
    cpp = 3.4 if precision == "f64" else 6.0   # the plans' default widths at these tolerances
    uvw = W.uvw_disk(16, 60.0, 40.0, 0)
    plan = phi.Plan(torch.from_numpy(uvw), image_n=128, fov_rad=math.radians(20.0),
                    n_stacks=1, precision=precision, quad_rel_tol=tol, quad_abs_tol=tol,
                    cycles_per_panel=cpp)
    info = plan.info()
    prm = phi.WKernelParams(du=info["du"], window_radius=info["window_radius"],
                            kb_beta=info["beta"], quad_rel_tol=tol, quad_abs_tol=tol,
                            cycles_per_panel=cpp, support=4, max_refine=3,
                            max_panels=phi.WKERNEL_NOALLOC_MAX_PANELS,
                            precision=phi.PHI_F64 if precision == "f64" else phi.PHI_F32)
    return plan, prm


def _raw_call(prm, rho, dw):
    """Call the C entry point with caller-owned buffers only."""
    cd = torch.complex128 if prm.precision == phi.PHI_F64 else torch.complex64
    out = torch.empty(rho.numel(), dtype=cd, device="cuda")
    bad = ctypes.c_int64(-1)
    st = phi.lib().phi_wkernel_noalloc(ctypes.byref(prm), ctypes.c_void_p(rho.data_ptr()),
                                       ctypes.c_void_p(dw.data_ptr()), rho.numel(),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.byref(bad),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out, bad.value


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_noalloc_matches_plan_evaluator_twice(precision):
    plan, prm = _plan_and_params(precision)
    tol = 1e-11 if precision == "f64" else 1e-5
    rng = np.random.default_rng(5)
    for call in range(2):
        rho = np.concatenate([[0.0, 2.0], rng.uniform(0, 25, 400)])
        dw = np.concatenate([[0.0, -30.0], rng.uniform(-120, 120, 400)]) * (1 + call)
        rt = torch.from_numpy(rho).cuda()
        dt = torch.from_numpy(dw).cuda()
        ref, bad_ref = plan.wkernel(rt, dt)
        st, got, bad = _raw_call(prm, rt, dt)
        assert st == phi.PHI_OK
        assert bad == bad_ref == 0
        assert torch.max(torch.abs(got - ref)).item() <= tol
    plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    _, prm = _plan_and_params("f32")
    prm.max_panels = phi.WKERNEL_NOALLOC_MAX_PANELS + 1
    rho = torch.zeros(4, dtype=torch.float64, device="cuda")
    st, _, _ = _raw_call(prm, rho, rho)
    assert st == phi.PHI_ERR_ARG


def test_noalloc_counts_points_beyond_its_panel_cap():
    """With max_panels = 2 the wide chirps of large |dw| cannot meet the
    tolerance: the points are evaluated on the capped partition (finite
    values) and counted; the Python wrapper and the raw C call agree."""
    _, prm = _plan_and_params("f32")
    prm.max_panels = 2
    rng = np.random.default_rng(9)
    rt = torch.from_numpy(rng.uniform(5, 20, 64)).cuda()
    dt = torch.from_numpy(rng.uniform(200, 400, 64)).cuda()
    st, raw, bad = _raw_call(prm, rt, dt)
    assert st == phi.PHI_OK
    assert 0 < bad <= 64
    assert torch.isfinite(torch.view_as_real(raw)).all()
    k, bad_w = phi.wkernel_noalloc(prm, rt, dt)
    assert bad_w == bad
    assert torch.equal(k, raw)

"""The C-ABI library builds, loads and exports every symbol include/phi.h
declares; the Python mirrors of its structs match the C layout; host-side
validation rejects bad descriptors before touching a device (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

import paper_1903_06555_gb300 as phi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "phi.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(phi_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = phi.lib()
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(L, n), n


def test_no_oracle_in_product():
    """The product never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1903_06555_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f
    out = subprocess.run(["nm", "-D", phi.lib_path()], capture_output=True, text=True).stdout
    assert "orc_" not in out


def _c_layout():
    code = r"""
#include <stddef.h>
#include <stdio.h>
#include "phi.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("phi_plan_desc %zu\n", sizeof(phi_plan_desc));
  printf("phi_plan_summary %zu\n", sizeof(phi_plan_summary));
  O(phi_plan_desc, tile); O(phi_plan_desc, oversample); O(phi_plan_desc, cycles_per_panel);
  O(phi_plan_summary, image_n); O(phi_plan_summary, du); O(phi_plan_summary, support_coeff);
  O(phi_plan_summary, kernel_mode); O(phi_plan_summary, table_n_rho); O(phi_plan_summary, table_h_w);
  O(phi_plan_desc, kernel_mode); O(phi_plan_desc, table_tol); O(phi_plan_desc, max_grid_mib);
  O(phi_plan_desc, grid_deterministic); O(phi_plan_summary, group);
  printf("phi_wkernel_params %zu\n", sizeof(phi_wkernel_params));
  O(phi_wkernel_params, cycles_per_panel); O(phi_wkernel_params, precision);
  return 0;
}
"""
    tmp = os.path.join(os.environ.get("TMPDIR", "/tmp"), f"phi_layout_{os.getpid()}")
    with open(tmp + ".c", "w") as f:
        f.write(code)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), tmp + ".c", "-o", tmp], check=True)
    out = subprocess.run([tmp], capture_output=True, text=True, check=True).stdout
    os.remove(tmp)
    os.remove(tmp + ".c")
    return dict(line.rsplit(" ", 1) for line in out.strip().splitlines())


def test_struct_layout_matches_c():
    lay = _c_layout()
    assert int(lay["phi_plan_desc"]) == ctypes.sizeof(phi.PlanDesc)
    assert int(lay["phi_plan_summary"]) == ctypes.sizeof(phi.PlanSummary)
    assert int(lay["phi_wkernel_params"]) == ctypes.sizeof(phi.WKernelParams)
    classes = {"phi_plan_desc": phi.PlanDesc, "phi_plan_summary": phi.PlanSummary,
               "phi_wkernel_params": phi.WKernelParams}
    for key, val in lay.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(classes[t], f).offset == int(val), key


def test_defaults_and_error_strings():
    d = phi.default_desc()
    assert d.support == 4 and d.kmeans_max_iter == 100 and d.kmeans_tol == 1e-3
    assert d.quad_rel_tol == 1e-6 and d.quad_abs_tol == 1e-6 and d.alpha == 1.0
    assert d.max_support == 64 and d.precision == phi.PHI_F32
    assert d.kernel_mode == phi.PHI_KERNEL_QUADRATURE and d.table_tol == 1e-4
    assert d.grid_staging == 0
    L = phi.lib()
    assert L.phi_error_string(0) == b"ok"
    for s in range(1, 8):
        assert L.phi_error_string(s) not in (b"ok", b"unknown status")
    assert L.phi_error_string(99) == b"unknown status"


BAD = [dict(image_n=127), dict(image_n=0), dict(support=3), dict(n_stacks=0),
       dict(n_stacks=200), dict(precision=5), dict(oversample=1.25), dict(fov_rad=-1.0),
       dict(max_support=2), dict(quad_rel_tol=0.0), dict(support_rule=3), dict(max_refine=-1),
       dict(kernel_mode=3), dict(kernel_mode=1, table_tol=0.0), dict(grid_staging=2),
       dict(kernel_mode=2, grid_staging=1),
       dict(grid_staging=1), dict(max_grid_mib=-1), dict(grid_deterministic=2),
       dict(grid_deterministic=1, kernel_mode=1, grid_staging=1)]


@pytest.mark.parametrize("bad", BAD)
def test_invalid_descriptors_rejected_on_host(bad):
    kw = dict(image_n=128, fov_rad=0.35, n_stacks=1)
    kw.update(bad)
    d = phi.default_desc(**kw)
    h = ctypes.c_void_p(123)
    st = phi.lib().phi_plan_create(ctypes.byref(h), ctypes.byref(d), None, None, 0, None)
    assert st == phi.PHI_ERR_ARG
    assert h.value is None


def test_horizon_rejected_on_host():
    # window radius R/du = os * fov / 2 >= 1
    d = phi.default_desc(image_n=128, fov_rad=1.2, n_stacks=1)
    h = ctypes.c_void_p()
    assert phi.lib().phi_plan_create(ctypes.byref(h), ctypes.byref(d), None, None, 0, None) \
        == phi.PHI_ERR_HORIZON


def test_null_handles_rejected():
    L = phi.lib()
    assert L.phi_degrid(None, None, None, None) == phi.PHI_ERR_ARG
    assert L.phi_grid(None, None, None, None) == phi.PHI_ERR_ARG
    assert L.phi_wkernel(None, None, None, 0, None, None, None) == phi.PHI_ERR_ARG
    assert L.phi_degrid_dde(None, None, None, None, 5, None, None) == phi.PHI_ERR_ARG
    assert L.phi_grid_dde(None, None, None, None, 5, None, None) == phi.PHI_ERR_ARG
    assert L.phi_plan_info(None, None, None, None, None) == phi.PHI_ERR_ARG
    L.phi_plan_destroy(None)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_no_device_is_an_error_not_a_fallback():
    d = phi.default_desc(image_n=128, fov_rad=0.35, n_stacks=1)
    h = ctypes.c_void_p()
    st = phi.lib().phi_plan_create(ctypes.byref(h), ctypes.byref(d), None, None, 0, None)
    assert st == phi.PHI_ERR_CUDA
    with pytest.raises(Exception):
        phi.Plan(torch.zeros(4, 3, dtype=torch.float64), image_n=128, fov_rad=0.35)


def test_binding_constants_match_the_header():
    """The Python binding's copies of the header's #define limits."""
    import re
    text = open(os.path.join(ROOT, "include", "phi.h")).read()
    m = re.search(r"#define PHI_WKERNEL_NOALLOC_MAX_PANELS (\d+)", text)
    assert m and int(m.group(1)) == phi.WKERNEL_NOALLOC_MAX_PANELS

"""Host logic of the serving engine that needs no GPU: the admission estimate
charges the padded grids of a plan's whole stack group (up to max_grid_mib),
the most stacks a raised request can reach, and only inputs and outputs for
a resident plan."""
import math

import numpy as np

from paper_1903_06555_gb300 import serve as S


def req(n, k, m=10000, raise_stacks=False, **desc):
    d = dict(image_n=n, fov_rad=math.radians(20.0), n_stacks=k)
    d.update(desc)
    return S.Request(0, np.zeros((m, 3)), d, raise_stacks=raise_stacks)


def test_grids_of_the_whole_group_are_charged():
    grid = 8 * 1024 * 1024                      # 512^2 image, 1024^2 complex64 grid
    e1, e8, e64 = (S.estimate_bytes(req(512, k)) for k in (1, 8, 64))
    assert e8 - e1 == 2 * 7 * grid              # group grids + batched workspace
    assert e64 - e8 == 2 * 56 * grid


def test_group_is_capped_by_max_grid_mib():
    grid = 8 * 16384 * 16384                    # 8192^2 image: 2 GiB per grid
    e2, e64 = (S.estimate_bytes(req(8192, k)) for k in (2, 64))
    assert e64 == e2                            # 4 GiB default: 2 grids per group
    small_cap = S.estimate_bytes(req(8192, 64, max_grid_mib=2048))
    assert e2 - small_cap == 2 * grid


def test_raised_requests_are_charged_for_126_stacks():
    assert S.estimate_bytes(req(512, 4, raise_stacks=True)) == S.estimate_bytes(req(512, 126))


def test_resident_plan_charges_inputs_and_outputs_only():
    r = req(512, 8, m=20000)
    io = 20000 * 2 * 8 + 512 * 512 * 2 * 4 + (16 << 20)
    assert S.estimate_bytes(r, planned=True) == io
    r64 = req(512, 8, m=20000, precision="f64")
    assert S.estimate_bytes(r64, planned=True) == 20000 * 2 * 16 + 512 * 512 * 2 * 8 + (16 << 20)


def test_padded_grid_size_rounds_halves_up_like_the_library():
    """The plan sizes its grid as lround(os * N), halves away from zero:
    os = 2.5, N = 77 gives 192.5 -> 193 (Python's round() would give 192)."""
    r = req(77, 1, oversample=2.5)
    grid_193, grid_192 = 8 * 193 * 193, 8 * 192 * 192
    base = S.estimate_bytes(req(77, 1, oversample=2.5 - 1e-9))   # 192.49... -> 192
    # one stack: its grid, one batched-transform workspace grid, one more
    assert S.estimate_bytes(r) - base == 3 * (grid_193 - grid_192)


def test_deterministic_plans_are_charged_for_their_fixed_point_grids():
    """grid_deterministic adds two int64 per cell of each resident grid and
    counts them against max_grid_mib when sizing the stack group."""
    grid = 8 * 1024 * 1024                      # 512^2 image, 1024^2 complex64 grid
    fixed = 16 * 1024 * 1024
    assert (S.estimate_bytes(req(512, 8, grid_deterministic=1)) -
            S.estimate_bytes(req(512, 8)) == 8 * fixed)
    # 8192^2 image: a 2 GiB grid and 4 GiB of sums per stack exceed the 4 GiB
    # default, so one stack per group: 3 grids + 1 set of sums, against
    # 5 grids for the plain plan's groups of 2
    big = 8 * 16384 * 16384
    e_plain = S.estimate_bytes(req(8192, 64))
    e_det = S.estimate_bytes(req(8192, 64, grid_deterministic=1))
    assert e_det - e_plain == (3 * big + 2 * big) - 5 * big
    assert (S.estimate_bytes(req(8192, 1, grid_deterministic=1)) -
            S.estimate_bytes(req(8192, 1)) == 2 * big)

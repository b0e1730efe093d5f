"""The single-launch step (volume and face / update work of one solve in one
cooperative persistent kernel, tiles published and awaited through readiness
values) against the two-kernel step it replaces.

Both run the same per-tile arithmetic (the fused kernel reads the other CTAs'
records through L2); the compiler may contract or order a few operations
differently in the larger kernel, so the increments of every chunk of steps
must agree to round-off of the increment (FP64 1e-12, FP32 1e-4, relative
L2 and per-variable nodal maximum) and dt to 1e-14 / 1e-6.  A missing or early
readiness value would let a tile read another step's records, an error of the
size of the increment itself.  Cases: meshes with many tiles per CTA, tiles
whose neighbours wrap around the periodic box, ragged last tiles, long runs.
The single-launch form is selected with CRKFR_STEP_KERNELS=fused when a
context is created (the two kernels are the default: the single launch
measured slower).
"""
import os

import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs
from parity_util import check_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return crkfr


def _solver(cr, mesh, prec, split):
    old = os.environ.get("CRKFR_STEP_KERNELS")
    try:
        if split:
            os.environ.pop("CRKFR_STEP_KERNELS", None)
        else:
            os.environ["CRKFR_STEP_KERNELS"] = "fused"
        return cr.Solver(mesh, prec=prec)
    finally:
        if old is None:
            os.environ.pop("CRKFR_STEP_KERNELS", None)
        else:
            os.environ["CRKFR_STEP_KERNELS"] = old


# long runs in FP64, where the two forms' rounding differences stay at 1e-16 and
# a stale record would stand out; FP32 over a few steps (its rounding
# differences grow chaotically over long runs)
CASES = [("shear256_N3", "fp32", 3), ("shear256_N3", "fp64", 40), ("smooth2d_N2_odd", "fp64", 300),
         ("smooth2d_N2_odd", "fp32", 3), ("smooth2d_N5", "fp32", 3), ("smooth2d_N5", "fp64", 30),
         ("smooth2d_N4", "fp64", 30), ("wave1d_N3_long", "fp64", 300), ("wave1d_N3_long", "fp32", 3),
         ("tgv3d_N3", "fp32", 3), ("tgv3d_N2", "fp64", 50), ("strip2d_N3", "fp64", 100), ("single2d_N3", "fp64", 50),
         ("single2d_N3", "fp32", 3)]


def _case(name):
    if name == "shear256_N3":
        return inputs.shear_layer_2d(cells=(256, 256), N=3)
    if name == "smooth2d_N2_odd":   # 33 x 37: tiles straddle rows, neighbours wrap inside a tile
        mesh = inputs.mesh_dict("euler", 2, 2, [33, 37], [0, 0], [1.0, 1.1], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=61, amp=0.2)
    if name == "smooth2d_N5":
        mesh = inputs.mesh_dict("euler", 2, 5, [40, 24], [0, 0], [1.0, 1.0], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=62, amp=0.2)
    if name == "smooth2d_N4":
        mesh = inputs.mesh_dict("euler", 2, 4, [48, 40], [0, 0], [1.0, 1.0], 1.4, vol="kep")
        return mesh, inputs.smooth_random_field(mesh, seed=63, amp=0.2)
    if name == "wave1d_N3_long":
        return inputs.density_wave_1d(cells=5000, N=3)
    if name == "tgv3d_N3":
        return inputs.tgv_3d(cells=(24, 20, 16), N=3, mach=0.3)
    if name == "tgv3d_N2":
        return inputs.tgv_3d(cells=(17, 9, 11), N=2, mach=0.3)
    if name == "strip2d_N3":       # one element across y: the y neighbours are the element itself
        mesh = inputs.mesh_dict("euler", 2, 3, [200, 1], [0, 0], [2.0, 0.1], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=64, amp=0.2)
    if name == "single2d_N3":
        mesh = inputs.mesh_dict("euler", 2, 3, [1, 1], [0, 0], [1.0, 1.0], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=65, amp=0.2)
    raise KeyError(name)


@pytest.mark.parametrize("name,prec,steps", CASES)
def test_fused_equals_split(cr, name, prec, steps):
    mesh, U = _case(name)
    fused = _solver(cr, mesh, prec, split=False)
    split = _solver(cr, mesh, prec, split=True)
    assert fused.tuning_info()["step"] == "fused"
    assert split.tuning_info()["step"] == "split"
    for s in (fused, split):
        s.set_state(U)
    a0, b0 = U, U
    # FP32: the flux-differencing sums cancel about 1e2-fold, so one ulp of a
    # pair flux moves a node's increment by about 1e-5 of its largest value
    tol = 1e-12 if prec == "fp64" else 1e-4
    done = 0
    for chunk in (1, 2, 16, steps):        # single-step and 16-step graphs, every phase
        n = min(chunk, steps - done)
        if n <= 0:
            break
        fused.step(n)
        split.step(n)
        done += n
        a, b = fused.get_state(), split.get_state()
        ia, ib = fused.info(), split.info()
        assert ia["status"] == 0 and ib["status"] == 0
        assert ia["steps"] == ib["steps"] == done
        assert abs(ia["dt"] - ib["dt"]) <= (1e-14 if prec == "fp64" else 1e-6) * ib["dt"]
        check_close(a - a0, b - b0, tol, (name, done))
        a0, b0 = a, b
    fused.close()
    split.close()


def test_fused_kernel_timing_entry(cr):
    """cr_time_kernels times the single launch (ms[1] = 0) and advances the
    state bit for bit like cr_step."""
    import torch
    mesh, U = _case("smooth2d_N2_odd")
    a = _solver(cr, mesh, "fp32", split=False)
    b = _solver(cr, mesh, "fp32", split=False)
    a.set_state(U)
    b.set_state(U)
    flush = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    ms = a.time_kernels(7, flush)
    b.step(7)
    assert ms[0] > 0 and ms[1] == 0
    assert np.array_equal(a.get_state(), b.get_state())
    assert a.info()["t"] == b.info()["t"]
    a.close()
    b.close()

"""The measurement entry points: unit-throughput probes and per-kernel timing.

cr_time_kernels launches the kernels of every step directly between CUDA
events (the two kernels, or the single fused launch); the state must advance
exactly as with cr_step (bit for bit: the same kernels in the same order), for
a single solve and for a batch.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return crkfr


def test_probe_peaks_are_plausible(cr):
    p = cr.probe_peaks()
    for k, v in p.items():
        assert math.isfinite(v) and v > 0, (k, v)
    assert 1e13 < p["ffma"] < 2e14            # FP32 FMA lane-operations/s of one GB300
    assert p["dfma"] < p["ffma"] / 10          # the narrow FP64 pipe
    assert 1e12 < p["copy_bytes"] < 2e13      # device copy, bytes/s read + write
    for k in ("h2d_bytes", "d2h_bytes", "duplex_bytes_per_direction"):
        assert 1e10 < p[k] < 2e12
    r = ctypes.c_double()
    assert cr.load_library().cr_probe_peak(9, ctypes.byref(r)) == cr.CR_EINVAL


@pytest.mark.parametrize("step_kernels", ["fused", "split"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_time_kernels_advances_like_step(cr, prec, step_kernels, monkeypatch):
    """split (the default): the volume and face / update kernels timed apart;
    fused (CRKFR_STEP_KERNELS=fused): the single launch in ms[0], ms[1] = 0."""
    if step_kernels == "fused":
        monkeypatch.setenv("CRKFR_STEP_KERNELS", "fused")
    else:
        monkeypatch.delenv("CRKFR_STEP_KERNELS", raising=False)
    mesh, U = inputs.shear_layer_2d(cells=(40, 24), N=3)
    with cr.Solver(mesh, prec=prec) as a, cr.Solver(mesh, prec=prec) as b:
        assert a.tuning_info()["step"] == step_kernels
        a.set_state(U)
        b.set_state(U)
        a.step(2)
        vol, face = a.time_kernels(3)
        b.step(5)
        assert vol > 0 and (face > 0 if step_kernels == "split" else face == 0)
        assert a.info()["steps"] == 5
        assert np.array_equal(a.get_state(), b.get_state())
        assert a.info()["dt"] == b.info()["dt"]


def test_time_kernels_batched(cr):
    # FP64: the two contexts autotune independently and may pick different
    # kernel shapes, which changes FP32 rounding but not FP64 arithmetic
    specs = inputs.batched_2d_specs(n_solves=6, seed=9, side_lo=3, side_hi=9)
    batch = [inputs.batched_2d_solve(sp) for sp in specs]
    meshes = [m for m, _ in batch]
    with cr.Solver(meshes, prec="fp64") as a, cr.Solver(meshes, prec="fp64") as b:
        for k, (_, U) in enumerate(batch):
            a.set_state(U, solve=k)
            b.set_state(U, solve=k)
        a.step(1)
        vol, face = a.time_kernels(2)
        b.step(3)
        assert vol > 0 and face > 0
        for k in range(len(batch)):
            assert np.array_equal(a.get_state(solve=k), b.get_state(solve=k))

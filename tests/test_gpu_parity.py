"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: FP64 path <= 1e-12 relative L2 per step from an identical state (and
over short free runs), dt identical to 1e-14; FP32 pair-flux form <= 1e-5
relative L2 after 100 steps on smooth data.  Every comparison also bounds the
per-variable largest nodal difference by the same tolerance (parity_util).
Sizes span several CTAs of the volume kernel with a ragged tail of elements.
"""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _case(name):
    if name == "wave1d_N3":
        return inputs.density_wave_1d(cells=64, N=3)
    if name.startswith("wave1d_N"):
        N = int(name[-1])
        return inputs.density_wave_1d(cells=13, N=N, cfl=inputs.default_cfl(N))
    if name == "shear2d_N3":
        return inputs.shear_layer_2d(cells=(11, 7), N=3)
    if name == "shear2d_N3_kep":
        return inputs.shear_layer_2d(cells=(9, 8), N=3, vol="kep")
    if name.startswith("smooth2d_N"):
        N = int(name[-1])
        mesh = inputs.mesh_dict("euler", 2, N, [7, 6], [0, 0], [1.0, 1.3], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=N, amp=0.2)
    if name == "central2d_N3":
        mesh = inputs.mesh_dict("euler", 2, 3, [5, 9], [0, 0], [1.0, 1.0], 1.4, vol="central")
        return mesh, inputs.smooth_random_field(mesh, seed=9, amp=0.2)
    if name == "tgv3d_N3":
        return inputs.tgv_3d(cells=(4, 3, 5), N=3, mach=0.3)
    if name == "tgv3d_N2":
        return inputs.tgv_3d(cells=(3, 4, 3), N=2, mach=0.3)
    if name in ("tgv3d_N1", "tgv3d_N4", "tgv3d_N5"):
        # 3D N = 4, 5: the tile-form volume kernel (the lane layout does not fit);
        # N = 5: the per-node face / update kernel
        N = int(name[-1])
        return inputs.tgv_3d(cells=(3, 4, 3) if N < 5 else (3, 2, 3), N=N, mach=0.3, cfl=inputs.default_cfl(N))
    if name.startswith("mhd2d_N"):
        # N = 5 in FP64: the tile-form volume kernel
        N = int(name[-1])
        return inputs.mhd_vortex_2d(cells=(6, 5) if N < 5 else (7, 5), N=N, cfl=inputs.default_cfl(N))
    if name == "mhd2d_central":
        return inputs.mhd_vortex_2d(cells=(5, 5), N=3, vol="central")
    if name == "single2d_N3":   # one element: its own periodic neighbour in both directions
        mesh = inputs.mesh_dict("euler", 2, 3, [1, 1], [0, 0], [1.0, 1.0], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=11, amp=0.2)
    if name == "single1d_N5":
        mesh = inputs.mesh_dict("euler", 1, 5, [1], [0], [2.0], 1.4, cfl=inputs.default_cfl(5))
        return mesh, inputs.smooth_random_field(mesh, seed=12, amp=0.2)
    if name == "strip2d_N2":    # one element across y
        mesh = inputs.mesh_dict("euler", 2, 2, [37, 1], [0, 0], [2.0, 0.1], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=13, amp=0.2)
    raise KeyError(name)


FP64_CASES = ["wave1d_N3", "wave1d_N1", "wave1d_N2", "wave1d_N4", "wave1d_N5", "shear2d_N3", "shear2d_N3_kep",
              "smooth2d_N1", "smooth2d_N2", "smooth2d_N4", "smooth2d_N5", "central2d_N3", "tgv3d_N3", "tgv3d_N2",
              "mhd2d_N3", "mhd2d_N4", "mhd2d_N2", "mhd2d_central", "single2d_N3", "single1d_N5", "strip2d_N2",
              "tgv3d_N1", "tgv3d_N4", "tgv3d_N5", "mhd2d_N1", "mhd2d_N5"]


@pytest.mark.parametrize("name", FP64_CASES)
def test_fp64_per_step_parity(cr, orc, name):
    mesh, U = _case(name)
    with cr.Solver(mesh, prec="fp64") as s:
        for k in range(3):
            s.set_state(U)
            dt = orc.cfl_dt(mesh, U)
            ref = orc.step(mesh, U, dt)
            s.step(1)
            out = s.get_state()
            info = s.info()
            assert abs(info["dt"] - dt) <= 1e-14 * dt, (info["dt"], dt)
            assert info["steps"] == 1
            check_close(out, ref, 1e-12, (name, k))
            U = ref


@pytest.mark.parametrize("name", ["wave1d_N3", "shear2d_N3", "mhd2d_N4", "tgv3d_N3"])
def test_fp64_free_run(cr, orc, name):
    mesh, U = _case(name)
    nsteps = 100 if name == "wave1d_N3" else 20
    ref, dts = orc.run(mesh, U, nsteps)
    with cr.Solver(mesh, prec="fp64") as s:
        s.set_state(U)
        s.step(nsteps)
        out = s.get_state()
        info = s.info()
    assert info["steps"] == nsteps
    assert abs(info["t"] - sum(dts)) <= 1e-12 * sum(dts)
    check_close(out, ref, 1e-12, name)


@pytest.mark.parametrize("name,steps", [("wave1d_N3", 100), ("shear2d_N3", 100), ("mhd2d_N4", 100),
                                        ("mhd2d_N5", 100), ("mhd2d_N3", 100), ("tgv3d_N3", 100),
                                        ("smooth2d_N5", 100), ("smooth2d_N2", 100), ("smooth2d_N4", 100),
                                        ("tgv3d_N4", 100), ("tgv3d_N5", 100), ("tgv3d_N1", 100),
                                        ("mhd2d_N1", 100), ("wave1d_N1", 100), ("wave1d_N5", 100),
                                        ("smooth2d_N1", 100), ("tgv3d_N2", 100), ("mhd2d_N2", 100)])
def test_fp32_pairflux_error(cr, orc, name, steps):
    mesh, U = _case(name)
    ref, dts = orc.run(mesh, U, steps)
    with cr.Solver(mesh, prec="fp32") as s:
        s.set_state(U)
        s.step(steps)
        out = s.get_state()
    check_close(out, ref, 1e-5, name)


@pytest.mark.parametrize("name,cons", [("shear2d_N3", range(4)), ("tgv3d_N3", range(5)), ("mhd2d_N4", [0])])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_conservation(cr, orc, name, cons, prec):
    mesh, U = _case(name)
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        T0 = s.info(totals=True)["totals"]
        s.step(100)
        T1 = s.info(totals=True)["totals"]
    A = orc.totals(mesh, np.abs(U))
    ref = orc.totals(mesh, U)
    np.testing.assert_allclose(T0[:len(cons)], ref[:len(cons)], rtol=1e-13, atol=1e-13 * A.max())
    # FP64: exact telescoping to round-off.  FP32 pair fluxes: the weighted
    # sums of 2 D_pq f_pq cancel only to FP32 round-off, so the totals drift
    # at the FP32 level (the state update itself is FP64)
    tol = 1e-13 if prec == "fp64" else 1e-6
    dim = mesh["dim"]
    mom_scale = A[1:1 + dim].max() if mesh["eq"] == "euler" else A[1:4].max()
    for v in cons:
        # a momentum total that starts at zero is measured against the momentum scale
        denom = max(abs(T0[v]), A[v], mom_scale if 1 <= v <= dim else 0.0)
        assert abs(T1[v] - T0[v]) / denom < tol, (v, T0[v], T1[v])


def test_free_stream(cr):
    mesh = inputs.mesh_dict("euler", 2, 4, [5, 4], [0, 0], [1, 1], 1.4)
    X = inputs.node_coords(mesh)
    one = np.ones_like(X[0])
    U = inputs.euler_cons(1.4, 1.2 * one, [0.3 * one, -0.2 * one], 0.9 * one)
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-6)):
        with cr.Solver(mesh, prec=prec) as s:
            s.set_state(U)
            s.step(10)
            out = s.get_state()
        assert np.max(np.abs(out - U)) <= tol * np.max(np.abs(U)), prec


def test_nonphysical_state_reported(cr):
    mesh, U = inputs.shear_layer_2d(cells=(4, 4), N=3)
    bad = U.copy()
    bad[0, 3, 5] = -1.0
    with cr.Solver(mesh) as s:
        with pytest.raises(cr.CrError) as ei:
            s.set_state(bad)
        assert ei.value.status == cr.CR_ENONPHYSICAL
        with pytest.raises(cr.CrError):
            s.step(1)             # no valid state
        s.set_state(U)            # context still usable
        s.step(2)
        s.sync()


def test_invalid_descriptors(cr):
    mesh, U = inputs.shear_layer_2d(cells=(4, 4), N=3)
    for bad in ({"N": 0}, {"N": 6}, {"dim": 4}, {"gamma": 1.0}, {"cells": [0, 4, 1]}, {"cfl": 0.0}):
        m = dict(mesh, **bad)
        with pytest.raises(cr.CrError) as ei:
            cr.Solver(m)
        assert ei.value.status == cr.CR_EINVAL
    with pytest.raises(cr.CrError):
        cr.Solver(dict(mesh, eq="glm_mhd", dim=3, cells=[2, 2, 2]))


def test_fixed_dt_and_time(cr, orc):
    mesh, U = _case("wave1d_N3")
    with cr.Solver(mesh, dt_fixed=1e-3) as s:
        s.set_state(U)
        s.step(7)
        info = s.info()
        out = s.get_state()
    ref, _ = orc.run(mesh, U, 7, dt_fixed=1e-3)
    assert info["dt"] == 1e-3 and abs(info["t"] - 7e-3) < 1e-15
    check_close(out, ref, 1e-12)


def test_device_pointers_and_torch_stream(cr, orc):
    import torch
    mesh, U = _case("shear2d_N3")
    dt = orc.cfl_dt(mesh, U)
    ref = orc.step(mesh, U, dt)
    stream = torch.cuda.Stream()
    Ud = torch.from_numpy(U).cuda()
    out = torch.empty_like(Ud)
    with torch.cuda.stream(stream):
        with cr.Solver(mesh, stream=stream) as s:
            s.set_state(Ud)
            s.step(1)
            s.get_state(out)
    check_close(out.cpu().numpy(), ref, 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_async_transfers_pipelined(cr, prec):
    """Three contexts on their own streams, each fed from pinned host memory
    with the asynchronous copies (set, step, get, no host sync in between):
    every output equals the synchronous single-context step bit for bit."""
    import torch
    mesh, U = inputs.shear_layer_2d(cells=(19, 13), N=3)
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(2)
        ref = s.get_state()
    Uh = torch.from_numpy(U).pin_memory()
    outs = [torch.empty_like(Uh).pin_memory() for _ in range(3)]
    solvers = [cr.Solver(mesh, prec=prec, stream=torch.cuda.Stream()) for _ in range(3)]
    for it in range(6):
        s = solvers[it % 3]
        s.set_state(Uh, sync=False)
        s.step(2)
        s.get_state(outs[it % 3], sync=False)
    for s in solvers:
        s.sync()
        s.close()
    for o in outs:
        assert np.array_equal(o.numpy(), ref)


"""Multi-stage RKFR scheme (eq. rkfr.non.cons) on the GPU against the oracle.

The multi-stage step runs the volume kernel with a single stage on each RK
stage state and the face / update kernel in stage mode (the stage's increment
K_j, the next stage state u^n + sum_q a_{j+1,q} K_q, the final combination with
b).  Bars as for the single-stage step: FP64 1e-12 relative L2 per step, the
FP32 pair-flux form 1e-5 after 100 steps, dt equal to the oracle's CFL rule.
Cases cover every Butcher tableau (N = 1..5), the lane and tile forms of both
kernels, meshes whose element count is not a multiple of the 32-element tile,
the degenerate meshes of one element (its own periodic neighbour) and of one
element across y, Euler in 1D/2D/3D (EC and KEP) and GLM-MHD.
"""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def case(name):
    """(mesh, U) of a small seeded case: 35, 36 or 37 elements (ragged tiles), or
    a degenerate mesh (one element, or one element across y)."""
    kind, N = name.rsplit("_N", 1)
    N = int(N)
    if kind == "euler1d":
        mesh = inputs.mesh_dict("euler", 1, N, [37], [0.0], [2.0], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=40 + N, amp=0.2)
    if kind == "shear2d":
        return inputs.shear_layer_2d(cells=(5, 7), N=N)
    if kind == "tgv3d":
        return inputs.tgv_3d(cells=(3, 3, 4), N=N, mach=0.3)
    if kind == "mhd2d":
        return inputs.mhd_vortex_2d(cells=(5, 7), N=N)
    if kind == "kep2d":
        return inputs.shear_layer_2d(cells=(6, 5), N=N, vol="kep")
    if kind == "single2d":      # one element: its own periodic neighbour in both directions
        mesh = inputs.mesh_dict("euler", 2, N, [1, 1], [0, 0], [1.0, 1.0], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=50 + N, amp=0.2)
    if kind == "single1d":
        mesh = inputs.mesh_dict("euler", 1, N, [1], [0], [2.0], 1.4, cfl=inputs.default_cfl(N))
        return mesh, inputs.smooth_random_field(mesh, seed=60 + N, amp=0.2)
    if kind == "strip2d":       # one element across y
        mesh = inputs.mesh_dict("euler", 2, N, [37, 1], [0, 0], [2.0, 0.1], 1.4)
        return mesh, inputs.smooth_random_field(mesh, seed=70 + N, amp=0.2)
    if kind == "singlemhd":
        return inputs.mhd_vortex_2d(cells=(1, 1), N=N)
    raise ValueError(name)


CASES = ["euler1d_N1", "euler1d_N2", "euler1d_N3", "euler1d_N4", "euler1d_N5", "shear2d_N3", "shear2d_N4",
         "tgv3d_N2", "tgv3d_N4", "mhd2d_N3", "mhd2d_N5", "kep2d_N3", "single2d_N3", "single1d_N5", "strip2d_N2",
         "singlemhd_N3"]


@pytest.mark.parametrize("name", CASES)
def test_rkfr_fp64_steps(cr, orc, name):
    mesh, U = case(name)
    with cr.Solver(mesh, prec="fp64", scheme="rkfr") as s:
        s.set_state(U)
        Uo = U
        for k in range(3):
            dt = orc.cfl_dt(mesh, Uo)
            s.step(1)
            info = s.info()
            assert info["steps"] == k + 1
            assert abs(info["dt"] - dt) <= 1e-14 * dt
            G = s.get_state()
            Uo = orc.rkfr_step(mesh, Uo, info["dt"])
            assert rel(G, Uo) <= 1e-12 * (k + 1), (k, rel(G, Uo))
        tun = s.tuning_info()
    assert tun["scheme"] == "rkfr"


@pytest.mark.parametrize("name", ["euler1d_N5", "shear2d_N3", "shear2d_N4", "tgv3d_N2", "mhd2d_N3", "mhd2d_N5"])
def test_rkfr_fp32_100_steps(cr, orc, name):
    mesh, U = case(name)
    with cr.Solver(mesh, prec="fp32", scheme="rkfr") as s:
        s.set_state(U)
        s.step(100)
        G = s.get_state()
        info = s.info()
    ref, dts = orc.rkfr_run(mesh, U, 100)
    assert info["steps"] == 100
    assert abs(info["t"] - sum(dts)) <= 1e-6 * sum(dts)
    assert rel(G, ref) <= 1e-5, rel(G, ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rkfr_full_size_one_step(cr, orc, prec):
    """256 x 256 shear layer, N = 3, every node against the oracle."""
    mesh, U = inputs.shear_layer_2d(cells=(256, 256), N=3)
    with cr.Solver(mesh, prec=prec, scheme="rkfr") as s:
        s.set_state(U)
        s.step(1)
        G = s.get_state()
        info = s.info()
    dt = orc.cfl_dt(mesh, U)
    assert abs(info["dt"] - dt) <= (1e-14 if prec == "fp64" else 1e-6) * dt
    O = orc.rkfr_step(mesh, U, info["dt"])
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel(G, O) <= tol, rel(G, O)
    for v in range(O.shape[0]):
        scale = max(np.max(np.abs(O[v])), 0.1 * np.max(np.abs(O)))
        assert np.max(np.abs(G[v] - O[v])) / scale <= tol, v


def test_rkfr_differs_from_crkfr_at_second_order(cr):
    """The two schemes on the GPU share the first-order term: their difference
    relative to the step's increment at least halves with dt (the oracle
    relation of test_oracle_rkfr.py, here through both GPU paths)."""
    mesh, U = case("shear2d_N3")
    out = []
    for dtf in (2e-3, 1e-3, 5e-4):
        res = {}
        for scheme in ("crkfr", "rkfr"):
            with cr.Solver(mesh, prec="fp64", dt_fixed=dtf, scheme=scheme) as s:
                s.set_state(U)
                s.step(1)
                res[scheme] = s.get_state()
        out.append(np.linalg.norm(res["crkfr"] - res["rkfr"]) / np.linalg.norm(res["crkfr"] - U))
    assert out[0] / out[1] >= 1.75 and out[1] / out[2] >= 1.75, out
    assert out[2] > 1e-6, out


def test_rkfr_time_kernels_advance_like_step(cr):
    """cr_time_kernels launches the same 2 s kernels per step as the graphs."""
    mesh, U = case("shear2d_N4")
    with cr.Solver(mesh, prec="fp64", scheme="rkfr") as a, cr.Solver(mesh, prec="fp64", scheme="rkfr") as b:
        a.set_state(U)
        b.set_state(U)
        a.step(3)
        ms = b.time_kernels(3)
        assert ms[0] > 0 and ms[1] > 0
        np.testing.assert_array_equal(a.get_state(), b.get_state())
        assert a.info()["t"] == b.info()["t"]


def test_rkfr_nonphysical_reported(cr):
    """A state that turns non-physical inside a step is reported by the next
    sync, as for the single-stage step."""
    mesh, U = case("euler1d_N3")
    with cr.Solver(mesh, prec="fp64", dt_fixed=5.0, scheme="rkfr") as s:
        s.set_state(U)
        s.step(3)
        with pytest.raises(cr.CrError) as ei:
            s.get_state()
        assert ei.value.status == cr.CR_ENONPHYSICAL

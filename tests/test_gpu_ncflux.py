"""Stage-wise non-conservative numerical flux (eq. bad.numflux.non.cons) on the
GPU against the oracle.

With CR_NCFLUX_STAGES the GLM-MHD volume kernel leaves, at every stage, seven
primitives (v, B, psi) of every face trace after the face records, and the face
kernel applies sum_j b_j B(u^(j)_own) g^avg(u^(j)) instead of the reduced-
communication B(u^n_own) g^avg(U).  Bars as for the reduced flux: FP64 1e-12
relative L2 per step, FP32 pair fluxes 1e-5 after 100 steps, dt equal to the
oracle's CFL rule; the lane form (N <= 4) and the tile form (FP64, N = 5), EC
and central volume fluxes, a mesh of 35 elements (ragged last tile).
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


def stages_mesh(N, vol="ec", cells=(5, 7)):
    mesh, U = inputs.mhd_vortex_2d(cells=cells, N=N, vol=vol)
    return dict(mesh, ncflux="stages"), U


@pytest.mark.parametrize("N,vol,cells", [(2, "ec", (5, 7)), (3, "ec", (5, 7)), (4, "ec", (5, 7)), (5, "ec", (5, 7)),
                                         (3, "central", (5, 7)),
                                         (3, "ec", (1, 1)),     # one element: its own neighbour on every face
                                         (2, "ec", (7, 1))])    # one element across y
def test_stagewise_fp64_steps(cr, orc, N, vol, cells):
    mesh, U = stages_mesh(N, vol, cells)
    with cr.Solver(mesh, prec="fp64") as s:
        s.set_state(U)
        Uo = U
        for k in range(3):
            dt = orc.cfl_dt(mesh, Uo)
            s.step(1)
            info = s.info()
            assert abs(info["dt"] - dt) <= 1e-14 * dt
            G = s.get_state()
            Uo = orc.step(mesh, Uo, info["dt"])
            assert rel(G, Uo) <= 1e-12 * (k + 1), (k, rel(G, Uo))
    # the two fluxes give different steps (the GPU path honours the option)
    red = orc.step(dict(mesh, ncflux="reduced"), U, orc.cfl_dt(mesh, U))
    with cr.Solver(mesh, prec="fp64") as s:
        s.set_state(U)
        s.step(1)
        G = s.get_state()
    assert rel(G, red) > 1e3 * rel(G, orc.step(mesh, U, orc.cfl_dt(mesh, U)))


@pytest.mark.parametrize("N", [3, 4, 5])
def test_stagewise_fp32_100_steps(cr, orc, N):
    mesh, U = stages_mesh(N)
    with cr.Solver(mesh, prec="fp32") as s:
        s.set_state(U)
        s.step(100)
        G = s.get_state()
    ref, _ = orc.run(mesh, U, 100)
    assert rel(G, ref) <= 1e-5, rel(G, ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_stagewise_full_size_one_step(cr, orc, prec):
    """128 x 128 GLM-MHD vortex, N = 4, every node against the oracle."""
    mesh, U = stages_mesh(4, cells=(128, 128))
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(1)
        G = s.get_state()
        info = s.info()
    O = orc.step(mesh, U, info["dt"])
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel(G, O) <= tol, rel(G, O)
    floor = 0.1 * np.max(np.abs(O))
    for v in range(O.shape[0]):
        assert np.max(np.abs(G[v] - O[v])) / max(np.max(np.abs(O[v])), floor) <= tol, v


def test_stagewise_rejected_outside_glm_mhd_crkfr(cr):
    mesh, _ = inputs.shear_layer_2d(cells=(4, 4), N=3)
    with pytest.raises(cr.CrError) as ei:
        cr.Solver(dict(mesh, ncflux="stages"))
    assert ei.value.status == cr.CR_EINVAL
    mh, _ = stages_mesh(3)
    with pytest.raises(cr.CrError) as ei:
        cr.Solver(mh, scheme="rkfr")
    assert ei.value.status == cr.CR_EINVAL

"""Pins of the oracle's stage-wise non-conservative numerical flux, CPU only.

The cRKFR step of the paper takes the non-conservative numerical flux
B(u^{n,+-}) g^avg(U) (the reduced-communication choice, used for all its
results); eq. bad.numflux.non.cons time-averages the stage fluxes instead,
sum_j b_j B(u^{(j),+-}) g^avg(u^(j)), which needs the face traces of every stage.
The oracle computes either (mesh key ncflux = 'reduced' | 'stages').  Pins:

* one stage (forward Euler): the two fluxes coincide, and the cRKFR step equals
  the multi-stage RKFR step with the same tableau (both are u - dt R_FR(u));
* b = e_1 (only the first stage, u^(1) = u^n, is weighted): the two coincide;
* the step is affine in b for a fixed A (stage states depend on A only);
* b = e_j, j > 1: the difference of the two steps is exactly the correction
  -dt (B(u^(j)_own) - B(u^n_own)) g^avg(u^(j)) g'(xi)/dx of the face terms,
  rebuilt here from the stage states of the oracle's element-stage routine;
* the two steps agree to O(dt^2); free stream; density conserved.
"""
import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs

from test_oracle_step import _const_state, _totals, _weights

FE = (np.zeros((1, 1)), np.array([1.0]))


def _mhd(N=3, cells=(4, 4)):
    return inputs.mhd_vortex_2d(cells=cells, N=N)


def _rel(a, b, scale):
    return np.max(np.abs(a - b)) / scale


@pytest.mark.parametrize("N", [2, 3, 4])
def test_forward_euler_reductions(orc, N):
    mesh, U = _mhd(N)
    dt = orc.cfl_dt(mesh, U)
    red = orc.step(dict(mesh, tableau=FE), U, dt)
    stg = orc.step(dict(mesh, tableau=FE, ncflux="stages"), U, dt)
    rk = orc.rkfr_step(dict(mesh, tableau=FE), U, dt)
    inc = np.max(np.abs(red - U))
    assert _rel(stg, red, inc) <= 1e-15
    assert _rel(rk, red, inc) <= 1e-13


@pytest.mark.parametrize("case", ["euler2d", "euler3d", "euler1d_N5"])
def test_forward_euler_crkfr_equals_rkfr_euler(orc, case):
    """Ties the cRKFR step's volume and face code to the separately written
    semi-discrete right-hand side of the RKFR step."""
    if case == "euler2d":
        mesh, U = inputs.shear_layer_2d(cells=(4, 5), N=3)
    elif case == "euler3d":
        mesh, U = inputs.tgv_3d(cells=(2, 3, 2), N=2, mach=0.3)
    else:
        mesh = inputs.mesh_dict("euler", 1, 5, [5], [0.0], [2.0], 1.4)
        U = inputs.smooth_random_field(mesh, seed=8, amp=0.2)
    dt = orc.cfl_dt(mesh, U)
    a = orc.step(dict(mesh, tableau=FE), U, dt)
    b = orc.rkfr_step(dict(mesh, tableau=FE), U, dt)
    assert _rel(a, b, np.max(np.abs(a - U))) <= 1e-12


@pytest.mark.parametrize("N", [3, 4])
def test_first_stage_weight_reduces_to_reduced_flux(orc, N):
    mesh, U = _mhd(N)
    A, b = orc.butcher(N)
    e0 = np.zeros(len(b))
    e0[0] = 1.0
    dt = orc.cfl_dt(mesh, U)
    red = orc.step(dict(mesh, tableau=(A, e0)), U, dt)
    stg = orc.step(dict(mesh, tableau=(A, e0), ncflux="stages"), U, dt)
    assert _rel(stg, red, np.max(np.abs(red - U))) <= 1e-15


@pytest.mark.parametrize("ncflux", ["reduced", "stages"])
def test_step_is_affine_in_b(orc, ncflux):
    mesh, U = _mhd(3)
    A, b = orc.butcher(3)
    dt = orc.cfl_dt(mesh, U)
    rng = np.random.default_rng(11)
    w = rng.uniform(-0.5, 1.0, len(b))
    full = orc.step(dict(mesh, tableau=(A, w), ncflux=ncflux), U, dt)
    acc = U.copy()
    for j in range(len(b)):
        ej = np.zeros(len(b))
        ej[j] = 1.0
        acc += w[j] * (orc.step(dict(mesh, tableau=(A, ej), ncflux=ncflux), U, dt) - U)
    assert _rel(full, acc, np.max(np.abs(full - U))) <= 1e-12


def _stage_state(orc, mesh, U, A, j, dt):
    """u^(j) of every element ([var][elem][node]) from the element-stage routine
    with b = e_j (then its time-averaged solution is u^(j))."""
    ej = np.zeros(A.shape[0])
    ej[j] = 1.0
    m = dict(mesh, tableau=(A, ej))
    out = np.empty_like(U)
    for e in range(U.shape[1]):
        _, Ubar, _, _ = orc.element_stages(m, np.ascontiguousarray(U[:, e, :].T), dt)
        out[:, e, :] = Ubar.T
    return out


@pytest.mark.parametrize("j", [1, 2, 3])
def test_stagewise_difference_is_the_stage_trace_correction(orc, j):
    N = 3
    mesh, U = _mhd(N, cells=(3, 4))
    A, b = orc.butcher(N)
    ej = np.zeros(len(b))
    ej[j] = 1.0
    dt = orc.cfl_dt(mesh, U)
    red = orc.step(dict(mesh, tableau=(A, ej)), U, dt)
    stg = orc.step(dict(mesh, tableau=(A, ej), ncflux="stages"), U, dt)
    Uj = _stage_state(orc, mesh, U, A, j, dt)
    xi, w, D, dgL, dgR = orc.tables(N)
    n = N + 1
    nx, ny = mesh["cells"][:2]
    dx = [(mesh["hi"][k] - mesh["lo"][k]) / mesh["cells"][k] for k in range(2)]
    expect = np.zeros_like(U)

    def node(i, jj):
        return i + n * jj

    for ey in range(ny):
        for ex in range(nx):
            e = ex + nx * ey
            for d in range(2):
                for side in (0, 1):
                    off = 1 if side else -1
                    nb = ((ex + off) % nx + nx * ey) if d == 0 else (ex + nx * ((ey + off) % ny))
                    for f in range(n):
                        # face node: own end node and the neighbour's opposite end node
                        own_p = node(N if side else 0, f) if d == 0 else node(f, N if side else 0)
                        oth_p = node(0 if side else N, f) if d == 0 else node(f, 0 if side else N)
                        uj_own, uj_oth = Uj[:, e, own_p], Uj[:, nb, oth_p]
                        gavg_state = 0.5 * (uj_own + uj_oth)
                        corr = (orc.nc_product(mesh, d, uj_own, gavg_state)
                                - orc.nc_product(mesh, d, U[:, e, own_p], gavg_state))
                        for k in range(n):
                            p = node(k, f) if d == 0 else node(f, k)
                            dg = (dgR[k] if side else dgL[k]) / dx[d]
                            expect[:, e, p] -= dt * corr * dg
    diff = stg - red
    assert np.max(np.abs(diff)) > 1e-6 * np.max(np.abs(red - U))   # the fluxes do differ
    assert _rel(diff, expect, np.max(np.abs(diff))) <= 1e-10


def test_stagewise_and_reduced_agree_to_second_order(orc):
    mesh, U = _mhd(3)
    dt0 = orc.cfl_dt(mesh, U)
    rel = []
    for fac in (1.0, 0.5, 0.25):
        dt = dt0 * fac
        a = orc.step(mesh, U, dt)
        c = orc.step(dict(mesh, ncflux="stages"), U, dt)
        rel.append(np.linalg.norm(a - c) / np.linalg.norm(a - U))
    assert rel[0] / rel[1] >= 1.8 and rel[1] / rel[2] >= 1.8, rel
    assert rel[2] > 1e-8, rel


def test_stagewise_free_stream_and_density(orc):
    mesh = inputs.mesh_dict("glm_mhd", 2, 3, [3, 3], [0, 0], [1, 1], 5.0 / 3.0, c_h=1.5)
    U = _const_state(mesh)
    m = dict(mesh, ncflux="stages")
    np.testing.assert_allclose(orc.step(m, U, orc.cfl_dt(m, U)), U, rtol=1e-13, atol=1e-13)
    mesh, U = _mhd(3)
    m = dict(mesh, ncflux="stages")
    W = _weights(mesh, orc)
    T0, A0 = _totals(mesh, U, W)
    U1, _ = orc.run(m, U, 40)
    T1, _ = _totals(mesh, U1, W)
    assert abs(T1[0] - T0[0]) / A0[0] < 1e-13

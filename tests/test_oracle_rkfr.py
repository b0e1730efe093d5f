"""Pins of the oracle's multi-stage RKFR step (eq. rkfr.non.cons), CPU only.

The multi-stage step applies the degree's RK tableau to the semi-discrete FR
system (eq. general.non.conservative.fr.one) and exchanges face data at every
stage.  It is pinned against things other than its own formula:

* a library ODE integrator (scipy's DOP853 at tolerance 1e-13) on the same
  semi-discrete system: the one-step error falls at order p + 1 = N + 2;
* the single-stage cRKFR step, pinned on its own in test_oracle_step.py: the
  two schemes share their first-order term u^n - dt R_FR(u^n), so their
  difference, relative to the step's increment, at least halves with dt;
* the amplification matrix of the scheme's linear structure for u_t + u_x = 0
  with the upwind flux (every stage with the full FR operator);
* free stream, exact conservation, design-order convergence and the 1D
  reduction of the tensor-product reading.
"""
import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs

from test_oracle_step import _const_state, _totals, _weights


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_rkfr_local_error_order_against_ode_solver(orc, N):
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    mesh = inputs.mesh_dict("euler", 1, N, [4], [0.0], [2.0], 1.4)
    U = inputs.smooth_random_field(mesh, seed=31, amp=0.2)
    dt0 = orc.cfl_dt(mesh, U)

    def rhs(t, y):
        return orc.fr_rhs(mesh, y.reshape(U.shape)).ravel()

    errs = []
    for fac in (1.0, 0.5):
        dt = dt0 * fac
        ode = solve_ivp(rhs, (0.0, dt), U.ravel(), method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
        errs.append(np.linalg.norm(orc.rkfr_step(mesh, U, dt).ravel() - ode) / np.linalg.norm(ode))
    rate = np.log2(errs[0] / errs[1])
    # local error of an order-(N+1) method: O(dt^(N+2)); measured 3.01, 3.96,
    # 4.95, 6.36, 6.97 for N = 1..5.  The smaller error stays far above the
    # integrator's tolerance.
    assert errs[1] > 1e-11, errs
    assert rate >= N + 2 - 0.15, (errs, rate)


@pytest.mark.parametrize("case", ["shear2d", "mhd2d", "tgv3d", "wave1d_N5"])
def test_rkfr_and_crkfr_share_the_first_order_term(orc, case):
    if case == "shear2d":
        mesh, U = inputs.shear_layer_2d(cells=(4, 4), N=3)
    elif case == "mhd2d":
        mesh, U = inputs.mhd_vortex_2d(cells=(4, 4), N=3)
    elif case == "tgv3d":
        mesh, U = inputs.tgv_3d(cells=(2, 2, 2), N=2, mach=0.3)
    else:
        mesh = inputs.mesh_dict("euler", 1, 5, [4], [0.0], [2.0], 1.4)
        U = inputs.smooth_random_field(mesh, seed=4, amp=0.2)
    dt0 = orc.cfl_dt(mesh, U)
    rel = []
    for fac in (1.0, 0.5, 0.25):
        dt = dt0 * fac
        crk = orc.step(mesh, U, dt)
        rk = orc.rkfr_step(mesh, U, dt)
        rel.append(np.linalg.norm(crk - rk) / np.linalg.norm(crk - U))
    # a first-order discrepancy (a face or volume term that differs) keeps the
    # ratio near 1; agreement to O(dt^2) gives 2 (noisy data), O(dt^3) gives 4
    # (smooth data, where the face corrections of the inner stages are small)
    assert rel[1] / rel[2] >= 1.8, rel
    assert rel[0] / rel[1] >= 1.75, rel
    # ... and the two schemes are not the same scheme
    assert rel[2] > 1e-5, rel


def _rkfr_scalar_model(orc, N, cfl, E=5):
    """Amplification matrix of RKFR for u_t + u_x = 0 with the upwind flux:
    every stage applies the full FR operator L (local derivative plus the g2
    correction of the upwind face jump), u^(i) = u + dt sum_j a_ij L u^(j),
    u^{n+1} = u + dt sum_i b_i L u^(i)."""
    xi, w, D, dgL, dgR = orc.tables(N)
    A, b = orc.butcher(N)
    n = N + 1
    dx = 1.0 / E
    L = np.zeros((E * n, E * n))
    for e in range(E):
        L[e * n:(e + 1) * n, e * n:(e + 1) * n] = -D / dx
    for e in range(E):
        im, ip = e * n + N, ((e + 1) % E) * n
        L[ip, im] += -dgL[0] / dx
        L[ip, ip] += dgL[0] / dx
    dt = cfl * dx
    I = np.eye(E * n)
    P = [I]
    for i in range(1, len(b)):
        P.append(I + dt * sum(A[i, j] * (L @ P[j]) for j in range(i)))
    G = I + dt * L @ sum(b[i] * P[i] for i in range(len(b)))
    return np.max(np.abs(np.linalg.eigvals(G)))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_rkfr_linear_stability_at_cfl(orc, N):
    """Spectral radius of the linearised RKFR step around a constant state
    (central differences of the oracle step) equals that of the scalar model
    and is at most 1 at the CFL numbers of the cRKFR step (RKFR's own limits
    are higher: 0.45, 0.29, 0.23, 0.10 for N = 2..5)."""
    mesh = inputs.mesh_dict("euler", 1, N, [5], [0.0], [1.0], 1.4)
    U0 = _const_state(mesh, seed=3)
    dt = orc.cfl_dt(mesh, U0)
    n = U0.size
    J = np.zeros((n, n))
    h = 1e-5
    for k in range(n):
        dU = np.zeros(n)
        dU[k] = h
        J[:, k] = (orc.rkfr_step(mesh, (U0.ravel() + dU).reshape(U0.shape), dt).ravel()
                   - orc.rkfr_step(mesh, (U0.ravel() - dU).reshape(U0.shape), dt).ravel()) / (2 * h)
    rho = np.max(np.abs(np.linalg.eigvals(J)))
    model = _rkfr_scalar_model(orc, N, inputs.default_cfl(N))
    assert abs(rho - model) < 1e-8, (rho, model)
    assert rho <= 1.0 + 1e-9, rho


@pytest.mark.parametrize("eq,dim,N", [("euler", 1, 3), ("euler", 2, 2), ("euler", 3, 2), ("glm_mhd", 2, 3)])
def test_rkfr_free_stream(orc, eq, dim, N):
    if eq == "euler":
        mesh = inputs.mesh_dict(eq, dim, N, [3] * dim, [0] * dim, [1.0] * dim, 1.4)
    else:
        mesh = inputs.mesh_dict(eq, 2, N, [3, 3], [0, 0], [1, 1], 5.0 / 3.0, c_h=1.5)
    U = _const_state(mesh)
    U1 = orc.rkfr_step(mesh, U, orc.cfl_dt(mesh, U))
    np.testing.assert_allclose(U1, U, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("case", ["shear", "mhd"])
def test_rkfr_conservation(orc, case):
    if case == "shear":
        mesh, U = inputs.shear_layer_2d(cells=(6, 6), N=3)
        cons = range(4)
    else:
        mesh, U = inputs.mhd_vortex_2d(cells=(4, 4), N=3)
        cons = [0]          # the Powell / GLM terms are non-conservative
    W = _weights(mesh, orc)
    T0, A0 = _totals(mesh, U, W)
    U1, _ = orc.rkfr_run(mesh, U, 40)
    T1, A1 = _totals(mesh, U1, W)
    for v in cons:
        denom = max(abs(T0[v]), A0[v], A1[v])
        assert abs(T1[v] - T0[v]) / denom < 1e-13, (v, T0[v], T1[v])


@pytest.mark.parametrize("N,cells", [(2, (8, 16, 32)), (3, (8, 16, 32))])
def test_rkfr_density_wave_convergence(orc, N, cells):
    errs = []
    for c in cells:
        mesh, U = inputs.density_wave_1d(cells=c, N=N)
        dx = 2.0 / c
        T = 0.5
        nsteps = int(np.ceil(T / (inputs.default_cfl(N) * dx / 3.0)))
        U1, _ = orc.rkfr_run(mesh, U, nsteps, dt_fixed=T / nsteps)
        ex = inputs.density_wave_exact_1d(mesh, T)
        xi, w, *_ = orc.tables(N)
        errs.append(np.sqrt(np.sum((U1[0] - ex) ** 2 * w[None, :]) * dx))
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(cells[i + 1] / cells[i]) for i in range(len(cells) - 1)]
    assert rates[-1] >= N + 0.5, (errs, rates)


def test_rkfr_multid_reduces_to_1d(orc):
    N, dim = 3, 2
    mesh1, U1d = inputs.density_wave_1d(cells=6, N=N)
    meshd = inputs.mesh_dict("euler", dim, N, [6, 2], [0.0, 0.0], [2.0, 0.7], 1.4)
    X = inputs.node_coords(meshd)
    rho = 1.0 + 0.5 * np.sin(np.pi * X[0])
    U = inputs.euler_cons(1.4, rho, [np.ones_like(rho), np.zeros_like(rho)], np.ones_like(rho))
    for _ in range(3):
        U1d = orc.rkfr_step(mesh1, U1d, 0.01)
        U = orc.rkfr_step(meshd, U, 0.01)
    n = N + 1
    for e in range(inputs.num_elems(meshd)):
        for p in range(n ** dim):
            for v, v1 in [(0, 0), (1, 1), (3, 2)]:
                assert abs(U[v, e, p] - U1d[v1, e % 6, p % n]) < 1e-13
            assert abs(U[2, e, p]) < 1e-14

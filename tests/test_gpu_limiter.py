"""GPU parity of the subcell blending limiter (CR_LIMITER_BLENDING) against
the FP64 oracle's limited step (readings R19-R23: the paper's Sec. 4 runs
blend the cRKFR update with a first-order subcell finite-volume update,
coefficient capped by alpha_max).

* every Euler variant (dim 1-3, N = 1..5, both precisions, every volume flux):
  one step from a state with steep fronts, so that the coefficient takes 0,
  intermediate values and the cap in different elements; state and increment
  compared node by node (1e-12 / 1e-10 FP64, 1e-5 / 1e-3 FP32), dt as in the
  unlimited step;
* alpha_max = 0: the limited path (ping-pong buffers, per-node kernel) gives
  the unlimited step;
* free runs (FP64 <= 1e-12 over 20 steps; FP32 <= 1e-5 over 100 steps);
* conservation over 100 steps (FP64 1e-13, FP32 1e-6);
* positivity: on a node-to-node oscillation of density and pressure (ratio
  1000) every element takes alpha = 1 and the step is the first-order one,
  which stays positive under the first-order time step bound;
* the 256^2 shear layer at N = 3 with the KEP flux and alpha_max = 0.008 (the
  paper's Kelvin-Helmholtz setting), one step on every node;
* the coefficients a step used (cr_get_blend_alpha) against the oracle's:
  the same elements at zero, at the cap and in between, FP64 to 1e-12 and
  FP32 (energy fractions in FP32, FP64 near the clip thresholds) to 1e-5.
"""
import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs
from parity_util import check_close, check_increment

pytestmark = pytest.mark.gpu

STATE_TOL = {"fp64": 1e-12, "fp32": 1e-5}
INC_TOL = {"fp64": 1e-10, "fp32": 1e-3}
DT_TOL = {"fp64": 1e-14, "fp32": 1e-6}
CELLS = {1: [37], 2: [7, 5], 3: [3, 4, 3]}


@pytest.fixture(scope="module")
def cr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return crkfr


def fronts_state(dim, N, vol, seed, alpha_max=0.7):
    """A smooth seeded field times a density / pressure slab with steep edges
    across x (ratio about 3), on a small mesh with a ragged last tile."""
    mesh = inputs.mesh_dict("euler", dim, N, CELLS[dim], [0.0] * dim, [1.0, 1.3, 0.9][:dim], 1.4, vol=vol)
    mesh = dict(mesh, limiter=True, alpha_max=alpha_max)
    U = inputs.smooth_random_field(mesh, seed=seed, amp=0.1)
    X = inputs.node_coords(mesh)
    steep = 40.0 if dim > 1 else 150.0      # the 1D mesh has more elements across the slab
    slab = 1.0 + 1.0 * (np.tanh(steep * (X[0] - 0.3)) - np.tanh(steep * (X[0] - 0.65)))
    rho = U[0] * slab
    vel = [U[1 + k] / U[0] for k in range(dim)]
    p = (1.4 - 1.0) * (U[dim + 1] - 0.5 * U[0] * sum(v * v for v in vel)) * slab
    return mesh, inputs.euler_cons(1.4, rho, vel, p)


VARIANTS = [(dim, N, prec, vol) for prec in ("fp64", "fp32") for dim in (1, 2, 3) for N in range(1, 6)
            for vol in ("ec", "kep", "central")]


@pytest.mark.parametrize("var", VARIANTS, ids=lambda v: "%dd-N%d-%s-%s" % v)
def test_limited_variant_one_step(cr, orc, var):
    dim, N, prec, vol = var
    mesh, U = fronts_state(dim, N, vol, seed=300 + 11 * N + dim)
    _, a = orc.blend_alpha(mesh, U)
    assert a.max() > 0.0                    # the limiter acts somewhere
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(1)
        G = s.get_state()
        info = s.info()
    assert info["status"] == 0 and info["steps"] == 1
    dt = orc.cfl_dt(mesh, U)
    assert abs(info["dt"] - dt) <= DT_TOL[prec] * dt
    O = orc.step(mesh, U, info["dt"])
    what = "%dd-N%d-%s-%s" % var
    check_close(G, O, STATE_TOL[prec], what)
    check_increment(G, O, U, INC_TOL[prec], what)


def test_coefficient_spread(orc):
    """The fronts state exercises every branch of the coefficient: zero,
    intermediate (smoothing) and capped elements."""
    mesh, U = fronts_state(2, 3, "ec", seed=1)
    _, a = orc.blend_alpha(mesh, U)
    assert np.any(a == 0.0) and np.any(a == 0.7) and np.any((a > 0.0) & (a < 0.7))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_alpha_max_zero_is_the_unlimited_step(cr, orc, prec):
    mesh, U = fronts_state(2, 4, "ec", seed=7, alpha_max=0.0)
    plain = dict(mesh, limiter=False)
    with cr.Solver(mesh, prec=prec) as s, cr.Solver(plain, prec=prec) as p:
        s.set_state(U)
        p.set_state(U)
        s.step(3)
        p.step(3)
        G, P = s.get_state(), p.get_state()
    check_close(G, P, 1e-13 if prec == "fp64" else 1e-6)
    O, _ = orc.run(plain, U, 3)
    check_close(G, O, STATE_TOL[prec])


@pytest.mark.parametrize("dim,N,steps,prec", [(2, 3, 20, "fp64"), (1, 4, 20, "fp64"), (3, 2, 10, "fp64"),
                                              (2, 3, 100, "fp32"), (1, 5, 100, "fp32")])
def test_limited_free_run(cr, orc, dim, N, steps, prec):
    mesh, U = fronts_state(dim, N, "ec", seed=20 + N)
    ref, dts = orc.run(mesh, U, steps)
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(steps)
        G = s.get_state()
        info = s.info()
    assert info["steps"] == steps
    check_close(G, ref, STATE_TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_limited_conservation(cr, orc, prec):
    mesh, U = fronts_state(2, 3, "kep", seed=31)
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        T0 = s.info(totals=True)["totals"]
        s.step(100)
        T1 = s.info(totals=True)["totals"]
    A = orc.totals(mesh, np.abs(U))
    tol = 1e-13 if prec == "fp64" else 1e-6
    for v in range(4):
        denom = max(abs(T0[v]), A[v], A[1:3].max() if v in (1, 2) else 0.0)
        assert abs(T1[v] - T0[v]) / denom < tol, (v, T0[v], T1[v])


def test_first_order_positivity(cr, orc):
    """rho and p alternate between 1 and 1e-3 from node to node: every element's
    energy sits in its highest mode, so alpha = 1 everywhere and the step is
    first-order finite volumes, positive under dt sum lambda/(w_min dx) <= 1."""
    N = 3
    mesh = dict(inputs.mesh_dict("euler", 1, N, [16], [0.0], [1.0], 1.4), limiter=True, alpha_max=1.0)
    (x,) = inputs.node_coords(mesh)
    osc = np.where((np.arange(x.size).reshape(x.shape) % 2) == 0, 1.0, 1e-3)
    U = inputs.euler_cons(1.4, osc, [0.3 * np.ones_like(x)], osc)
    _, a = orc.blend_alpha(mesh, U)
    assert np.all(a == 1.0)
    w_min = 1.0 / (N * (N + 1))                     # GLL end weight on [0,1]
    lam = np.max(0.3 + np.sqrt(1.4 * osc / osc))
    dt = 0.9 * w_min * (1.0 / 16) / lam
    with cr.Solver(mesh, prec="fp64", dt_fixed=dt) as s:
        s.set_state(U)
        ref = U
        for k in range(40):
            s.step(1)
            G = s.get_state()
            ref = orc.step(mesh, ref, dt)
            check_close(G, ref, 1e-12, k)
            rho = G[0]
            p = 0.4 * (G[2] - 0.5 * G[1] ** 2 / rho)
            assert rho.min() > 0 and p.min() > 0


@pytest.mark.parametrize("case", ["kh", "fronts"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_256(cr, orc, prec, case):
    """kh: the shear layer with the KEP flux and alpha_max = 0.008 (the paper's
    Kelvin-Helmholtz setting; the initial layer is resolved, so alpha = 0 and
    the limited kernels must reproduce the unlimited step); fronts: the same
    mesh with a steep density / pressure slab and alpha_max = 0.7."""
    if case == "kh":
        mesh, U = inputs.shear_layer_2d(cells=(256, 256), N=3, vol="kep")
        mesh = dict(mesh, limiter=True, alpha_max=0.008)
    else:
        mesh = dict(inputs.mesh_dict("euler", 2, 3, [256, 256], [0.0, 0.0], [1.0, 1.0], 1.4), limiter=True,
                    alpha_max=0.7)
        X = inputs.node_coords(mesh)
        slab = 1.0 + (np.tanh(300.0 * (X[0] - 0.3)) - np.tanh(300.0 * (X[0] - 0.65)))
        one = np.ones_like(X[0])
        U = inputs.euler_cons(1.4, slab * (1.0 + 0.1 * np.sin(2 * np.pi * X[1])), [0.4 * one, 0.1 * one], slab)
        _, a = orc.blend_alpha(mesh, U)
        assert a.max() == 0.7 and np.mean(a > 0) < 0.2
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(1)
        G = s.get_state()
        info = s.info()
    dt = orc.cfl_dt(mesh, U)
    assert abs(info["dt"] - dt) <= DT_TOL[prec] * dt
    O = orc.step(mesh, U, info["dt"])
    check_close(G, O, STATE_TOL[prec])
    check_increment(G, O, U, INC_TOL[prec])


@pytest.mark.parametrize("dim,N", [(1, 2), (1, 5), (2, 1), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_blend_coefficients_match_oracle(cr, orc, dim, N, prec):
    mesh, U = fronts_state(dim, N, "ec", seed=700 + 10 * dim + N)
    _, ref = orc.blend_alpha(mesh, U)
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        assert np.all(s.blend_alpha() == 0.0)      # before the first step
        s.step(1)
        a = s.blend_alpha()
    am = mesh["alpha_max"]
    assert np.array_equal(a == 0.0, ref == 0.0)
    assert np.array_equal(a == am, ref == am) or prec == "fp32"
    assert np.max(np.abs(a - ref)) <= (1e-12 if prec == "fp64" else 1e-5), np.max(np.abs(a - ref))
    assert np.any(ref > 0.0)


def test_blend_alpha_needs_the_limiter(cr):
    mesh, U = inputs.shear_layer_2d(cells=(8, 8), N=3)
    with cr.Solver(mesh) as s:
        with pytest.raises(cr.CrError):
            s.blend_alpha()

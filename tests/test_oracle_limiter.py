"""Pins of the oracle's subcell blending limiter (the paper's Sec. 4 runs blend
the cRKFR update with a first-order subcell finite-volume update, coefficient
capped by alpha_max; readings in the oracle's limiter section).

Each pin ties the oracle to something outside it:
* alpha = 0 in every element gives the unlimited cRKFR step bit for bit;
* alpha = 1 gives the first-order finite-volume step on the subcells, written
  here independently on the global grid of GLL nodes (subcell widths from
  numpy's Legendre routines, Euler flux and wave speed typed here);
* the limited step conserves every total (telescoping fluxes) over 100 steps;
* positivity: on a 1000:1 density and pressure jump the alpha = 1 step keeps
  rho, p > 0 under the first-order time step bound, where the unlimited step
  does not;
* the smoothness indicator: closed-form highest-mode energy fractions of
  rho p = a + b P_N (1D) and a + b P_N(x) P_N(y) (2D), the logistic map and
  its clipping, the neighbour smoothing rule;
* the limited face flux: alpha_f = 0 returns the high-order flux exactly,
  alpha_f = 1 the Rusanov flux of the traces, and for seeded random data the
  end-subcell states it produces keep the stated density / pressure bounds,
  with no change where the blended flux already keeps them.
A planted error in the blend weights, the subcell widths, the face-flux
selection or the correction fails one of them.
"""
import numpy as np
import pytest
from numpy.polynomial import legendre as L

from paper_2604_02125_gb300 import inputs


def _w01(N):
    """GLL weights on [0,1] from numpy: 1/(N(N+1) P_N(x)^2)."""
    x = 2.0 * inputs.gll_points01(N) - 1.0
    c = np.zeros(N + 1)
    c[N] = 1.0
    return 1.0 / (N * (N + 1) * L.legval(x, c) ** 2)


def _euler_flux(u, d, g):
    """Euler flux in direction d and wave speed |v_d| + c; u is [M][...]."""
    dim = u.shape[0] - 2
    rho = u[0]
    v = [u[1 + k] / rho for k in range(dim)]
    p = (g - 1.0) * (u[dim + 1] - 0.5 * rho * sum(vk * vk for vk in v))
    f = np.empty_like(u)
    f[0] = rho * v[d]
    for k in range(dim):
        f[1 + k] = rho * v[d] * v[k] + (p if k == d else 0.0)
    f[dim + 1] = v[d] * (u[dim + 1] + p)
    return f, np.abs(v[d]) + np.sqrt(g * p / rho)


def _to_grid(mesh, U):
    """[M][E][NP] -> [M][nx*n, ny*n, ...] (global grid of the GLL nodes)."""
    dim, n = mesh["dim"], mesh["N"] + 1
    cells = mesh["cells"][:dim]
    M = U.shape[0]
    A = U.reshape([M] + cells[::-1] + [n] * dim)                   # [M][ez][ey][ex][k][j][i]
    # interleave element and node axes per direction: (e_d, node_d) -> global
    axes = [0]
    for k in range(dim):
        axes += [dim - k, 2 * dim - k]                              # x: (ex, i), y: (ey, j), ...
    G = A.transpose(axes)                                           # [M][ex][i][ey][j]...
    return G.reshape([M] + [cells[k] * n for k in range(dim)])


def _from_grid(mesh, G):
    dim, n = mesh["dim"], mesh["N"] + 1
    cells = mesh["cells"][:dim]
    M = G.shape[0]
    A = G.reshape([M] + sum([[cells[k], n] for k in range(dim)], []))
    axes = [0] + [2 * k + 1 for k in range(dim)][::-1] + [2 * k + 2 for k in range(dim)][::-1]
    return A.transpose(axes).reshape(M, int(np.prod(cells)), n ** dim)


def fo_subcell_step(mesh, U, dt):
    """First-order finite volumes on the subcells: node g of the global grid
    owns a subcell of width w_i dx; every subcell face, inside an element or
    between two, takes the Rusanov flux of its two node values."""
    dim, N = mesh["dim"], mesh["N"]
    g = mesh["gamma"]
    G = _to_grid(mesh, U)
    w = _w01(N)
    out = G.copy()
    for d in range(dim):
        dx = (mesh["hi"][d] - mesh["lo"][d]) / mesh["cells"][d]
        R = np.roll(G, -1, axis=1 + d)                              # right neighbour node
        fL, lL = _euler_flux(G, d, g)
        fR, lR = _euler_flux(R, d, g)
        F = 0.5 * (fL + fR) - 0.5 * np.maximum(lL, lR) * (R - G)    # flux at the right face of each subcell
        Fm = np.roll(F, 1, axis=1 + d)                              # at the left face
        width = np.tile(w, mesh["cells"][d]) * dx
        shape = [1] * (dim + 1)
        shape[1 + d] = -1
        out -= dt * (F - Fm) / width.reshape(shape)
    return _from_grid(mesh, out)


def _lim(mesh, **kw):
    return dict(mesh, limiter=True, **kw)


@pytest.mark.parametrize("dim,N,vol", [(1, 1, "ec"), (1, 5, "kep"), (2, 3, "ec"), (2, 4, "central"), (2, 2, "kep"),
                                       (3, 2, "ec"), (3, 3, "kep")])
def test_alpha_zero_is_the_unlimited_step(orc, dim, N, vol):
    cells = {1: [9], 2: [5, 4], 3: [3, 2, 3]}[dim]
    mesh = inputs.mesh_dict("euler", dim, N, cells, [0.0] * dim, [1.0] * dim, 1.4, vol=vol)
    U = inputs.smooth_random_field(mesh, seed=40 + N, amp=0.3)
    dt = orc.cfl_dt(mesh, U)
    assert np.array_equal(orc.step(mesh, U, dt), orc.step(_lim(mesh, alpha_fixed=0.0), U, dt))


def test_grid_mapping_roundtrip():
    mesh = inputs.mesh_dict("euler", 2, 3, [3, 2], [0, 0], [1, 1], 1.4)
    X = inputs.node_coords(mesh)
    G = _to_grid(mesh, np.stack([X[0], X[1]]))
    # x along axis 0, y along axis 1 (element end nodes share a coordinate)
    assert np.all(np.diff(G[0], axis=0) >= 0) and np.all(np.diff(G[1], axis=1) >= 0)
    assert np.all(np.diff(G[0], axis=1) == 0) and np.all(np.diff(G[1], axis=0) == 0)
    U = np.arange(2 * 6 * 16, dtype=float).reshape(2, 6, 16)
    assert np.array_equal(_from_grid(mesh, _to_grid(mesh, U)), U)


@pytest.mark.parametrize("dim,N", [(1, 3), (1, 1), (2, 2), (2, 4), (3, 2)])
def test_alpha_one_is_first_order_subcell_fv(orc, dim, N):
    cells = {1: [11], 2: [4, 5], 3: [3, 2, 2]}[dim]
    mesh = inputs.mesh_dict("euler", dim, N, cells, [0.0] * dim, [1.0, 1.2, 0.8][:dim], 1.4)
    U = inputs.smooth_random_field(mesh, seed=50 + N, amp=0.3)
    dt = 0.5 * orc.cfl_dt(mesh, U)
    got = orc.step(_lim(mesh, alpha_fixed=1.0), U, dt)
    ref = fo_subcell_step(mesh, U, dt)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-14
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))


def test_planted_width_error_is_caught(orc):
    """The alpha = 1 pin distinguishes the subcell widths w_p dx from equal widths."""
    mesh = inputs.mesh_dict("euler", 1, 3, [11], [0.0], [1.0], 1.4)
    U = inputs.smooth_random_field(mesh, seed=53, amp=0.3)
    dt = 0.5 * orc.cfl_dt(mesh, U)
    got = orc.step(_lim(mesh, alpha_fixed=1.0), U, dt)
    w = _w01(3)
    _w01_saved = globals()["_w01"]
    try:
        globals()["_w01"] = lambda N: np.full(N + 1, 1.0 / (N + 1))
        wrong = fo_subcell_step(mesh, U, dt)
    finally:
        globals()["_w01"] = _w01_saved
    assert w[0] != 0.25
    assert np.linalg.norm(got - wrong) / np.linalg.norm(wrong) > 1e-6


def _jump_1d(N, cells=40, ratio=1e-3):
    """1D Euler: a periodic slab of rho = p = 1 in a background of rho = p = ratio, u = 0.5."""
    mesh = inputs.mesh_dict("euler", 1, N, [cells], [0.0], [1.0], 1.4)
    (x,) = inputs.node_coords(mesh)
    inside = (x > 0.3) & (x < 0.6)
    rho = np.where(inside, 1.0, ratio)
    p = np.where(inside, 1.0, ratio)
    return mesh, inputs.euler_cons(1.4, rho, [0.5 * np.ones_like(x)], p)


def _lo_dt(mesh, U):
    """First-order bound: dt max_d sum lambda_d / (w_min dx_d) <= 1, with a 0.9 margin."""
    N = mesh["N"]
    lam = 0.0
    for d in range(mesh["dim"]):
        dx = (mesh["hi"][d] - mesh["lo"][d]) / mesh["cells"][d]
        _, l = _euler_flux(U.reshape(U.shape[0], -1), d, mesh["gamma"])
        lam += l / (_w01(N).min() * dx)
    return 0.9 / np.max(lam)


def _rho_p(U, g=1.4):
    dim = U.shape[0] - 2
    rho = U[0]
    ke = 0.5 * sum(U[1 + k] ** 2 for k in range(dim)) / rho
    return rho, (g - 1.0) * (U[dim + 1] - ke)


def test_positivity_on_a_sharp_jump(orc):
    mesh, U0 = _jump_1d(3)
    U = U0.copy()
    for _ in range(60):
        U = orc.step(_lim(mesh, alpha_fixed=1.0), U, _lo_dt(mesh, U))
        rho, p = _rho_p(U)
        assert rho.min() > 0 and p.min() > 0
    # the unlimited step loses positivity on the same data at the same dt
    V = U0.copy()
    lost = False
    for _ in range(60):
        V = orc.step(mesh, V, _lo_dt(mesh, U0))
        rho, p = _rho_p(V)
        if not (rho.min() > 0 and p.min() > 0):
            lost = True
            break
    assert lost


def test_conservation_with_the_indicator(orc):
    mesh, U = inputs.shear_layer_2d(cells=(12, 12), N=3)
    m = _lim(mesh, alpha_max=1.0)
    _, a = orc.blend_alpha(m, U)
    assert a.max() > 0.5 and a.min() == 0.0          # both limited and unlimited elements
    T0 = orc.totals(mesh, U)
    A = orc.totals(mesh, np.abs(U))
    for _ in range(100):
        U = orc.step(m, U, orc.cfl_dt(mesh, U))
    T1 = orc.totals(mesh, U)
    for v in range(4):
        scale = max(abs(T0[v]), A[v], A[1:3].max() if v in (1, 2) else 0.0)
        assert abs(T1[v] - T0[v]) / scale < 1e-13, v


def _one_element(dim, N):
    return inputs.mesh_dict("euler", dim, N, [1] * dim, [0.0] * dim, [1.0] * dim, 1.4)


def _state_rho_p(mesh, p_nodes):
    X = inputs.node_coords(mesh)
    one = np.ones_like(X[0])
    return inputs.euler_cons(1.4, one, [0.0 * one] * mesh["dim"], p_nodes)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_indicator_closed_form_1d(orc, N):
    """rho = 1, p = a + b P_N(x): the orthonormal modes are m_0 = a sqrt(2),
    m_N = b sqrt(2/(2N+1)), so E = b^2 / ((2N+1) a^2 + b^2)."""
    mesh = _one_element(1, N)
    x = 2.0 * inputs.gll_points01(N) - 1.0
    c = np.zeros(N + 1)
    c[N] = 1.0
    a, b = 1.0, 0.3
    U = _state_rho_p(mesh, (a + b * L.legval(x, c))[None, :])
    E = orc.indicator_energy(mesh, U[:, 0, :].T)
    assert abs(E - b * b / ((2 * N + 1) * a * a + b * b)) < 1e-14


@pytest.mark.parametrize("N", [2, 3, 5])
def test_indicator_closed_form_2d(orc, N):
    """rho = 1, p = a + b P_N(x) P_N(y): E = b^2 / ((2N+1)^2 a^2 + b^2); a mode
    of degree N - 1 in x only gives the second fraction c^2/((2N-1) a^2 + c^2)."""
    mesh = _one_element(2, N)
    x, y = (2.0 * X - 1.0 for X in inputs.node_coords(mesh))
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    cM = np.zeros(N + 1)
    cM[N - 1] = 1.0
    a, b = 1.0, 0.4
    U = _state_rho_p(mesh, a + b * L.legval(x, cN) * L.legval(y, cN))
    E = orc.indicator_energy(mesh, U[:, 0, :].T)
    assert abs(E - b * b / ((2 * N + 1) ** 2 * a * a + b * b)) < 1e-13
    c = 0.2
    U = _state_rho_p(mesh, a + c * L.legval(x, cM))
    E = orc.indicator_energy(mesh, U[:, 0, :].T)
    assert abs(E - c * c / ((2 * N - 1) * a * a + c * c)) < 1e-13


def test_logistic_map_clipping_and_smoothing(orc):
    N = 3
    T = 0.5 * 10 ** (-1.8 * (N + 1) ** 0.25)
    s = np.log(9999.0)
    # one element (its own neighbour): alpha = logistic(E) with the clips and the cap
    mesh = _one_element(1, N)
    x = 2.0 * inputs.gll_points01(N) - 1.0
    c = np.zeros(N + 1)
    c[N] = 1.0
    for b in (0.002, 0.01, 0.02, 0.05, 0.5):
        U = _state_rho_p(mesh, (1.0 + b * L.legval(x, c))[None, :])
        E = b * b / ((2 * N + 1) + b * b)
        al = 1.0 / (1.0 + np.exp(-s / T * (E - T)))
        al = 0.0 if al < 0.001 else (1.0 if al > 0.999 else al)
        for amax in (1.0, 0.3):
            raw, a = orc.blend_alpha(_lim(mesh, alpha_max=amax), U)
            assert abs(raw[0] - min(al, amax)) < 1e-12 and a[0] == raw[0]
    # smoothing: a limited element raises its face neighbours to half its value
    mesh = inputs.mesh_dict("euler", 1, N, [7], [0.0], [1.0], 1.4)
    (xx,) = inputs.node_coords(mesh)
    p = np.ones_like(xx)
    p[3] = 1.0 + 0.5 * L.legval(x, c)                 # element 3 carries a degree-N mode
    U = _state_rho_p(mesh, p)
    raw, a = orc.blend_alpha(_lim(mesh, alpha_max=0.8), U)
    assert raw[3] == 0.8 and np.all(np.delete(raw, 3) == 0.0)
    assert a[3] == 0.8 and a[2] == 0.4 and a[4] == 0.4 and a[0] == a[1] == a[5] == a[6] == 0.0


def _lo_end_states(mesh, um, up, umi, upi, F, dt, dx, wN, w0):
    dim = mesh["dim"]
    f = lambda a, b: _rusanov(a, b, mesh["gamma"])
    lm = um - dim * dt / (wN * dx) * (F - f(umi, um))
    lp = up - dim * dt / (w0 * dx) * (f(up, upi) - F)
    return lm, lp


def _rusanov(a, b, g):
    fa, la = _euler_flux(a[:, None], 0, g)
    fb, lb = _euler_flux(b[:, None], 0, g)
    return (0.5 * (fa + fb) - 0.5 * np.maximum(la, lb) * (b[:, None] - a[:, None]))[:, 0]


def test_limited_face_flux(orc):
    mesh = inputs.mesh_dict("euler", 1, 3, [4], [0.0], [1.0], 1.4)
    rng = np.random.default_rng(2604021258)
    S = inputs.random_states("euler", 1, 400, seed=2604021259)
    w = _w01(3)
    corrected = 0
    for k in range(100):
        um, up, umi, upi = S[4 * k:4 * k + 4]
        Fho = _rusanov(um, up, 1.4) + rng.normal(0.0, 2.0, 3)      # a high-order flux far from f_lo
        dx, dt = 0.25, 0.05 * rng.uniform(0.1, 1.0)
        flo = _rusanov(um, up, 1.4)
        assert np.array_equal(orc.limited_face_flux(mesh, 0, um, up, umi, upi, Fho, 0.0, dt, dx, w[3], w[0]), Fho)
        F1 = orc.limited_face_flux(mesh, 0, um, up, umi, upi, Fho, 1.0, dt, dx, w[3], w[0])
        assert np.max(np.abs(F1 - flo)) < 1e-14 * np.max(np.abs(flo))
        a_f = rng.uniform(0.05, 0.95)
        F = orc.limited_face_flux(mesh, 0, um, up, umi, upi, Fho, a_f, dt, dx, w[3], w[0])
        Fb = (1 - a_f) * Fho + a_f * flo
        lo = _lo_end_states(mesh, um, up, umi, upi, flo, dt, dx, w[3], w[0])
        got = _lo_end_states(mesh, um, up, umi, upi, F, dt, dx, w[3], w[0])
        blend = _lo_end_states(mesh, um, up, umi, upi, Fb, dt, dx, w[3], w[0])
        ok_lo = all(_rho_p(s[:, None])[0][0] > 0 and _rho_p(s[:, None])[1][0] > 0 for s in lo)
        if not ok_lo:
            continue
        for s0, s1 in zip(lo, got):
            r0, p0 = (v[0] for v in _rho_p(s0[:, None]))
            r1, p1 = (v[0] for v in _rho_p(s1[:, None]))
            assert r1 >= 0.1 * r0 * (1 - 1e-12) and p1 >= 0.1 * p0 * (1 - 1e-12)
        keeps = all(_rho_p(b[:, None])[0][0] >= 0.1 * _rho_p(s0[:, None])[0][0]
                    and _rho_p(b[:, None])[1][0] >= 0.1 * _rho_p(s0[:, None])[1][0] for b, s0 in zip(blend, lo))
        if keeps:
            assert np.max(np.abs(F - Fb)) <= 1e-14 * np.max(np.abs(Fb))
        else:
            corrected += 1
    assert corrected > 5

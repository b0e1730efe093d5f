"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself.  CPU only.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a missing factor 2) fails it:

* GLL points against numpy's Legendre roots; weights against exactness of the
  quadrature; D against exact derivatives of polynomials; SBP property.
* g2 correction derivatives at GLL nodes equal -delta_p0/w_0 and
  +delta_pN/w_N (follows from quadrature exactness, Sec. 2.1 and the
  GLL/g2 choice of Sec. 2.3).
* Butcher tableaux: rooted-tree order conditions to order N+1 (eq. butcher).
* Logarithmic mean against 50-digit mpmath.
* Physical flux + non-conservative term: eigenvalues of f'(u) + B(u) g'(u)
  (eq. flux.and.non.cons) against the textbook wave speeds; Euler flux
  homogeneity f(u) = f'(u) u.
* Two-point fluxes: symmetry and consistency (Sec. 3), Tadmor's condition for
  the EC fluxes (entropy variables pinned against finite differences of the
  entropy), Kennedy-Gruber's kinetic-energy structure.
* Flux differencing with the central flux equals collocation D f and the
  non-conservative product B_p sum_q D_pq g_q (Sec. 3).
* Semi-discrete entropy conservation of EC volume + EC surface fluxes.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs


# --------------------------------------------------------------------------
# reference element
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_gll_points_and_weights(orc, N):
    xi, w, D, dgL, dgR = orc.tables(N)
    np.testing.assert_allclose(xi, inputs.gll_points01(N), rtol=0, atol=2e-15)
    # GLL quadrature on [0,1] is exact for degree <= 2N-1
    for k in range(2 * N):
        assert abs(np.dot(w, xi ** k) - 1.0 / (k + 1)) < 1e-14
    # ... and not for degree 2N
    assert abs(np.dot(w, xi ** (2 * N)) - 1.0 / (2 * N + 1)) > 1e-6


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_differentiation_matrix(orc, N):
    xi, w, D, dgL, dgR = orc.tables(N)
    for k in range(N + 1):
        exact = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** k, exact, atol=1e-12)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12)
    W = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    np.testing.assert_allclose(W @ D + D.T @ W, B, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_g2_correction_derivatives(orc, N):
    xi, w, D, dgL, dgR = orc.tables(N)
    eL = np.zeros(N + 1)
    eL[0] = -1.0 / w[0]
    eR = np.zeros(N + 1)
    eR[N] = 1.0 / w[N]
    np.testing.assert_allclose(dgL, eL, atol=1e-11)
    np.testing.assert_allclose(dgR, eR, atol=1e-11)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_lagrange_basis(orc, N):
    xi = inputs.gll_points01(N)
    for q in range(N + 1):
        for p in range(N + 1):
            assert abs(orc.lagrange(N, q, xi[p]) - (1.0 if p == q else 0.0)) < 1e-13
    s = 0.3141
    assert abs(sum(orc.lagrange(N, q, s) for q in range(N + 1)) - 1.0) < 1e-13


# --------------------------------------------------------------------------
# Butcher tableaux: rooted-tree order conditions
# --------------------------------------------------------------------------
def _trees(order):
    if order == 1:
        return [()]
    out = set()

    def parts(n, mx):
        if n == 0:
            yield []
            return
        for k in range(min(n, mx), 0, -1):
            for rest in parts(n - k, k):
                yield [k] + rest

    for p in parts(order - 1, order - 1):
        for combo in itertools.product(*[_trees(k) for k in p]):
            out.add(tuple(sorted(combo)))
    return sorted(out)


def _size(t):
    return 1 + sum(_size(c) for c in t)


def _gamma(t):
    g = _size(t)
    for c in t:
        g *= _gamma(c)
    return g


def _phi(t, A):
    s = A.shape[0]
    v = np.ones(s)
    for c in t:
        v = v * (A @ _phi(c, A))
    return v


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_butcher_order_conditions(orc, N):
    A, b = orc.butcher(N)
    assert np.allclose(np.triu(A), 0.0)          # explicit: A strictly lower triangular
    for order in range(1, N + 2):
        for t in _trees(order):
            assert abs(b @ _phi(t, A) - 1.0 / _gamma(t)) < 1e-13, (order, t)
    # number of trees: 1, 1, 2, 4, 9, 20 (OEIS A000081) -- checks the tree generator
    assert [len(_trees(k)) for k in range(1, 7)] == [1, 1, 2, 4, 9, 20]


# --------------------------------------------------------------------------
# logarithmic mean
# --------------------------------------------------------------------------
def test_logmean_high_precision(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(7)
    a = rng.uniform(0.1, 10.0, 2000)
    rel = np.concatenate([10.0 ** rng.uniform(-12, 0, 1500), rng.uniform(0.9, 5.0, 500)])
    b = a * (1.0 + rel * rng.choice([-0.5, 0.5], a.size))
    b = np.abs(b) + 1e-3
    worst = 0.0
    for x, y in zip(a, b):
        X, Y = mpmath.mpf(float(x)), mpmath.mpf(float(y))
        ref = X if X == Y else (X - Y) / (mpmath.log(X) - mpmath.log(Y))
        worst = max(worst, abs(float((orc.logmean(x, y) - ref) / ref)))
    assert worst < 1.2e-15, worst   # a few ulp
    assert orc.logmean(1.7, 1.7) == 1.7


# --------------------------------------------------------------------------
# physics: wave structure of f'(u) + B(u) g'(u)
# --------------------------------------------------------------------------
def _jac(fun, u, h=1e-6):
    M = u.size
    J = np.zeros((M, M))
    for k in range(M):
        e = np.zeros(M)
        e[k] = h * max(1.0, abs(u[k]))
        J[:, k] = (fun(u + e) - fun(u - e)) / (2 * e[k])
    return J


def _euler_mesh(dim):
    return inputs.mesh_dict("euler", dim, 3, [4] * dim, [0] * dim, [1] * dim, 1.4)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_flux_eigenvalues(orc, dim):
    mesh = _euler_mesh(dim)
    g = mesh["gamma"]
    for u in inputs.random_states("euler", dim, 20, seed=11 + dim):
        rho = u[0]
        v = u[1:1 + dim] / rho
        p = (g - 1) * (u[-1] - 0.5 * rho * v @ v)
        c = np.sqrt(g * p / rho)
        for d in range(dim):
            J = _jac(lambda x: orc.phys_flux(mesh, d, x), u)
            ev = np.sort(np.linalg.eigvals(J).real)
            ref = np.sort([v[d] - c] + [v[d]] * dim + [v[d] + c])
            np.testing.assert_allclose(ev, ref, atol=1e-6)
            # homogeneity of degree one: f(u) = f'(u) u
            np.testing.assert_allclose(J @ u, orc.phys_flux(mesh, d, u), rtol=1e-7, atol=1e-7)
            assert abs(orc.wave_speed(mesh, d, u) - (abs(v[d]) + c)) < 1e-13
            np.testing.assert_allclose(orc.nc_product(mesh, d, u, u), 0.0)


def _mhd_mesh(c_h=1.3):
    m = inputs.mesh_dict("glm_mhd", 2, 3, [4, 4], [0, 0], [1, 1], 5.0 / 3.0, c_h=c_h)
    return m


def _mhd_prim(u, g):
    rho = u[0]
    v = u[1:4] / rho
    B = u[5:8]
    psi = u[8]
    p = (g - 1) * (u[4] - 0.5 * rho * v @ v - 0.5 * B @ B - 0.5 * psi * psi)
    return rho, v, p, B, psi


def test_glm_mhd_eigenvalues(orc):
    mesh = _mhd_mesh(c_h=2.7)
    g = mesh["gamma"]
    for u in inputs.random_states("glm_mhd", 2, 20, seed=5):
        rho, v, p, B, psi = _mhd_prim(u, g)
        a2 = g * p / rho
        b2 = B @ B / rho
        for d in range(2):
            J = _jac(lambda x: orc.phys_flux(mesh, d, x), u)
            # B(u) g'(u): nc_product is linear in its second argument
            J += _jac(lambda x: orc.nc_product(mesh, d, u, x), u)
            ev = np.sort(np.linalg.eigvals(J).real)
            bd2 = B[d] ** 2 / rho
            disc = np.sqrt((a2 + b2) ** 2 - 4 * a2 * bd2)
            cf = np.sqrt(0.5 * (a2 + b2 + disc))
            cs = np.sqrt(max(0.5 * (a2 + b2 - disc), 0.0))
            ca = np.sqrt(bd2)
            # the GLM cleaning pair moves with the flow: v_d -+ c_h
            ref = np.sort([v[d] - cf, v[d] - ca, v[d] - cs, v[d], v[d] + cs, v[d] + ca, v[d] + cf,
                           v[d] - mesh["c_h"], v[d] + mesh["c_h"]])
            np.testing.assert_allclose(ev, ref, atol=2e-5)
            lam = abs(v[d]) + max(cf, mesh["c_h"])
            assert abs(orc.wave_speed(mesh, d, u) - lam) < 1e-12


# --------------------------------------------------------------------------
# two-point fluxes
# --------------------------------------------------------------------------
def _entropy(u, g, eq):
    if eq == "euler":
        rho = u[0]
        m = u[1:-1]
        p = (g - 1) * (u[-1] - 0.5 * m @ m / rho)
    else:
        rho, v, p, B, psi = _mhd_prim(u, g)
    s = np.log(p) - g * np.log(rho)
    return -rho * s / (g - 1)


def _entropy_vars(u, g, eq):
    """Closed-form entropy variables (pinned below against finite differences)."""
    if eq == "euler":
        rho = u[0]
        v = u[1:-1] / rho
        p = (g - 1) * (u[-1] - 0.5 * rho * v @ v)
        s = np.log(p) - g * np.log(rho)
        return np.concatenate([[(g - s) / (g - 1) - rho * v @ v / (2 * p)], rho * v / p, [-rho / p]])
    rho, v, p, B, psi = _mhd_prim(u, g)
    s = np.log(p) - g * np.log(rho)
    beta = rho / (2 * p)
    return np.concatenate([[(g - s) / (g - 1) - beta * v @ v], 2 * beta * v, [-2 * beta], 2 * beta * B,
                           [2 * beta * psi]])


@pytest.mark.parametrize("eq,dim", [("euler", 1), ("euler", 2), ("euler", 3), ("glm_mhd", 2)])
def test_entropy_variables_are_entropy_gradient(orc, eq, dim):
    g = 1.4 if eq == "euler" else 5.0 / 3.0
    for u in inputs.random_states(eq, dim, 5, seed=3):
        fd = np.array([(_entropy(u + e, g, eq) - _entropy(u - e, g, eq)) / (2e-6)
                       for e in np.eye(u.size) * 1e-6])
        np.testing.assert_allclose(_entropy_vars(u, g, eq), fd, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("vol", ["ec", "kep", "central"])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_two_point_symmetric_consistent(orc, vol, dim):
    mesh = _euler_mesh(dim)
    mesh["vol"] = vol
    S = inputs.random_states("euler", dim, 60, seed=21)
    for uL, uR in zip(S[:30], S[30:]):
        for d in range(dim):
            f1 = orc.two_point_flux(mesh, d, uL, uR)
            f2 = orc.two_point_flux(mesh, d, uR, uL)
            np.testing.assert_allclose(f1, f2, rtol=1e-14, atol=1e-14)
            np.testing.assert_allclose(orc.two_point_flux(mesh, d, uL, uL), orc.phys_flux(mesh, d, uL),
                                       rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_ranocha_tadmor(orc, dim):
    mesh = _euler_mesh(dim)
    g = mesh["gamma"]
    S = inputs.random_states("euler", dim, 2000, seed=31)
    for uL, uR in zip(S[:1000], S[1000:]):
        d = int(uL[0] * 1000) % dim
        f = orc.two_point_flux(mesh, d, uL, uR)
        wL, wR = _entropy_vars(uL, g, "euler"), _entropy_vars(uR, g, "euler")
        psiL, psiR = uL[1 + d], uR[1 + d]                 # psi = rho v_d
        lhs = (wR - wL) @ f
        scale = np.abs(wR - wL) @ np.abs(f) + abs(psiR) + abs(psiL)
        assert abs(lhs - (psiR - psiL)) < 1e-13 * scale


def test_euler_ranocha_tadmor_fails_for_kep(orc):
    """The Tadmor check is sharp: the KG flux (not EC) violates it."""
    mesh = _euler_mesh(2)
    mesh["vol"] = "kep"
    g = mesh["gamma"]
    S = inputs.random_states("euler", 2, 20, seed=32)
    worst = 0.0
    for uL, uR in zip(S[:10], S[10:]):
        f = orc.two_point_flux(mesh, 0, uL, uR)
        worst = max(worst, abs((_entropy_vars(uR, g, "euler") - _entropy_vars(uL, g, "euler")) @ f - (uR[1] - uL[1])))
    assert worst > 1e-4


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kennedy_gruber_kep_structure(orc, dim):
    """KEP (Jameson's condition): momentum flux = f_rho * {{v}} + p_avg n."""
    mesh = _euler_mesh(dim)
    mesh["vol"] = "kep"
    g = mesh["gamma"]
    S = inputs.random_states("euler", dim, 40, seed=41)
    for uL, uR in zip(S[:20], S[20:]):
        vL, vR = uL[1:-1] / uL[0], uR[1:-1] / uR[0]
        pL = (g - 1) * (uL[-1] - 0.5 * uL[0] * vL @ vL)
        pR = (g - 1) * (uR[-1] - 0.5 * uR[0] * vR @ vR)
        for d in range(dim):
            f = orc.two_point_flux(mesh, d, uL, uR)
            mom = f[0] * 0.5 * (vL + vR)
            mom[d] += 0.5 * (pL + pR)
            np.testing.assert_allclose(f[1:-1], mom, rtol=1e-13, atol=1e-14)
            # mass flux uses arithmetic means only
            assert abs(f[0] - 0.25 * (uL[0] + uR[0]) * (vL[d] + vR[d])) < 1e-14


def test_glm_mhd_ec_flux(orc):
    """Symmetry, consistency and the entropy condition with the Powell term:
    [[w]].f = [[psi]] + {{theta}} [[B_d]], psi = w.f - F, theta = w.phi_Powell."""
    mesh = _mhd_mesh(c_h=1.7)
    g = mesh["gamma"]
    S = inputs.random_states("glm_mhd", 2, 1000, seed=51)
    for uL, uR in zip(S[:500], S[500:]):
        for d in range(2):
            f = orc.two_point_flux(mesh, d, uL, uR)
            np.testing.assert_allclose(f, orc.two_point_flux(mesh, d, uR, uL), rtol=1e-13, atol=1e-13)
            wL, wR = _entropy_vars(uL, g, "glm_mhd"), _entropy_vars(uR, g, "glm_mhd")

            def psi(u, w):
                rho, v, p, B, ps = _mhd_prim(u, g)
                F = -rho * v[d] * (np.log(p) - g * np.log(rho)) / (g - 1)
                return w @ orc.phys_flux(mesh, d, u) - F

            def theta(u):
                rho, v, p, B, ps = _mhd_prim(u, g)
                return rho * (v @ B) / p

            lhs = (wR - wL) @ f
            rhs = psi(uR, wR) - psi(uL, wL) + 0.5 * (theta(uL) + theta(uR)) * (uR[5 + d] - uL[5 + d])
            scale = np.abs(wR - wL) @ np.abs(f) + abs(psi(uR, wR)) + abs(psi(uL, wL))
            assert abs(lhs - rhs) < 2e-13 * scale
    u = S[0]
    for d in range(2):
        np.testing.assert_allclose(orc.two_point_flux(mesh, d, u, u), orc.phys_flux(mesh, d, u), rtol=1e-13, atol=1e-13)


def test_glm_mhd_entropy_potential_closed_form(orc):
    """psi = w.f - F equals rho v_d + beta v_d |B|^2 - 2 beta B_d (v.B) + 2 beta c_h psi B_d."""
    mesh = _mhd_mesh(c_h=1.1)
    g = mesh["gamma"]
    for u in inputs.random_states("glm_mhd", 2, 20, seed=52):
        rho, v, p, B, ps = _mhd_prim(u, g)
        beta = rho / (2 * p)
        w = _entropy_vars(u, g, "glm_mhd")
        for d in range(2):
            F = -rho * v[d] * (np.log(p) - g * np.log(rho)) / (g - 1)
            psi = w @ orc.phys_flux(mesh, d, u) - F
            ref = rho * v[d] + beta * v[d] * (B @ B) - 2 * beta * B[d] * (v @ B) + 2 * beta * mesh["c_h"] * ps * B[d]
            assert abs(psi - ref) < 1e-12 * (1 + abs(ref))


# --------------------------------------------------------------------------
# flux differencing reduces to collocation for the central flux (Sec. 3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("eq,dim,N", [("euler", 1, 3), ("euler", 2, 2), ("euler", 3, 3), ("glm_mhd", 2, 4),
                                      ("euler", 2, 5)])
def test_central_flux_differencing_is_collocation(orc, eq, dim, N):
    if eq == "euler":
        mesh = inputs.mesh_dict("euler", dim, N, [3] * dim, [0] * dim, [1.5] * dim, 1.4, vol="central")
    else:
        mesh = inputs.mesh_dict("glm_mhd", 2, N, [3, 2], [0, 0], [1.5, 1.0], 5.0 / 3.0, vol="central", c_h=1.0)
    U = inputs.smooth_random_field(mesh, seed=61, amp=0.2)
    M, E, npe = U.shape
    xi, w, D, _, _ = orc.tables(N)
    n = N + 1
    e = 1
    ue = U[:, e, :].T.copy()                     # [node][var]
    R = orc.local_residual(mesh, ue)
    dx = [(mesh["hi"][k] - mesh["lo"][k]) / mesh["cells"][k] for k in range(dim)]
    ref = np.zeros_like(ue)
    shape = (n,) * dim
    for p in range(npe):
        ijk = np.unravel_index(p, shape[::-1])[::-1]       # i fastest
        for d in range(dim):
            for qd in range(n):
                qijk = list(ijk)
                qijk[d] = qd
                q = np.ravel_multi_index(tuple(qijk[::-1]), shape[::-1])
                ref[p] += D[ijk[d], qd] * orc.phys_flux(mesh, d, ue[q]) / dx[d]
                # B(u_p) g(u_q) summed with D (no factor 2)
                ref[p] += D[ijk[d], qd] * orc.nc_product(mesh, d, ue[p], ue[q]) / dx[d]
    np.testing.assert_allclose(R, ref, rtol=1e-12, atol=1e-11)


# --------------------------------------------------------------------------
# semi-discrete entropy conservation (EC volume + EC surface), Sec. 3
# --------------------------------------------------------------------------
@pytest.mark.parametrize("eq,dim,N", [("euler", 1, 3), ("euler", 2, 3), ("euler", 3, 2), ("glm_mhd", 2, 3),
                                      ("glm_mhd", 2, 4), ("euler", 2, 5)])
def test_semidiscrete_entropy_conservation(orc, eq, dim, N):
    if eq == "euler":
        mesh = inputs.mesh_dict("euler", dim, N, [3] * dim, [0] * dim, [2.0] * dim, 1.4, vol="ec", surf="ec")
    else:
        mesh = inputs.mesh_dict("glm_mhd", 2, N, [3, 3], [0, 0], [1.0, 1.0], 5.0 / 3.0, vol="ec", surf="ec",
                                c_h=1.2)
    U = inputs.smooth_random_field(mesh, seed=71, amp=0.3)
    rhs = orc.fr_rhs(mesh, U)
    xi, w, *_ = orc.tables(N)
    n = N + 1
    Wn = np.ones(n ** dim)
    for p in range(n ** dim):
        ijk = np.unravel_index(p, (n,) * dim)[::-1]
        for k in ijk:
            Wn[p] *= w[k]
    g = mesh["gamma"]
    M, E, npe = U.shape
    total, scale = 0.0, 0.0
    for e in range(E):
        for p in range(npe):
            wv = _entropy_vars(U[:, e, p], g, eq)
            total += Wn[p] * wv @ rhs[:, e, p]
            scale += Wn[p] * np.abs(wv) @ np.abs(rhs[:, e, p])
    assert abs(total) < 1e-13 * scale, (total, scale)
    # with the dissipative Rusanov surface flux entropy decays (noisy data, so
    # that the interface jumps are not negligible)
    mesh["surf"] = "rusanov"
    rng = np.random.default_rng(72)
    U = U * (1.0 + 1e-2 * rng.standard_normal(U.shape))
    rhs = orc.fr_rhs(mesh, U)
    total = sum(Wn[p] * _entropy_vars(U[:, e, p], g, eq) @ rhs[:, e, p] for e in range(E) for p in range(npe))
    scale = sum(Wn[p] * np.abs(_entropy_vars(U[:, e, p], g, eq)) @ np.abs(rhs[:, e, p])
                for e in range(E) for p in range(npe))
    assert total < -1e-8 * scale, (total, scale)

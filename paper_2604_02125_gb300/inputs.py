"""Seeded synthetic initial states for the cRKFR workloads.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle: it produces FP64 conserved-variable arrays in the library's
layout [var][elem][node] (node index i fastest, then j, k; element index x
fastest) and plain mesh dicts.  It contains none of the method's arithmetic:
GLL point positions come from numpy's Legendre routines, and the only physics
is the conversion of primitive initial data to conserved variables.

Mesh dict keys: eq ('euler' | 'glm_mhd'), dim, N, cells, lo, hi, gamma, cfl,
c_h, vol ('ec' | 'kep' | 'central'), surf ('rusanov'); optional, read by the
library binding and the oracle: scheme ('crkfr' | 'rkfr'), ncflux ('reduced' |
'stages', GLM-MHD).

Workloads (the paper's own test cases need a limiter or equations that are not
printed, so these smooth periodic problems stand in for them):
  density_wave_1d   1D Euler density wave rho = 1 + 0.5 sin(pi x), u = 1, p = 1
  shear_layer_2d    2D Euler shear layer (Kelvin-Helmholtz-type initial data)
  mhd_vortex_2d     2D ideal GLM-MHD Orszag-Tang-type vortex with noise
  tgv_3d            3D Euler Taylor-Green vortex at Mach 0.1
  batched_2d        512 independent 2D Euler solves of uneven size and degree
"""
import math

import numpy as np
from numpy.polynomial import legendre as _leg

SEEDS = {"shear_layer_2d": 2604021252, "mhd_vortex_2d": 2604021253,
         "batched_2d": 2604021254}


def default_cfl(N):
    """CFL number per degree (reading of the paper's unstated time step rule)."""
    return {1: 0.1, 2: 0.1, 3: 0.1, 4: 0.07, 5: 0.05}[N]


def gll_points01(N):
    """GLL points on [0,1]: the endpoints and the roots of P_N' (numpy)."""
    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(_leg.legroots(_leg.legder(c)))) if N > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (x + 1.0)


def nvars(mesh):
    return mesh["dim"] + 2 if mesh.get("eq", "euler") == "euler" else 9


def num_elems(mesh):
    return int(np.prod(mesh["cells"][:mesh["dim"]]))


def nodes_per_elem(mesh):
    return (mesh["N"] + 1) ** mesh["dim"]


def node_coords(mesh):
    """Physical coordinates of every node: list (per dim) of [elem][node] arrays."""
    dim, N = mesh["dim"], mesh["N"]
    xi = gll_points01(N)
    n = N + 1
    cells = mesh["cells"][:dim]
    E = num_elems(mesh)
    e = np.arange(E)
    ec = []
    rem = e.copy()
    for k in range(dim):
        ec.append(rem % cells[k])
        rem //= cells[k]
    p = np.arange(n ** dim)
    pc = []
    rem = p.copy()
    for k in range(dim):
        pc.append(rem % n)
        rem //= n
    X = []
    for k in range(dim):
        dx = (mesh["hi"][k] - mesh["lo"][k]) / cells[k]
        X.append(mesh["lo"][k] + (ec[k][:, None] + xi[pc[k]][None, :]) * dx)
    return X


def euler_cons(gamma, rho, vel, p):
    """Primitive (rho, v, p) -> conserved (rho, rho v, E) as [var][elem][node]."""
    out = [rho] + [rho * v for v in vel]
    E = p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    out.append(E)
    return np.ascontiguousarray(np.stack(out).astype(np.float64))


def mhd_cons(gamma, rho, vel, p, B, psi):
    """Primitive -> conserved GLM-MHD (rho, rho v1..3, E, B1..3, psi)."""
    E = (p / (gamma - 1.0) + 0.5 * rho * sum(v * v for v in vel)
         + 0.5 * sum(b * b for b in B) + 0.5 * psi * psi)
    out = [rho, rho * vel[0], rho * vel[1], rho * vel[2], E, B[0], B[1], B[2], psi]
    return np.ascontiguousarray(np.stack(out).astype(np.float64))


def mesh_dict(eq, dim, N, cells, lo, hi, gamma, vol="ec", cfl=None, c_h=0.0, surf="rusanov"):
    cells = list(cells) + [1] * (3 - len(cells))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    return {"eq": eq, "dim": dim, "N": N, "cells": cells, "lo": lo, "hi": hi,
            "gamma": gamma, "cfl": default_cfl(N) if cfl is None else cfl,
            "c_h": c_h, "vol": vol, "surf": surf}


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def density_wave_1d(cells=64, N=3, vol="ec", cfl=0.1):
    """1D Euler, periodic [0,2], rho = 1 + 0.5 sin(pi x), u = 1, p = 1, gamma 1.4.
    Exact solution rho(x - t)."""
    mesh = mesh_dict("euler", 1, N, [cells], [0.0], [2.0], 1.4, vol=vol, cfl=cfl)
    (x,) = node_coords(mesh)
    rho = 1.0 + 0.5 * np.sin(np.pi * x)
    return mesh, euler_cons(1.4, rho, [np.ones_like(x)], np.ones_like(x))


def density_wave_exact_1d(mesh, t):
    (x,) = node_coords(mesh)
    return 1.0 + 0.5 * np.sin(np.pi * (x - t))


def density_wave_2d(cells=(16, 16), N=3, vol="ec", cfl=0.1):
    """2D Euler density wave along the diagonal: rho = 1 + 0.5 sin(pi(x + y)),
    v = (1, 1), p = 1 on [0,2]^2 (exact solution rho(x + y - 2t))."""
    mesh = mesh_dict("euler", 2, N, list(cells), [0.0, 0.0], [2.0, 2.0], 1.4, vol=vol, cfl=cfl)
    x, y = node_coords(mesh)
    rho = 1.0 + 0.5 * np.sin(np.pi * (x + y))
    one = np.ones_like(x)
    return mesh, euler_cons(1.4, rho, [one, one], one)


def shear_layer_2d(cells=(256, 256), N=3, vol="ec", seed=SEEDS["shear_layer_2d"], cfl=None):
    """2D Euler shear layer on periodic [-1,1]^2: B = tanh(15y+7.5) - tanh(15y-7.5),
    rho = 0.5 + 0.75 B, vx = 0.5 (B - 1), vy = 0.1 sin(pi x) + 1e-3 N(0,1) per node, p = 1."""
    mesh = mesh_dict("euler", 2, N, list(cells), [-1.0, -1.0], [1.0, 1.0], 1.4, vol=vol, cfl=cfl)
    x, y = node_coords(mesh)
    rng = np.random.default_rng(seed)
    B = np.tanh(15.0 * y + 7.5) - np.tanh(15.0 * y - 7.5)
    rho = 0.5 + 0.75 * B
    vx = 0.5 * (B - 1.0)
    vy = 0.1 * np.sin(np.pi * x) + 1e-3 * rng.standard_normal(x.shape)
    return mesh, euler_cons(1.4, rho, [vx, vy], np.ones_like(x))


def mhd_vortex_2d(cells=(128, 128), N=4, vol="ec", seed=SEEDS["mhd_vortex_2d"], cfl=None):
    """2D ideal GLM-MHD on periodic [0,1]^2, gamma = 5/3:
    rho = 25/(36 pi), p = 5/(12 pi), v = (-sin 2pi y, sin 2pi x, 0) + 1e-3 N(0,1),
    B = (-sin 2pi y, sin 4pi x, 0)/sqrt(4 pi), psi = 0.  The GLM cleaning speed
    c_h is fixed to an upper bound of the initial fast speed:
    max|v| + sqrt(max(gamma p/rho + |B|^2/rho))."""
    g = 5.0 / 3.0
    mesh = mesh_dict("glm_mhd", 2, N, list(cells), [0.0, 0.0], [1.0, 1.0], g, vol=vol, cfl=cfl)
    x, y = node_coords(mesh)
    rng = np.random.default_rng(seed)
    rho = np.full_like(x, 25.0 / (36.0 * np.pi))
    p = np.full_like(x, 5.0 / (12.0 * np.pi))
    v1 = -np.sin(2 * np.pi * y) + 1e-3 * rng.standard_normal(x.shape)
    v2 = np.sin(2 * np.pi * x) + 1e-3 * rng.standard_normal(x.shape)
    v3 = np.zeros_like(x)
    s = 1.0 / np.sqrt(4.0 * np.pi)
    B1 = -np.sin(2 * np.pi * y) * s
    B2 = np.sin(4 * np.pi * x) * s
    B3 = np.zeros_like(x)
    vmax = float(np.max(np.abs(np.stack([v1, v2]))))
    cmax = float(np.sqrt(np.max(g * p / rho + (B1 * B1 + B2 * B2 + B3 * B3) / rho)))
    mesh["c_h"] = vmax + cmax
    return mesh, mhd_cons(g, rho, [v1, v2, v3], p, [B1, B2, B3], np.zeros_like(x))


def tgv_3d(cells=(64, 64, 64), N=3, vol="ec", mach=0.1, cfl=None):
    """3D Euler Taylor-Green vortex on periodic [0,2pi]^3, gamma 1.4, rho = 1,
    v = (sin x cos y cos z, -cos x sin y cos z, 0),
    p = 1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16."""
    g = 1.4
    tp = 2.0 * math.pi
    mesh = mesh_dict("euler", 3, N, list(cells), [0.0] * 3, [tp] * 3, g, vol=vol, cfl=cfl)
    x, y, z = node_coords(mesh)
    rho = np.ones_like(x)
    v1 = np.sin(x) * np.cos(y) * np.cos(z)
    v2 = -np.cos(x) * np.sin(y) * np.cos(z)
    v3 = np.zeros_like(x)
    p = 1.0 / (g * mach * mach) + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return mesh, euler_cons(g, rho, [v1, v2, v3], p)


def batched_2d_specs(n_solves=512, seed=SEEDS["batched_2d"], side_lo=16, side_hi=128,
                     degrees=(2, 3, 4, 5)):
    """Parameters of the batched workload: per solve a square side n ~ U{16..128},
    degree N ~ U{2,3,4,5}, amplitude a ~ U[0.1,0.5], wave numbers k in {1,2},
    shear amplitude b ~ U[0.01,0.1]."""
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(n_solves):
        side = int(rng.integers(side_lo, side_hi + 1))
        N = int(rng.choice(degrees))
        a = float(rng.uniform(0.1, 0.5))
        kx, ky = (int(k) for k in rng.integers(1, 3, size=2))
        b = float(rng.uniform(0.01, 0.1))
        specs.append({"side": side, "N": N, "a": a, "kx": kx, "ky": ky, "b": b})
    return specs


def batched_2d_solve(spec, vol="ec"):
    """One solve of the batched workload: periodic [-1,1]^2,
    rho = 1 + a sin(pi(kx x + ky y)), v = (0.5 + b sin(pi y), b sin(pi x)), p = 1."""
    mesh = mesh_dict("euler", 2, spec["N"], [spec["side"], spec["side"]],
                     [-1.0, -1.0], [1.0, 1.0], 1.4, vol=vol)
    x, y = node_coords(mesh)
    rho = 1.0 + spec["a"] * np.sin(np.pi * (spec["kx"] * x + spec["ky"] * y))
    vx = 0.5 + spec["b"] * np.sin(np.pi * y)
    vy = spec["b"] * np.sin(np.pi * x)
    return mesh, euler_cons(1.4, rho, [vx, vy], np.ones_like(x))


def random_states(eq, dim, count, seed, gamma=None):
    """Seeded random physical point states (for point-wise flux tests):
    rho in [0.5, 2], |v_k| <= 1, p in [0.5, 2]; MHD adds B_k in [-1,1], psi in [-0.5,0.5].
    Returns an array [count][M] of conserved variables."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, count)
    p = rng.uniform(0.5, 2.0, count)
    if eq == "euler":
        g = 1.4 if gamma is None else gamma
        vel = [rng.uniform(-1.0, 1.0, count) for _ in range(dim)]
        return euler_cons(g, rho, vel, p).T.copy()
    g = 5.0 / 3.0 if gamma is None else gamma
    vel = [rng.uniform(-1.0, 1.0, count) for _ in range(3)]
    B = [rng.uniform(-1.0, 1.0, count) for _ in range(3)]
    psi = rng.uniform(-0.5, 0.5, count)
    return mhd_cons(g, rho, vel, p, B, psi).T.copy()


def smooth_random_field(mesh, seed, amp=0.05):
    """A smooth seeded perturbation of a constant state (rho=1, v=0.1.., p=1)
    made of a few random Fourier modes: used for small parity cases."""
    rng = np.random.default_rng(seed)
    X = node_coords(mesh)
    dim = mesh["dim"]

    def field():
        f = np.zeros_like(X[0])
        for _ in range(3):
            k = rng.integers(1, 3, size=dim)
            ph = rng.uniform(0, 2 * np.pi)
            arg = ph + sum(np.pi * k[d] * (X[d] - mesh["lo"][d]) * 2.0 / (mesh["hi"][d] - mesh["lo"][d])
                           for d in range(dim))
            f += rng.uniform(-1, 1) * np.sin(arg)
        return f

    rho = 1.0 + amp * field()
    p = 1.0 + amp * field()
    g = mesh["gamma"]
    if mesh.get("eq", "euler") == "euler":
        vel = [0.3 + amp * field() for _ in range(dim)]
        return euler_cons(g, rho, vel, p)
    vel = [0.3 + amp * field() for _ in range(3)]
    B = [0.5 + amp * field() for _ in range(3)]
    psi = amp * field()
    return mhd_cons(g, rho, vel, p, B, psi)

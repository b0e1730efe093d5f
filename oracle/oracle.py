"""ctypes binding of the plain-C FP64 oracle (crkfr_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  Nothing in the product package
imports it.  The oracle is compiled with gcc (-O2, no fast-math, no FMA
contraction) so that it gives the same bits on x86_64 and aarch64.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crkfr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

EQ = {"euler": 0, "glm_mhd": 1}
VOL = {"ec": 0, "kep": 1, "central": 2}
SURF = {"rusanov": 0, "ec": 1}
NCFLUX = {"reduced": 0, "stages": 1}


def build(force=False):
    """Compile the oracle shared library (gcc) if it is missing or stale."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Desc(ctypes.Structure):
    _fields_ = [("eq", ctypes.c_int), ("dim", ctypes.c_int), ("N", ctypes.c_int),
                ("cells", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("gamma", ctypes.c_double),
                ("cfl", ctypes.c_double), ("c_h", ctypes.c_double),
                ("vol", ctypes.c_int), ("surf", ctypes.c_int), ("ncflux", ctypes.c_int),
                ("tab_s", ctypes.c_int), ("tab_A", ctypes.POINTER(ctypes.c_double)),
                ("tab_b", ctypes.POINTER(ctypes.c_double)), ("limiter", ctypes.c_int),
                ("alpha_max", ctypes.c_double), ("alpha_fixed", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(Desc)
        _lib.or_tables.argtypes = [ctypes.c_int, D, D, D, D, D]
        _lib.or_lagrange.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        _lib.or_lagrange.restype = ctypes.c_double
        _lib.or_butcher.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), D, D]
        _lib.or_logmean.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.or_logmean.restype = ctypes.c_double
        for name in ("or_phys_flux",):
            getattr(_lib, name).argtypes = [P, ctypes.c_int, D, D]
        _lib.or_two_point_flux.argtypes = [P, ctypes.c_int, D, D, D]
        _lib.or_nc_product.argtypes = [P, ctypes.c_int, D, D, D]
        _lib.or_wave_speed.argtypes = [P, ctypes.c_int, D]
        _lib.or_wave_speed.restype = ctypes.c_double
        _lib.or_cfl_dt.argtypes = [P, D]
        _lib.or_cfl_dt.restype = ctypes.c_double
        _lib.or_step.argtypes = [P, D, ctypes.c_double, D]
        _lib.or_step_elements.argtypes = [P, D, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int), D]
        _lib.or_element_stages.argtypes = [P, D, ctypes.c_double, D, D, D, D]
        _lib.or_local_residual.argtypes = [P, D, D]
        _lib.or_fr_rhs.argtypes = [P, D, D]
        _lib.or_rkfr_step.argtypes = [P, D, ctypes.c_double, D]
        _lib.or_totals.argtypes = [P, D, D]
        _lib.or_blend_alpha.argtypes = [P, D, D, D]
        _lib.or_indicator_energy.argtypes = [P, D]
        _lib.or_indicator_energy.restype = ctypes.c_double
        _lib.or_limited_face_flux.argtypes = [P, ctypes.c_int, D, D, D, D, D] + [ctypes.c_double] * 5 + [D]
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_desc(mesh):
    """Build the oracle descriptor from a mesh dict (keys as in
    paper_2604_02125_gb300.inputs: eq, dim, N, cells, lo, hi, gamma, cfl,
    c_h, vol, surf; optional: ncflux 'reduced' | 'stages' (the non-conservative
    numerical flux of the cRKFR step), tableau (A, b): an explicit RK tableau
    of s <= 7 stages in place of the degree's, limiter (bool: subcell blending),
    alpha_max, alpha_fixed (a blending coefficient forced in every element))."""
    d = Desc()
    d.eq = EQ[mesh.get("eq", "euler")]
    d.dim = mesh["dim"]
    d.N = mesh["N"]
    cells = list(mesh["cells"]) + [1] * (3 - len(mesh["cells"]))
    lo = list(mesh["lo"]) + [0.0] * (3 - len(mesh["lo"]))
    hi = list(mesh["hi"]) + [1.0] * (3 - len(mesh["hi"]))
    for k in range(3):
        d.cells[k] = cells[k]
        d.lo[k] = lo[k]
        d.hi[k] = hi[k]
    d.gamma = mesh.get("gamma", 1.4)
    d.cfl = mesh.get("cfl", 0.1)
    d.c_h = mesh.get("c_h", 0.0)
    d.vol = VOL[mesh.get("vol", "ec")]
    d.surf = SURF[mesh.get("surf", "rusanov")]
    d.ncflux = NCFLUX[mesh.get("ncflux", "reduced")]
    d.limiter = 1 if mesh.get("limiter") else 0
    d.alpha_max = float(mesh.get("alpha_max", 1.0))
    af = mesh.get("alpha_fixed")
    d.alpha_fixed = -1.0 if af is None else float(af)
    if mesh.get("tableau") is not None:
        A, b = mesh["tableau"]
        s = len(b)
        A7 = np.zeros((7, 7))
        A7[:s, :s] = np.asarray(A, dtype=np.float64)[:s, :s]
        b7 = np.zeros(7)
        b7[:s] = b
        d._keep = (A7, b7)            # the descriptor points into these arrays
        d.tab_s = s
        d.tab_A = _ptr(A7)
        d.tab_b = _ptr(b7)
    return d


def nvars(mesh):
    return mesh["dim"] + 2 if mesh.get("eq", "euler") == "euler" else 9


def tables(N):
    n = N + 1
    xi, w, dgL, dgR = (np.zeros(n) for _ in range(4))
    D = np.zeros((n, n))
    rc = lib().or_tables(N, _ptr(xi), _ptr(w), _ptr(D), _ptr(dgL), _ptr(dgR))
    if rc:
        raise ValueError("bad N")
    return xi, w, D, dgL, dgR


def lagrange(N, q, s):
    return lib().or_lagrange(N, q, s)


def butcher(N):
    s = ctypes.c_int(0)
    A = np.zeros((7, 7))
    b = np.zeros(7)
    if lib().or_butcher(N, ctypes.byref(s), _ptr(A), _ptr(b)):
        raise ValueError("bad N")
    return A[:s.value, :s.value].copy(), b[:s.value].copy()


def logmean(a, b):
    return lib().or_logmean(float(a), float(b))


def phys_flux(mesh, direction, u):
    d = make_desc(mesh)
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(nvars(mesh))
    lib().or_phys_flux(ctypes.byref(d), direction, _ptr(u), _ptr(f))
    return f


def two_point_flux(mesh, direction, uL, uR):
    d = make_desc(mesh)
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    f = np.zeros(nvars(mesh))
    lib().or_two_point_flux(ctypes.byref(d), direction, _ptr(uL), _ptr(uR), _ptr(f))
    return f


def nc_product(mesh, direction, ua, ub):
    d = make_desc(mesh)
    ua = np.ascontiguousarray(ua, dtype=np.float64)
    ub = np.ascontiguousarray(ub, dtype=np.float64)
    out = np.zeros(nvars(mesh))
    lib().or_nc_product(ctypes.byref(d), direction, _ptr(ua), _ptr(ub), _ptr(out))
    return out


def wave_speed(mesh, direction, u):
    d = make_desc(mesh)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_wave_speed(ctypes.byref(d), direction, _ptr(u))


def cfl_dt(mesh, U):
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().or_cfl_dt(ctypes.byref(d), _ptr(U))


def step(mesh, U, dt):
    """One cRKFR step with the given dt; U is [var][elem][node] FP64."""
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    if lib().or_step(ctypes.byref(d), _ptr(U), float(dt), _ptr(out)):
        raise ValueError("oracle rejected the mesh descriptor")
    return out


def step_elements(mesh, U, dt, elems):
    """The step's result for the listed elements only: [var][k][node] for
    elems[k] (stages of those elements and their neighbours, then their update)."""
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    sel = np.ascontiguousarray(elems, dtype=np.int32)
    out = np.empty((U.shape[0], len(sel), U.shape[2]), dtype=np.float64)
    if lib().or_step_elements(ctypes.byref(d), _ptr(U), float(dt), len(sel),
                              sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(out)):
        raise ValueError("oracle rejected the mesh descriptor or an element index")
    return out


def run(mesh, U, nsteps, dt_fixed=None):
    """nsteps steps; dt from the CFL rule on each step's u^n unless dt_fixed.
    Returns (U, list of dt)."""
    dts = []
    for _ in range(nsteps):
        dt = dt_fixed if dt_fixed is not None else cfl_dt(mesh, U)
        U = step(mesh, U, dt)
        dts.append(dt)
    return U, dts


def rkfr_step(mesh, U, dt):
    """One multi-stage RKFR step (eq. rkfr.non.cons: the degree's RK tableau on
    the semi-discrete FR system, one face exchange per stage) with the given
    dt; U is [var][elem][node] FP64."""
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    if lib().or_rkfr_step(ctypes.byref(d), _ptr(U), float(dt), _ptr(out)):
        raise ValueError("oracle rejected the mesh descriptor")
    return out


def rkfr_run(mesh, U, nsteps, dt_fixed=None):
    """nsteps RKFR steps, dt as in run().  Returns (U, list of dt)."""
    dts = []
    for _ in range(nsteps):
        dt = dt_fixed if dt_fixed is not None else cfl_dt(mesh, U)
        U = rkfr_step(mesh, U, dt)
        dts.append(dt)
    return U, dts


def local_residual(mesh, ue):
    """R(u) of one element; ue is [node][var]."""
    d = make_desc(mesh)
    ue = np.ascontiguousarray(ue, dtype=np.float64)
    R = np.zeros_like(ue)
    lib().or_local_residual(ctypes.byref(d), _ptr(ue), _ptr(R))
    return R


def element_stages(mesh, ue, dt):
    d = make_desc(mesh)
    ue = np.ascontiguousarray(ue, dtype=np.float64)
    Rbar = np.zeros_like(ue)
    Ubar = np.zeros_like(ue)
    Fbar = np.zeros((mesh["dim"],) + ue.shape)
    Fnc = np.zeros((mesh["dim"],) + ue.shape)
    lib().or_element_stages(ctypes.byref(d), _ptr(ue), float(dt), _ptr(Rbar), _ptr(Ubar), _ptr(Fbar), _ptr(Fnc))
    return Rbar, Ubar, Fbar, Fnc


def fr_rhs(mesh, U):
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    if lib().or_fr_rhs(ctypes.byref(d), _ptr(U), _ptr(out)):
        raise ValueError("oracle rejected the mesh descriptor")
    return out


def totals(mesh, U):
    """[M] conserved totals, kinetic energy, entropy (FP64, quadrature-weighted)."""
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(nvars(mesh) + 2)
    lib().or_totals(ctypes.byref(d), _ptr(U), _ptr(out))
    return out


def blend_alpha(mesh, U):
    """(raw, smoothed) blending coefficient per element of the subcell
    blending limiter (Euler)."""
    d = make_desc(mesh)
    U = np.ascontiguousarray(U, dtype=np.float64)
    E = U.shape[1]
    raw, a = np.zeros(E), np.zeros(E)
    if lib().or_blend_alpha(ctypes.byref(d), _ptr(U), _ptr(raw), _ptr(a)):
        raise ValueError("oracle rejected the mesh descriptor")
    return raw, a


def indicator_energy(mesh, ue):
    """Highest-mode energy fraction of rho p of one element; ue is [node][var]."""
    d = make_desc(mesh)
    ue = np.ascontiguousarray(ue, dtype=np.float64)
    return lib().or_indicator_energy(ctypes.byref(d), _ptr(ue))


def limited_face_flux(mesh, direction, um, up, umi, upi, Fho, a_f, dt, dx, wN, w0):
    """The limited element-face flux of the subcell blending limiter."""
    d = make_desc(mesh)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (um, up, umi, upi, Fho)]
    F = np.zeros(nvars(mesh))
    if lib().or_limited_face_flux(ctypes.byref(d), direction, *[_ptr(a) for a in arrs], float(a_f), float(dt),
                                  float(dx), float(wN), float(w0), _ptr(F)):
        raise ValueError("oracle rejected the arguments")
    return F

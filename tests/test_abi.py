"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/*.h declares; the ctypes descriptor has the C
layout (checked against gcc's own sizeof/offsetof of cr_mesh_desc)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return crkfr.load_library()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(cr_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"cr_init_mesh", "cr_set_state", "cr_step", "cr_get_state"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_2604_02125_gb300 import crkfr
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert crkfr.status_string(s)
    assert "non-physical" in crkfr.status_string(-4)


def test_null_context_is_rejected_without_gpu(lib):
    # argument checks happen before any CUDA call
    assert lib.cr_step(None, 1) == -1
    assert lib.cr_sync(None) == -1
    assert lib.cr_destroy(None) == -1
    assert lib.cr_init_mesh(None, None, 1, None) == -1


def test_descriptor_layout_matches_c(tmp_path):
    from paper_2604_02125_gb300 import crkfr
    src = tmp_path / "lay.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cr.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cr_mesh_desc),'
                   'offsetof(cr_mesh_desc, lo), offsetof(cr_mesh_desc, gamma),'
                   'offsetof(cr_mesh_desc, dt_fixed), offsetof(cr_mesh_desc, prec), offsetof(cr_mesh_desc, scheme),'
                   'offsetof(cr_mesh_desc, ncflux), offsetof(cr_mesh_desc, limiter), offsetof(cr_mesh_desc, alpha_max));'
                   ' return 0;}\n')
    exe = tmp_path / "lay"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    D = crkfr.MeshDesc
    assert got == [ctypes.sizeof(D), D.lo.offset, D.gamma.offset, D.dt_fixed.offset, D.prec.offset, D.scheme.offset,
                   D.ncflux.offset, D.limiter.offset, D.alpha_max.offset]


def _init_status(lib, mesh, prec="fp64"):
    from paper_2604_02125_gb300 import crkfr
    d = crkfr.make_desc(mesh, prec)
    h = ctypes.c_void_p()
    return lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d), 1, None)


def test_invalid_descriptors_rejected_without_gpu(lib):
    """Descriptor validation runs before any CUDA call, so every malformed or
    unsupported descriptor is CR_EINVAL on any machine."""
    from paper_2604_02125_gb300 import crkfr, inputs
    base = inputs.mesh_dict("euler", 2, 3, [4, 4], [0, 0], [1.0, 1.0], 1.4)
    bad = [dict(base, N=0), dict(base, N=6), dict(base, dim=0), dict(base, dim=4), dict(base, cells=[0, 4]),
           dict(base, hi=[0.0, 1.0]), dict(base, gamma=1.0), dict(base, cfl=0.0),
           dict(base, cells=[32768, 32768], N=1),                  # 2^32 nodes: beyond 32-bit node indices
           dict(base, eq="glm_mhd", dim=3, cells=[2, 2, 2]), dict(base, eq="glm_mhd", vol="kep")]
    for m in bad:
        assert _init_status(lib, m) == crkfr.CR_EINVAL, m
    d = crkfr.make_desc(base)
    h = ctypes.c_void_p()
    for field, value in (("surf", 1), ("prec", 2), ("vol", 3), ("dt_fixed", -1.0), ("dt_fixed", float("nan")),
                         ("gamma", float("nan")), ("cfl", float("nan")), ("c_h", float("nan")), ("scheme", 2), ("scheme", -1),
                         ("ncflux", 2), ("ncflux", 1)):           # the stage-wise flux is for GLM-MHD only
        d2 = crkfr.make_desc(base)
        setattr(d2, field, value)
        assert lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d2), 1, None) == crkfr.CR_EINVAL, field
    # ... and for the single-stage scheme only
    mh = inputs.mesh_dict("glm_mhd", 2, 3, [4, 4], [0, 0], [1.0, 1.0], 5.0 / 3.0, c_h=1.0)
    d2 = crkfr.make_desc(dict(mh, ncflux="stages"), scheme="rkfr")
    assert lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d2), 1, None) == crkfr.CR_EINVAL
    # the subcell blending limiter: Euler, single-stage scheme, 0 <= alpha_max <= 1
    for m, sch in ((dict(mh, limiter=True), None), (dict(base, limiter=True), "rkfr"),
                   (dict(base, limiter=True, alpha_max=1.5), None), (dict(base, limiter=True, alpha_max=-0.1), None),
                   (dict(base, limiter=True, alpha_max=float("nan")), None)):
        d2 = crkfr.make_desc(m, scheme=sch)
        assert lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d2), 1, None) == crkfr.CR_EINVAL, m
    d2 = crkfr.make_desc(base)
    d2.limiter = 2
    assert lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d2), 1, None) == crkfr.CR_EINVAL
    assert lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d), 0, None) == crkfr.CR_EINVAL


def test_noalloc_size_limit_without_gpu(lib):
    """cr_step_noalloc rejects a mesh whose scratch exceeds its static array
    (CR_ETOOLARGE) and a malformed descriptor (CR_EINVAL) before any CUDA
    call; the state pointers are not touched on those paths."""
    from paper_2604_02125_gb300 import crkfr, inputs
    big = crkfr.make_desc(inputs.mesh_dict("euler", 2, 3, [128, 128], [0, 0], [1.0, 1.0], 1.4))
    dummy = ctypes.c_void_p(256)
    assert lib.cr_step_noalloc(ctypes.byref(big), dummy, dummy, None, None) == crkfr.CR_ETOOLARGE
    bad = crkfr.make_desc(inputs.mesh_dict("euler", 2, 3, [4, 4], [0, 0], [1.0, 1.0], 1.4))
    bad.degree_N = 9
    assert lib.cr_step_noalloc(ctypes.byref(bad), dummy, dummy, None, None) == crkfr.CR_EINVAL
    # the allocation-free step is the single-stage scheme only
    rk = crkfr.make_desc(inputs.mesh_dict("euler", 2, 3, [4, 4], [0, 0], [1.0, 1.0], 1.4), scheme="rkfr")
    assert lib.cr_step_noalloc(ctypes.byref(rk), dummy, dummy, None, None) == crkfr.CR_EINVAL
    ns = crkfr.make_desc(dict(inputs.mesh_dict("glm_mhd", 2, 3, [4, 4], [0, 0], [1.0, 1.0], 5.0 / 3.0, c_h=1.0),
                              ncflux="stages"))
    assert lib.cr_step_noalloc(ctypes.byref(ns), dummy, dummy, None, None) == crkfr.CR_EINVAL
    lim = crkfr.make_desc(dict(inputs.mesh_dict("euler", 2, 3, [4, 4], [0, 0], [1.0, 1.0], 1.4), limiter=True))
    assert lib.cr_step_noalloc(ctypes.byref(lim), dummy, dummy, None, None) == crkfr.CR_EINVAL
    assert lib.cr_step_noalloc(None, dummy, dummy, None, None) == crkfr.CR_EINVAL


def _valid(d):
    """The descriptor rules of include/cr.h (cr_init_mesh), restated."""
    import math
    if d.eq not in (0, 1) or not (1 <= d.dim <= 3) or not (1 <= d.degree_N <= 5):
        return False
    if d.eq == 1 and (d.dim != 2 or d.vol == 1):
        return False
    if d.vol not in (0, 1, 2) or d.surf != 0 or d.prec not in (0, 1) or d.scheme not in (0, 1):
        return False
    if d.ncflux != 0 and (d.ncflux != 1 or d.eq != 1 or d.scheme != 0):
        return False
    if not (d.gamma > 1.0) or not (d.cfl > 0.0) or not (d.dt_fixed >= 0.0) or not (d.c_h >= 0.0):
        return False
    if d.limiter != 0 and (d.limiter != 1 or d.eq != 0 or d.scheme != 0 or not (0.0 <= d.alpha_max <= 1.0)):
        return False
    nodes = 1
    for k in range(d.dim):
        if d.cells[k] < 1 or not (d.hi[k] > d.lo[k]) or math.isnan(d.hi[k] - d.lo[k]):
            return False
        nodes *= d.cells[k] * (d.degree_N + 1)
    return nodes < 2 ** 31


def test_random_descriptors_rejected_without_gpu(lib):
    """Seeded random descriptors: every one that breaks a documented rule is
    CR_EINVAL before any CUDA call, and none crashes the library.  (Descriptors
    that satisfy every rule are not passed in: on a GPU machine they would
    allocate.)"""
    import numpy as np
    from paper_2604_02125_gb300 import crkfr
    rng = np.random.default_rng(20261203)
    h = ctypes.c_void_p()
    pick = lambda vals: vals[int(rng.integers(len(vals)))]   # noqa: E731
    tried = 0
    for _ in range(3000):
        d = crkfr.MeshDesc()
        d.eq, d.dim, d.degree_N = pick([0, 1, 2, -1]), pick([0, 1, 2, 3, 4]), pick([0, 1, 3, 5, 6])
        for k in range(3):
            d.cells[k] = pick([-1, 0, 1, 7, 65536])
            d.lo[k] = pick([0.0, -1.0, float("nan")])
            d.hi[k] = pick([1.0, 0.0, -2.0, float("inf")])
        d.gamma, d.cfl = pick([1.4, 1.0, 0.5, float("nan")]), pick([0.1, 0.0, -1.0, float("nan")])
        d.c_h, d.dt_fixed = pick([0.0, 1.0, -1.0, float("nan")]), pick([0.0, 1e-3, -1.0, float("nan")])
        d.vol, d.surf, d.prec = pick([0, 1, 2, 3]), pick([0, 1]), pick([0, 1, 2])
        d.scheme, d.ncflux = pick([0, 1, 2]), pick([0, 1, 2])
        d.limiter, d.alpha_max = pick([0, 0, 1, 2]), pick([0.0, 0.5, 1.5, float("nan")])
        if _valid(d):
            continue
        tried += 1
        assert lib.cr_init_mesh(ctypes.byref(h), ctypes.byref(d), 1, None) == crkfr.CR_EINVAL, (
            [getattr(d, f) for f, _ in d._fields_ if f not in ("cells", "lo", "hi")])
        assert not h.value
    assert tried > 2500


def test_workspace_bytes_without_gpu(lib):
    """cr_workspace_bytes follows the documented buffer list (no CUDA call):
    the state, R-bar, face records, step record and totals of the plain
    step; a second state buffer, per-element coefficients and flags and the
    list of touched elements with the limiter;
    the stage state and s - 1 stage increments with the multi-stage scheme.
    cr_init_mesh_ws rejects a NULL, misaligned or too small workspace before
    any CUDA call."""
    from paper_2604_02125_gb300 import crkfr, inputs
    al = lambda b: (b + 255) // 256 * 256   # noqa: E731
    mesh = inputs.mesh_dict("euler", 2, 3, [10, 7], [0, 0], [1.0, 1.0], 1.4)
    E, NP, M, NF = 70, 16, 4, 4
    nodes = E * NP
    for prec, R in (("fp64", 8), ("fp32", 4)):
        # the step record: three CFL slots of 32 64-bit words, three epochs and
        # a pad word, dt, t, the wave-speed maximum, the step count, status, pad
        step_record = 3 * 32 * 8 + 4 * 4 + 3 * 8 + 8 + 2 * 4
        plain = (al(8 * M * nodes) + al(R * M * nodes) + al(R * 2 * 2 * (2 * M + 1) * NF * E) + al(step_record)
                 + al(8 * ((nodes + 255) // 256) * (M + 2)))
        assert crkfr.workspace_bytes(mesh, prec) == plain
        lim = plain + al(8 * M * nodes) + al(8 * E) + al(8 * E) + al(E) + al(4 * E) + al(4)
        assert crkfr.workspace_bytes(dict(mesh, limiter=True), prec) == lim
        rk = plain + al(8 * M * nodes) + al(R * 3 * M * nodes)
        assert crkfr.workspace_bytes(mesh, prec, scheme="rkfr") == rk
    n = ctypes.c_size_t()
    bad = crkfr.make_desc(dict(mesh, N=7))
    assert lib.cr_workspace_bytes(ctypes.byref(bad), ctypes.byref(n)) == crkfr.CR_EINVAL
    d = crkfr.make_desc(mesh)
    h = ctypes.c_void_p()
    need = crkfr.workspace_bytes(mesh)
    assert lib.cr_init_mesh_ws(ctypes.byref(h), ctypes.byref(d), None, need, None) == crkfr.CR_EINVAL
    assert lib.cr_init_mesh_ws(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(4096 + 8), need, None) == \
        crkfr.CR_EINVAL
    assert lib.cr_init_mesh_ws(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(4096), need - 1, None) == \
        crkfr.CR_EINVAL
    assert not h.value

"""Every variant cr_init_mesh accepts, against the FP64 oracle, one step each.

The descriptor space of include/cr.h: Euler in 1, 2 and 3 dimensions and
GLM-MHD in 2, degrees N = 1..5, both precisions, every volume flux the system
takes (Euler: EC, KEP, central; GLM-MHD: EC, central), both schemes (the
cRKFR step of Sec. 2.3, eqs. crkfr.inner and crkfr.non.cons.final, and the
multi-stage RKFR step of eq. rkfr.non.cons), and for GLM-MHD with the cRKFR
step both non-conservative numerical fluxes (Sec. 2.3 and eq.
bad.numflux.non.cons).  Each case takes one step from a smooth seeded state
on a small mesh with a ragged last tile (the lane kernels take 32 elements per
CTA, the tile kernels a few) and is compared node by node:

* dt equal to the oracle's CFL dt within 1e-14 (FP64) or 1e-6 (FP32 wave
  speeds, reading R15);
* the state within 1e-12 (FP64) / 1e-5 (FP32) relative L2 and per-variable
  nodal maximum;
* the increment u^{n+1} - u^n within 1e-10 (FP64) / 1e-3 (FP32) on the same
  two measures: a one-step state comparison alone dilutes an error of the
  increment by ||u|| / ||du||.  The FP32 bound comes from the FP32 rounding of
  the stage states and pair fluxes, amplified by the differentiation matrix
  (|D| up to N(N+1)/(4 dx)).
"""
import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs
from parity_util import check_close, check_increment

pytestmark = pytest.mark.gpu

STATE_TOL = {"fp64": 1e-12, "fp32": 1e-5}
INC_TOL = {"fp64": 1e-10, "fp32": 1e-3}
DT_TOL = {"fp64": 1e-14, "fp32": 1e-6}

# small meshes whose element count leaves a ragged last tile of 32 (lane form)
# and spans several CTAs of the tile form
CELLS = {1: [37], 2: [7, 5], 3: [3, 4, 3]}


def _variants():
    out = []
    for scheme in ("crkfr", "rkfr"):
        for prec in ("fp64", "fp32"):
            for N in range(1, 6):
                for dim in (1, 2, 3):
                    for vol in ("ec", "kep", "central"):
                        out.append(("euler", dim, N, prec, vol, scheme, "reduced"))
                for vol in ("ec", "central"):
                    out.append(("glm_mhd", 2, N, prec, vol, scheme, "reduced"))
                    if scheme == "crkfr":
                        out.append(("glm_mhd", 2, N, prec, vol, scheme, "stages"))
    return out


VARIANTS = _variants()


def _id(v):
    eq, dim, N, prec, vol, scheme, nc = v
    return "%s%dd-N%d-%s-%s-%s%s" % ("euler" if eq == "euler" else "mhd", dim, N, prec, vol, scheme,
                                     "-ncstages" if nc == "stages" else "")


@pytest.fixture(scope="module")
def cr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return crkfr


def _state(eq, dim, N, vol, seed):
    cells = CELLS[dim]
    hi = [1.0, 1.3, 0.9][:dim]
    mesh = inputs.mesh_dict(eq, dim, N, cells, [0.0] * dim, hi, 1.4 if eq == "euler" else 5.0 / 3.0, vol=vol)
    U = inputs.smooth_random_field(mesh, seed=seed, amp=0.2)
    if eq == "glm_mhd":
        mesh["c_h"] = 2.0
    return mesh, U


def test_matrix_covers_every_accepted_variant(cr):
    """The matrix spans the descriptor space: every combination outside it is
    rejected by cr_init_mesh with CR_EINVAL."""
    import itertools
    covered = set(VARIANTS)
    rejected = 0
    for eq, dim, vol, scheme, nc, N, prec in itertools.product(
            ("euler", "glm_mhd"), (1, 2, 3), ("ec", "kep", "central"), ("crkfr", "rkfr"), ("reduced", "stages"),
            range(1, 6), ("fp64", "fp32")):
        if (eq, dim, N, prec, vol, scheme, nc) in covered:
            continue
        mesh = dict(inputs.mesh_dict(eq, dim, N, CELLS[dim], [0.0] * dim, [1.0] * dim, 1.4, vol=vol),
                    scheme=scheme, ncflux=nc)
        with pytest.raises(cr.CrError) as ei:
            cr.Solver(mesh, prec=prec)
        assert ei.value.status == cr.CR_EINVAL, (eq, dim, N, prec, vol, scheme, nc)
        rejected += 1
    assert rejected + len(covered) == 2 * 3 * 3 * 2 * 2 * 5 * 2


@pytest.mark.parametrize("var", VARIANTS, ids=_id)
def test_variant_one_step(cr, orc, var):
    eq, dim, N, prec, vol, scheme, nc = var
    seed = 1000 + 7 * N + 31 * dim + (0 if eq == "euler" else 500)
    mesh, U = _state(eq, dim, N, vol, seed)
    mesh = dict(mesh, scheme=scheme, ncflux=nc)
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(1)
        G = s.get_state()
        info = s.info()
    assert info["status"] == 0 and info["steps"] == 1
    dt = orc.cfl_dt(mesh, U)
    assert abs(info["dt"] - dt) <= DT_TOL[prec] * dt, (info["dt"], dt)
    step = orc.rkfr_step if scheme == "rkfr" else orc.step
    O = step(mesh, U, info["dt"])
    what = _id(var)
    check_close(G, O, STATE_TOL[prec], what)
    check_increment(G, O, U, INC_TOL[prec], what)

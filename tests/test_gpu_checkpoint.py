"""Checkpoint and resume through the C ABI: cr_get_state after k steps and
cr_set_state into a fresh context, then the remaining steps, give the same
state as the uninterrupted run, bit for bit.

The dt of the first resumed step comes from the CFL reduction of the set
state (k_lambda), which evaluates the wave speeds exactly as the face / update
kernel does for the state it produces, so every dt is the same too.  Rule for
time: cr_set_state starts t and the step count at 0 (include/cr.h), so the
resumed run's t is the time since the checkpoint; the caller adds the saved t.
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


def _case(name):
    if name == "shear2d":
        return inputs.shear_layer_2d(cells=(33, 20), N=3)
    if name == "mhd2d":
        return inputs.mhd_vortex_2d(cells=(9, 7), N=4)
    if name == "tgv3d":
        return inputs.tgv_3d(cells=(5, 4, 3), N=2, mach=0.3)
    if name == "limited":
        mesh = dict(inputs.mesh_dict("euler", 2, 3, [21, 6], [0.0, 0.0], [1.0, 1.0], 1.4), limiter=True,
                    alpha_max=0.5)
        X = inputs.node_coords(mesh)
        slab = 1.0 + (np.tanh(60.0 * (X[0] - 0.3)) - np.tanh(60.0 * (X[0] - 0.65)))
        one = np.ones_like(X[0])
        return mesh, inputs.euler_cons(1.4, slab, [0.3 * one, 0.1 * one], slab)
    raise KeyError(name)


@pytest.mark.parametrize("scheme", ["crkfr", "rkfr"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["shear2d", "mhd2d", "tgv3d", "limited"])
def test_resume_equals_uninterrupted(cr, name, prec, scheme):
    if name == "limited" and scheme == "rkfr":
        pytest.skip("the limiter is for the single-stage scheme")
    mesh, U = _case(name)
    with cr.Solver(mesh, prec=prec, scheme=scheme) as a:
        a.set_state(U)
        a.step(37)                     # odd: the resumed run starts from the other step parity
        ta = a.info()["t"]
        ckpt = a.get_state()
        a.step(63)
        full = a.get_state()
        ia = a.info()
    with cr.Solver(mesh, prec=prec, scheme=scheme) as b:
        b.set_state(ckpt)
        b.step(63)
        resumed = b.get_state()
        ib = b.info()
    assert np.array_equal(resumed, full)
    assert ib["steps"] == 63 and ia["steps"] == 100
    assert ib["dt"] == ia["dt"]
    assert abs((ta + ib["t"]) - ia["t"]) <= 1e-14 * ia["t"]

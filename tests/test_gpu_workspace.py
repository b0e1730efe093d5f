"""cr_init_mesh_ws: a context whose device buffers are carved out of a
caller's workspace (here a tensor from PyTorch's caching allocator) steps
exactly like a context that allocates its own, for the plain step, the
limiter and the multi-stage scheme, and does not allocate its buffers itself
(the device's free memory drops by far less than the workspace size); a
workspace on the host or too small is rejected."""
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


def _fronts():
    mesh = dict(inputs.mesh_dict("euler", 2, 3, [40, 24], [0.0, 0.0], [1.0, 1.0], 1.4), limiter=True, alpha_max=0.5)
    X = inputs.node_coords(mesh)
    slab = 1.0 + (np.tanh(60.0 * (X[0] - 0.3)) - np.tanh(60.0 * (X[0] - 0.65)))
    one = np.ones_like(X[0])
    return mesh, inputs.euler_cons(1.4, slab, [0.3 * one, 0.1 * one], slab)


@pytest.mark.parametrize("case,prec,scheme", [("shear", "fp32", None), ("shear", "fp64", None), ("shear", "fp32", "rkfr"),
                                              ("limited", "fp32", None), ("mhd", "fp64", None)])
def test_workspace_context_steps_like_owned(cr, case, prec, scheme):
    import torch
    if case == "shear":
        mesh, U = inputs.shear_layer_2d(cells=(96, 80), N=3)
    elif case == "mhd":
        mesh, U = inputs.mhd_vortex_2d(cells=(24, 20), N=4)
    else:
        mesh, U = _fronts()
    need = cr.workspace_bytes(mesh, prec, scheme=scheme)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with cr.Solver(mesh, prec=prec, scheme=scheme, workspace=ws) as a, cr.Solver(mesh, prec=prec, scheme=scheme) as b:
        a.set_state(U)
        b.set_state(U)
        a.step(21)
        b.step(21)
        assert np.array_equal(a.get_state(), b.get_state())
        ia, ib = a.info(totals=True), b.info(totals=True)
        assert ia["t"] == ib["t"] and ia["steps"] == 21 and np.array_equal(ia["totals"], ib["totals"])


def test_workspace_context_allocates_no_buffers(cr):
    """A 1024 x 512, N = 3, FP64 mesh needs about 0.5 GB of buffers; creating
    its context on a workspace lowers the device's free memory by far less
    (the library still creates its CUDA graphs, streams and events)."""
    import torch
    mesh, _ = inputs.shear_layer_2d(cells=(1024, 512), N=3)
    need = cr.workspace_bytes(mesh, "fp64")
    assert need > (400 << 20)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = cr.Solver(mesh, prec="fp64", workspace=ws)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    s.close()
    assert free0 - free1 < (64 << 20), (free0 - free1, need)


def test_workspace_rejected(cr):
    import torch
    mesh, U = inputs.shear_layer_2d(cells=(16, 16), N=3)
    need = cr.workspace_bytes(mesh, "fp32")
    for ws in (torch.empty(need, dtype=torch.uint8), torch.empty(need - 256, dtype=torch.uint8, device="cuda")):
        with pytest.raises((cr.CrError, ValueError)):
            cr.Solver(mesh, prec="fp32", workspace=ws)

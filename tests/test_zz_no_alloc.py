"""cr_step_noalloc: a time step that allocates no device memory.

It serves callers that cannot allocate while they advance a solve (their
memory pool already holds the device, or a cudaMalloc/cudaFree would stall
other streams by synchronising the device).  Its scratch is one static
per-device array inside the library, shared by every call.  This file is
collected last so that a failure here comes after every other test has run.

Checked through the C ABI: two calls in a row agree with the regular
cr_set_state / cr_step / cr_get_state path to the FP64 parity tolerance
(1e-12 relative L2) and with the FP64 oracle (1e-12 FP64, 1e-5 FP32), the dt
written to the device matches, in-place calls work, no device memory is
allocated by a call (torch's allocator and cudaMemGetInfo unchanged), and a
mesh beyond the static capacity is rejected with CR_ETOOLARGE.
"""
import numpy as np
import pytest

from paper_2604_02125_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_02125_gb300 import build, crkfr
    build.build()
    return torch, crkfr


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,case", [("fp64", "shear"), ("fp64", "mhd"), ("fp32", "shear")])
def test_two_calls_match_regular_path(env, orc, prec, case):
    torch, cr = env
    if case == "shear":
        mesh, U = inputs.shear_layer_2d(cells=(13, 9), N=3)
    else:
        mesh, U = inputs.mhd_vortex_2d(cells=(6, 7), N=4)
    # regular path: context-owned buffers
    with cr.Solver(mesh, prec=prec) as s:
        s.set_state(U)
        s.step(1)
        ref1 = s.get_state()
        dt1 = s.info()["dt"]
        s.step(1)
        ref2 = s.get_state()
        dt2 = s.info()["dt"]
    u0 = torch.from_numpy(U).cuda()
    u1 = torch.empty_like(u0)
    u2 = torch.empty_like(u0)
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    cr.step_noalloc(mesh, u0, u1, dt, prec=prec)     # first call: looks up the scratch address
    torch.cuda.synchronize()
    assert rel(u1.cpu().numpy(), ref1) <= 1e-12
    assert abs(dt.item() - dt1) <= 1e-14 * dt1
    # the oracle, from the same state with the dt the call used
    tol = 1e-12 if prec == "fp64" else 1e-5
    o1 = orc.step(mesh, U, dt.item())
    assert rel(u1.cpu().numpy(), o1) <= tol
    # a warmed-up call allocates nothing: neither torch's pool nor the device
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    cr.step_noalloc(mesh, u1, u2, dt, prec=prec)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0, (free0, free1)
    assert rel(u2.cpu().numpy(), ref2) <= 1e-12
    assert abs(dt.item() - dt2) <= 1e-14 * dt2
    o2 = orc.step(mesh, u1.cpu().numpy(), dt.item())
    assert rel(u2.cpu().numpy(), o2) <= tol
    # in place: u_out == u_in
    cr.step_noalloc(mesh, u0, u0, None, prec=prec)
    torch.cuda.synchronize()
    assert rel(u0.cpu().numpy(), ref1) <= 1e-12


def test_capacity_limit(env):
    torch, cr = env
    mesh, _ = inputs.shear_layer_2d(cells=(256, 256), N=3)
    u = torch.zeros(4 * 256 * 256 * 16, dtype=torch.float64, device="cuda")
    with pytest.raises(cr.CrError) as ei:
        cr.step_noalloc(mesh, u, u)
    assert ei.value.status == cr.CR_ETOOLARGE


def test_rejects_mismatched_tensors(env):
    """The binding checks what the C entry point cannot: size, type, layout
    and device of the caller's tensors (a raw pointer carries none of them)."""
    torch, cr = env
    mesh, U = inputs.shear_layer_2d(cells=(5, 4), N=3)
    u = torch.from_numpy(U).cuda()
    bad = [u[..., :-1].contiguous(), u.float(), u.transpose(1, 2), u.cpu()]
    for b in bad:
        with pytest.raises(ValueError):
            cr.step_noalloc(mesh, b, u)
        with pytest.raises(ValueError):
            cr.step_noalloc(mesh, u, b)
    for d in (torch.zeros(1, dtype=torch.float32, device="cuda"), torch.zeros(0, dtype=torch.float64, device="cuda")):
        with pytest.raises(ValueError):
            cr.step_noalloc(mesh, u, u, d)

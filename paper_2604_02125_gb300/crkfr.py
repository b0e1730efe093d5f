"""Thin Python binding of the C ABI in include/cr.h (argument marshalling only).

Every step of the cRKFR path runs in the CUDA library libcrkfr.so; this module
only builds descriptors and passes pointers.  PyTorch is used, when given, for
device memory (tensor data pointers) and streams.  There is no CPU fallback:
if the compiled library is missing, :func:`load_library` raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcrkfr.so")

CR_OK, CR_EINVAL, CR_ENOMEM, CR_ECUDA, CR_ENONPHYSICAL, CR_ETIMEOUT, CR_ENODEV, CR_ETOOLARGE = \
    0, -1, -2, -3, -4, -5, -6, -7
EQ = {"euler": 0, "glm_mhd": 1}
VOL = {"ec": 0, "kep": 1, "central": 2}
SURF = {"rusanov": 0}
PREC = {"fp64": 0, "fp32": 1}
SCHEME = {"crkfr": 0, "rkfr": 1}
NCFLUX = {"reduced": 0, "stages": 1}


class CrError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_string(status), status))


class MeshDesc(ctypes.Structure):
    _fields_ = [("eq", ctypes.c_int), ("dim", ctypes.c_int), ("degree_N", ctypes.c_int),
                ("cells", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("c_h", ctypes.c_double),
                ("dt_fixed", ctypes.c_double), ("vol", ctypes.c_int), ("surf", ctypes.c_int),
                ("prec", ctypes.c_int), ("scheme", ctypes.c_int), ("ncflux", ctypes.c_int),
                ("limiter", ctypes.c_int), ("alpha_max", ctypes.c_double)]


_lib = None

EXPORTS = ("cr_init_mesh", "cr_state_size", "cr_set_state", "cr_step", "cr_sync", "cr_get_state",
           "cr_get_info", "cr_time_kernels", "cr_destroy", "cr_status_string", "cr_step_noalloc",
           "cr_probe_peak", "cr_tuning_info", "cr_check_conversions", "cr_set_state_async", "cr_get_state_async",
           "cr_workspace_bytes", "cr_init_mesh_ws", "cr_get_blend_alpha")


def load_library(path=None):
    """Load libcrkfr.so (built by paper_2604_02125_gb300.build); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("the CUDA library %s is not built; run paper_2604_02125_gb300.build.build()" % p)
    lib = ctypes.CDLL(p)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.cr_init_mesh.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(MeshDesc), ip, vp]
    lib.cr_state_size.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)]
    lib.cr_set_state.argtypes = [vp, ip, vp, ip]
    lib.cr_step.argtypes = [vp, ip]
    lib.cr_sync.argtypes = [vp]
    lib.cr_get_state.argtypes = [vp, ip, vp, ip]
    lib.cr_set_state_async.argtypes = [vp, ip, vp, ip]
    lib.cr_get_state_async.argtypes = [vp, ip, vp, ip]
    lib.cr_get_info.argtypes = [vp, ip, dp, dp, ctypes.POINTER(ctypes.c_longlong), dp]
    lib.cr_time_kernels.argtypes = [vp, ip, vp, ctypes.c_size_t, dp]
    lib.cr_destroy.argtypes = [vp]
    lib.cr_step_noalloc.argtypes = [ctypes.POINTER(MeshDesc), vp, vp, vp, vp]
    lib.cr_probe_peak.argtypes = [ip, dp]
    lib.cr_tuning_info.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.cr_check_conversions.argtypes = [ctypes.c_longlong, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)]
    lib.cr_workspace_bytes.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(ctypes.c_size_t)]
    lib.cr_init_mesh_ws.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(MeshDesc), vp, ctypes.c_size_t, vp]
    lib.cr_get_blend_alpha.argtypes = [vp, dp, ip]
    lib.cr_status_string.argtypes = [ip]
    lib.cr_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "cr_status_string":
            getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def status_string(s):
    try:
        return load_library().cr_status_string(int(s)).decode()
    except RuntimeError:
        return "status %d" % s


def make_desc(mesh, prec="fp64", dt_fixed=0.0, scheme=None):
    """Descriptor of a mesh dict; scheme ('crkfr' or 'rkfr', the multi-stage
    scheme) defaults to the dict's 'scheme' key, else 'crkfr'; the dict's
    'ncflux' key ('reduced' or 'stages', GLM-MHD) selects the non-conservative
    numerical flux; 'limiter' (bool) and 'alpha_max' the subcell blending
    limiter (Euler)."""
    d = MeshDesc()
    d.eq = EQ[mesh.get("eq", "euler")]
    d.dim = mesh["dim"]
    d.degree_N = mesh["N"]
    cells = list(mesh["cells"]) + [1] * 3
    lo = list(mesh["lo"]) + [0.0] * 3
    hi = list(mesh["hi"]) + [1.0] * 3
    for k in range(3):
        d.cells[k], d.lo[k], d.hi[k] = int(cells[k]), float(lo[k]), float(hi[k])
    d.gamma = mesh.get("gamma", 1.4)
    d.cfl = mesh.get("cfl", 0.1)
    d.c_h = mesh.get("c_h", 0.0)
    d.dt_fixed = float(dt_fixed)
    d.vol = VOL[mesh.get("vol", "ec")]
    d.surf = SURF[mesh.get("surf", "rusanov")]
    d.prec = PREC[prec]
    d.scheme = SCHEME[scheme or mesh.get("scheme", "crkfr")]
    d.ncflux = NCFLUX[mesh.get("ncflux", "reduced")]
    d.limiter = 1 if mesh.get("limiter") else 0
    d.alpha_max = float(mesh.get("alpha_max", 1.0))
    return d


def _check(rc, what):
    if rc != CR_OK:
        raise CrError(rc, what)


def _ptr_and_location(a):
    """(pointer, on_device) of a C-contiguous float64 numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("state arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    import torch  # noqa: F401  (only for tensors)
    if a.dtype != __import__("torch").float64 or not a.is_contiguous():
        raise ValueError("state tensors must be contiguous float64")
    return a.data_ptr(), 1 if a.is_cuda else 0


class Solver:
    """One mesh (mesh dict) or a batch of meshes (list of mesh dicts).

    prec: 'fp64' (plain path) or 'fp32' (FP32 pair fluxes, FP64 update).
    scheme: 'crkfr' (the single-stage method) or 'rkfr' (the multi-stage
    scheme it is derived from, one face exchange per RK stage; one mesh only);
    default: each mesh dict's 'scheme' key, else 'crkfr'.
    stream: a cudaStream_t handle (int) or a torch.cuda.Stream; default: the
    current torch stream if torch has initialised CUDA, else the legacy stream.
    workspace: a CUDA uint8 tensor of at least workspace_bytes(mesh, prec)
    bytes (one mesh only): every device buffer of the context is carved out of
    it (cr_init_mesh_ws); the solver keeps a reference to it.
    """

    def __init__(self, mesh, prec="fp64", dt_fixed=0.0, stream=None, scheme=None, workspace=None):
        self.lib = load_library()
        meshes = mesh if isinstance(mesh, (list, tuple)) else [mesh]
        self.meshes = list(meshes)
        arr = (MeshDesc * len(meshes))(*[make_desc(m, prec, dt_fixed, scheme) for m in meshes])
        self._descs = arr
        if stream is None:
            stream = _current_torch_stream()
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream or 0)
        h = ctypes.c_void_p()
        if workspace is None:
            _check(self.lib.cr_init_mesh(ctypes.byref(h), arr, len(meshes), ctypes.c_void_p(self.stream)),
                   "cr_init_mesh")
        else:
            if len(meshes) != 1 or not getattr(workspace, "is_cuda", False) or not workspace.is_contiguous():
                raise ValueError("workspace: one mesh and a contiguous CUDA tensor")
            self._workspace = workspace
            nbytes = workspace.numel() * workspace.element_size()
            _check(self.lib.cr_init_mesh_ws(ctypes.byref(h), arr, ctypes.c_void_p(workspace.data_ptr()), nbytes,
                                            ctypes.c_void_p(self.stream)), "cr_init_mesh_ws")
        self.h = h

    def state_size(self, solve=0):
        nv = ctypes.c_int()
        nn = ctypes.c_longlong()
        _check(self.lib.cr_state_size(self.h, solve, ctypes.byref(nv), ctypes.byref(nn)), "cr_state_size")
        return nv.value, nn.value

    def set_state(self, u, solve=0, sync=True):
        """Copy a state in.  sync=False: enqueue only (cr_set_state_async);
        u must stay alive and unchanged until the next sync."""
        ptr, dev = _ptr_and_location(u)
        M, nodes = self.state_size(solve)
        count = u.size if isinstance(u, np.ndarray) else u.numel()
        if count != M * nodes:
            raise ValueError("state has %d values, expected %d" % (count, M * nodes))
        fn = self.lib.cr_set_state if sync else self.lib.cr_set_state_async
        _check(fn(self.h, solve, ctypes.c_void_p(ptr), dev), "cr_set_state" if sync else "cr_set_state_async")

    def step(self, nsteps=1):
        _check(self.lib.cr_step(self.h, int(nsteps)), "cr_step")

    def sync(self):
        _check(self.lib.cr_sync(self.h), "cr_sync")

    def get_state(self, out=None, solve=0, check=True, sync=True):
        """Copy the state out.  sync=False: enqueue only (cr_get_state_async;
        `out` is required and holds the state after the next sync)."""
        M, nodes = self.state_size(solve)
        mesh = self.meshes[solve]
        if out is None:
            if not sync:
                raise ValueError("get_state(sync=False) needs an output buffer")
            from . import inputs
            out = np.empty((M, inputs.num_elems(mesh), inputs.nodes_per_elem(mesh)))
        ptr, dev = _ptr_and_location(out)
        if not sync:
            _check(self.lib.cr_get_state_async(self.h, solve, ctypes.c_void_p(ptr), dev), "cr_get_state_async")
            return out
        rc = self.lib.cr_get_state(self.h, solve, ctypes.c_void_p(ptr), dev)
        if check:
            _check(rc, "cr_get_state")
        return out

    def info(self, solve=0, totals=False):
        t, dt = ctypes.c_double(), ctypes.c_double()
        steps = ctypes.c_longlong()
        M, _ = self.state_size(solve)
        tot = np.zeros(M + 2) if totals else None
        rc = self.lib.cr_get_info(self.h, solve, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(steps),
                                  tot.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if totals else None)
        out = {"t": t.value, "dt": dt.value, "steps": steps.value, "status": rc}
        if totals:
            out["totals"] = tot
        return out

    def time_kernels(self, nsteps, flush=None):
        """Mean per-launch durations (ms) of the volume and face/update kernels
        over nsteps further steps, each kernel between CUDA events on the
        solver's stream; `flush` (a torch CUDA tensor) is overwritten before
        every step to evict the L2."""
        ms = (ctypes.c_double * 2)()
        fp = ctypes.c_void_p(flush.data_ptr()) if flush is not None else None
        nb = flush.numel() * flush.element_size() if flush is not None else 0
        _check(self.lib.cr_time_kernels(self.h, int(nsteps), fp, nb, ms), "cr_time_kernels")
        return ms[0], ms[1]

    def blend_alpha(self):
        """Smoothed blending coefficients of the elements that the last step
        used (subcell blending limiter; cr_get_blend_alpha)."""
        from . import inputs
        out = np.zeros(inputs.num_elems(self.meshes[0]))
        _check(self.lib.cr_get_blend_alpha(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0),
               "cr_get_blend_alpha")
        return out

    def tuning_info(self):
        """The kernel configuration chosen for this context (JSON)."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        _check(self.lib.cr_tuning_info(self.h, buf, len(buf)), "cr_tuning_info")
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.cr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def step_noalloc(mesh, u_in, u_out, dt_out=None, prec="fp64", dt_fixed=0.0, stream=None):
    """One step through cr_step_noalloc: no device memory is allocated; the
    scratch is the library's static per-device array.  u_in, u_out (and dt_out,
    a 1-element float64 tensor) are CUDA tensors; u_out may be u_in.  Returns
    the C status (raises CrError on failure)."""
    import torch
    lib = load_library()
    d = make_desc(mesh, prec, dt_fixed)
    if stream is None:
        stream = _current_torch_stream()
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    # the C entry point takes raw device pointers and trusts their sizes: check
    # type, layout, size and device here, before any kernel can touch them
    from . import inputs
    need = inputs.nvars(mesh) * inputs.num_elems(mesh) * inputs.nodes_per_elem(mesh)
    dev = torch.cuda.current_device()
    for name, t in (("u_in", u_in), ("u_out", u_out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError("cr_step_noalloc: %s must be a CUDA tensor" % name)
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError("cr_step_noalloc: %s must be contiguous float64" % name)
        if t.numel() != need:
            raise ValueError("cr_step_noalloc: %s has %d values, the mesh needs %d" % (name, t.numel(), need))
        if t.device.index != dev:
            raise ValueError("cr_step_noalloc: %s is on cuda:%s, the current device is cuda:%d"
                             % (name, t.device.index, dev))
    if dt_out is not None:
        if (not isinstance(dt_out, torch.Tensor) or not dt_out.is_cuda or dt_out.dtype != torch.float64
                or dt_out.numel() < 1 or dt_out.device.index != dev):
            raise ValueError("cr_step_noalloc: dt_out must be a float64 CUDA tensor of at least one value "
                             "on the current device")
    rc = lib.cr_step_noalloc(ctypes.byref(d), ctypes.c_void_p(u_in.data_ptr()), ctypes.c_void_p(u_out.data_ptr()),
                             ctypes.c_void_p(dt_out.data_ptr()) if dt_out is not None else None,
                             ctypes.c_void_p(int(stream or 0)))
    _check(rc, "cr_step_noalloc")
    return rc


def workspace_bytes(mesh, prec="fp64", scheme=None):
    """Device bytes a single-solve context of this mesh needs (cr_workspace_bytes)."""
    lib = load_library()
    d = make_desc(mesh, prec, 0.0, scheme)
    n = ctypes.c_size_t(0)
    _check(lib.cr_workspace_bytes(ctypes.byref(d), ctypes.byref(n)), "cr_workspace_bytes")
    return n.value


PROBES = {"ffma": 0, "dfma": 1, "mufu_rcp": 2, "cvt_f64_f32": 3, "int_alu": 4, "copy_bytes": 5,
          "h2d_bytes": 6, "d2h_bytes": 7, "duplex_bytes_per_direction": 8}


def probe_peaks(kinds=None):
    """Measured unit throughputs of the current device (lane-ops/s; copy: bytes/s)."""
    lib = load_library()
    out = {}
    for name in (kinds or PROBES):
        r = ctypes.c_double()
        _check(lib.cr_probe_peak(PROBES[name], ctypes.byref(r)), "cr_probe_peak")
        out[name] = r.value
    return out


def _current_torch_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def check_conversions(n=1 << 24, seed=2604021255):
    """Mismatches of the FP32 form's integer float<->double conversions against
    the hardware conversions over n seeded bit patterns (0 expected)."""
    lib = load_library()
    r = ctypes.c_longlong(-1)
    _check(lib.cr_check_conversions(int(n), int(seed), ctypes.byref(r)), "cr_check_conversions")
    return int(r.value)

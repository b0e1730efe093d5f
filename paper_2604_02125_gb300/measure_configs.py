"""Per-workload throughput of the cRKFR step on one GPU.

  python -m paper_2604_02125_gb300.measure_configs [--steps K] [--budget-steps S] [--only NAME ...]

For each workload (1D density wave, 2D shear layer, 2D GLM-MHD vortex, 3D
Taylor-Green vortex, 512 batched 2D solves) and each form (FP64, FP32 pair
fluxes) prints one JSON line: DOF-updates/s over K steps timed with CUDA
events on the solver's stream (256 MiB L2 flush between steps), the mean
volume and face/update kernel times, the FP32-vs-FP64 relative L2 after 100
steps from the same state, the same timings of the multi-stage RKFR scheme
(one face exchange per RK stage) and its cost against the single-stage
step, and for the Taylor-Green vortex the FP64 kinetic
energy and entropy budgets over S steps; and the shear layer over its full
run length (--long-steps, 2000): FP32 against FP64, conservation, budgets.

Every form carries its roofline: the volume kernel's counted flops
(paper_2604_02125_gb300.work) per launch time against the FP32 peak (152 SMs
x 128 lanes x 2 x max SM clock) or the FP64 peak (twice the FP64 FMA rate
measured by cr_probe_peak), and the face / update kernel's algorithmic bytes
per launch time against the measured HBM copy bandwidth.  The subcell
blending limiter runs on the shear layer with the paper's Kelvin-Helmholtz
setting and on a mesh where it acts; the batched workload is also advanced
one solve at a time through 512 single-solve contexts (batched/sequential).

The headline measurement is bench.py (whose --cpu-baseline-configs option
times the FP64 oracle on reduced meshes of the same workloads); this script
fills the per-workload GPU table.
"""
import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2604_02125_gb300 import build, crkfr, inputs, work  # noqa: E402

WORKLOADS = {
    "wave1d_64_N3": (lambda: inputs.density_wave_1d(cells=64, N=3), "1D Euler density wave, 64 elements, N=3"),
    "shear2d_256_N3": (lambda: inputs.shear_layer_2d(cells=(256, 256), N=3),
                       "2D Euler shear layer, 256x256 quads, N=3, EC flux"),
    "shear2d_256_N3_kep": (lambda: inputs.shear_layer_2d(cells=(256, 256), N=3, vol="kep"),
                           "2D Euler shear layer, 256x256 quads, N=3, KEP flux"),
    "shear2d_256_N3_central": (lambda: inputs.shear_layer_2d(cells=(256, 256), N=3, vol="central"),
                               "2D Euler shear layer, 256x256 quads, N=3, central two-point flux (collocation FR)"),
    "mhd2d_128_N4": (lambda: inputs.mhd_vortex_2d(cells=(128, 128), N=4),
                     "2D GLM-MHD vortex, 128x128 quads, N=4, EC flux"),
    "mhd2d_128_N4_ncstages": (lambda: _stagewise(*inputs.mhd_vortex_2d(cells=(128, 128), N=4)),
                              "2D GLM-MHD vortex, 128x128 quads, N=4, EC flux, stage-wise non-conservative flux "
                              "(every stage's face traces exchanged)"),
    "tgv3d_64_N3": (lambda: inputs.tgv_3d(cells=(64, 64, 64), N=3), "3D Euler Taylor-Green vortex, 64^3 hexes, N=3"),
    "shear2d_256_N3_kep_limiter": (lambda: _limited(*inputs.shear_layer_2d(cells=(256, 256), N=3, vol="kep"), 0.008),
                                   "2D Euler shear layer, 256x256 quads, N=3, KEP flux, subcell blending limiter "
                                   "alpha_max = 0.008 (the paper's Kelvin-Helmholtz setting)"),
    "fronts2d_256_N3_limiter": (lambda: _fronts(), "2D Euler, 256x256 quads, N=3, EC flux, steep density / pressure "
                                                   "slab, subcell blending limiter alpha_max = 0.7 (acts on ~4% of "
                                                   "the elements)"),
}


def _limited(mesh, U, alpha_max):
    return dict(mesh, limiter=True, alpha_max=alpha_max), U


def _fronts():
    mesh = dict(inputs.mesh_dict("euler", 2, 3, [256, 256], [0.0, 0.0], [1.0, 1.0], 1.4), limiter=True,
                alpha_max=0.7)
    X = inputs.node_coords(mesh)
    slab = 1.0 + (np.tanh(300.0 * (X[0] - 0.3)) - np.tanh(300.0 * (X[0] - 0.65)))
    one = np.ones_like(X[0])
    return mesh, inputs.euler_cons(1.4, slab * (1.0 + 0.1 * np.sin(2 * np.pi * X[1])), [0.4 * one, 0.1 * one], slab)


_PEAKS = {}


def peaks():
    """FP32 peak (lanes x max clock), FP64 peak (measured FMA rate) in
    TFLOP/s and the measured HBM copy bandwidth in GB/s."""
    if not _PEAKS:
        try:
            with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                   "MEASURED_PEAKS.json")) as f:
                mp = json.load(f)
        except OSError:
            mp = {}
        _PEAKS["fp32_tflops"] = 152 * 128 * 2 * mp.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        _PEAKS["fp64_tflops"] = 2 * crkfr.probe_peaks(["dfma"])["dfma"] / 1e12
        _PEAKS["hbm_gbs"] = mp.get("hbm_gbs", 6800.0)
        _PEAKS["source"] = ("fp32: 152 SMs x 128 lanes x 2 x max SM clock; fp64: 2 x cr_probe_peak FP64 FMA rate; "
                            + ("hbm: MEASURED_PEAKS.json" if "hbm_gbs" in mp else "hbm: fallback 6.8 TB/s"))
    return _PEAKS


def roofline(mesh, prec, vol_ms, face_ms):
    """Volume kernel against the ALU peak of its precision, face / update
    kernel against HBM (counted work: paper_2604_02125_gb300.work)."""
    pk = peaks()
    vf = work.volume_flops(mesh)
    fb = work.face_bytes(mesh, 8 if prec == "fp64" else 4)
    vpeak = pk["fp64_tflops"] if prec == "fp64" else pk["fp32_tflops"]
    out = {"volume": {"bound": "alu", "gflop_per_launch": vf / 1e9, "tflops": vf / (vol_ms * 1e-3) / 1e12,
                      "peak_tflops": vpeak, "frac": vf / (vol_ms * 1e-3) / 1e12 / vpeak}}
    if face_ms:
        out["face_update"] = {"bound": "hbm", "mb_per_launch": fb / 1e6, "gbs": fb / (face_ms * 1e-3) / 1e9,
                              "peak_gbs": pk["hbm_gbs"], "frac": fb / (face_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
    return out


def _stagewise(mesh, U):
    return dict(mesh, ncflux="stages"), U


def nodes_of(mesh):
    return inputs.num_elems(mesh) * inputs.nodes_per_elem(mesh)


def time_solver(s, steps, stream, flush):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        s.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def measure_gpu(name, make, desc, steps, budget_steps):
    import torch
    mesh, U = make()
    nodes = nodes_of(mesh)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    out = {"workload": name, "description": desc, "nodes": nodes, "vars": int(U.shape[0]), "forms": {}}
    finals = {}
    with torch.cuda.stream(stream):
        for prec in ("fp64", "fp32"):
            s = crkfr.Solver(mesh, prec=prec, stream=stream)
            s.set_state(U)
            s.step(3)
            s.sync()
            ms = time_solver(s, steps, stream, flush)
            vol, face = s.time_kernels(max(3, min(steps, 20)), flush)
            out["forms"][prec] = {"dof_updates_per_s": nodes / (ms * 1e-3), "ms_per_step": ms,
                                  "volume_ms": vol, "face_update_ms": face, "status": crkfr.status_string(s.info()["status"])}
            if not mesh.get("limiter"):
                out["forms"][prec]["roofline"] = roofline(mesh, prec, vol, face)
            else:
                # the limiter: coefficient kernel + the same volume kernel, then
                # the per-node limited face / update kernel; against the
                # unlimited step on the same mesh
                out["forms"][prec]["volume_note"] = "volume_ms includes the coefficient kernel"
                p = crkfr.Solver(dict(mesh, limiter=False), prec=prec, stream=stream)
                p.set_state(U)
                p.step(3)
                p.sync()
                mp = time_solver(p, steps, stream, flush)
                p.close()
                out["forms"][prec]["unlimited_ms_per_step"] = mp
                out["forms"][prec]["limiter_cost"] = ms / mp
            s.close()
            # 100 steps from the initial state for the FP32-vs-FP64 error
            s = crkfr.Solver(mesh, prec=prec, stream=stream)
            s.set_state(U)
            s.step(100)
            finals[prec] = s.get_state()
            s.close()
        out["rel_l2_fp32_vs_fp64_after_100_steps"] = float(
            np.linalg.norm(finals["fp32"] - finals["fp64"]) / np.linalg.norm(finals["fp64"]))
        # the multi-stage RKFR scheme on the same workload and kernels (its
        # stages take the stage traces anyway: no stage-wise flux option)
        out["rkfr"] = {}
        for prec in (("fp64", "fp32") if mesh.get("ncflux", "reduced") == "reduced" and not mesh.get("limiter")
                     else ()):
            s = crkfr.Solver(mesh, prec=prec, stream=stream, scheme="rkfr")
            s.set_state(U)
            s.step(3)
            s.sync()
            ms = time_solver(s, steps, stream, flush)
            vol, face = s.time_kernels(max(3, min(steps, 20)), flush)
            out["rkfr"][prec] = {"dof_updates_per_s": nodes / (ms * 1e-3), "ms_per_step": ms,
                                 "volume_ms_per_step": vol, "face_update_ms_per_step": face,
                                 "crkfr_speedup": ms / out["forms"][prec]["ms_per_step"],
                                 "status": crkfr.status_string(s.info()["status"])}
            s.close()
        if name.startswith("tgv3d") and budget_steps > 0:
            out["budgets"] = {}
            for prec in ("fp64", "fp32"):
                s = crkfr.Solver(mesh, prec=prec, stream=stream)
                s.set_state(U)
                i0 = s.info(totals=True)
                s.step(budget_steps)
                i1 = s.info(totals=True)
                M = int(U.shape[0])
                ke0, ke1 = i0["totals"][M], i1["totals"][M]
                en0, en1 = i0["totals"][M + 1], i1["totals"][M + 1]
                out["budgets"][prec] = {"steps": budget_steps, "t": i1["t"],
                                        "kinetic_energy_rel_change": (ke1 - ke0) / abs(ke0),
                                        "entropy_change": en1 - en0, "entropy_rel_change": (en1 - en0) / abs(en0)}
                s.close()
    return out


def measure_long(steps):
    """The shear layer over its full run length: FP32 pair-flux form against the
    FP64 path (itself pinned to the oracle per step), FP64 totals of both."""
    import torch
    mesh, U = inputs.shear_layer_2d(cells=(256, 256), N=3)
    out = {"workload": "shear2d_256_N3_long", "steps": steps, "forms": {}}
    finals = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for prec in ("fp64", "fp32"):
            s = crkfr.Solver(mesh, prec=prec, stream=stream)
            s.set_state(U)
            i0 = s.info(totals=True)
            s.step(steps)
            i1 = s.info(totals=True)
            finals[prec] = s.get_state(check=False)
            M = int(U.shape[0])
            scale = np.abs(U).reshape(M, -1).sum(axis=1) / U[0].size
            out["forms"][prec] = {
                "status": crkfr.status_string(i1["status"]), "t": i1["t"],
                "conservation_rel": [float(abs(i1["totals"][v] - i0["totals"][v]) / max(abs(i0["totals"][v]), scale[v]))
                                     for v in range(M)],
                "kinetic_energy_rel_change": float((i1["totals"][M] - i0["totals"][M]) / abs(i0["totals"][M])),
                "entropy_rel_change": float((i1["totals"][M + 1] - i0["totals"][M + 1]) / abs(i0["totals"][M + 1]))}
            s.close()
    out["rel_l2_fp32_vs_fp64"] = float(np.linalg.norm(finals["fp32"] - finals["fp64"]) / np.linalg.norm(finals["fp64"]))
    return out


def measure_batched(steps):
    import torch
    specs = inputs.batched_2d_specs()
    solves = [inputs.batched_2d_solve(sp) for sp in specs]
    meshes = [m for m, _ in solves]
    nodes = sum(nodes_of(m) for m in meshes)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = crkfr.Solver(meshes, prec="fp32", stream=stream)
        for k, (_, U) in enumerate(solves):
            b.set_state(U, solve=k)
        b.step(2)
        b.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            ev[k][0].record(stream)
            b.step(1)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(c) for a, c in ev) / steps
        tuning = b.tuning_info()
        b.close()
        seq = sequential_batch(meshes, [U for _, U in solves], steps, stream)
    return {"workload": "batched2d_512", "description": "512 independent 2D Euler solves, sides 16..128, N 2..5",
            "nodes": nodes, "forms": {"fp32": {"dof_updates_per_s": nodes / (ms * 1e-3), "ms_per_step": ms}},
            "sequential": seq, "batched_vs_sequential": seq["ms_per_step"] / ms, "tuning": tuning}


def sequential_batch(meshes, states, steps, stream):
    """The same solves advanced one after another, each through its own
    single-solve FP32 context (its 1-step CUDA graph), on one stream: the
    alternative to the batched persistent kernels."""
    import torch
    ctxs = []
    for m, U in zip(meshes, states):
        c = crkfr.Solver(m, prec="fp32", stream=stream)
        c.set_state(U)
        ctxs.append(c)
    for c in ctxs:
        c.step(2)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        for c in ctxs:
            c.step(1)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    status = max(abs(c.info()["status"]) for c in ctxs)
    for c in ctxs:
        c.close()
    nodes = sum(nodes_of(m) for m in meshes)
    return {"dof_updates_per_s": nodes / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "status": status,
            "mode": "%d single-solve FP32 contexts, one 1-step graph launch each per step, one stream" % len(meshes)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--budget-steps", type=int, default=500)
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--long-steps", type=int, default=2000, help="run length of the shear-layer long run (0: skip)")
    a = ap.parse_args(argv)
    names = a.only or list(WORKLOADS) + ["batched2d_512", "shear2d_256_N3_long"]
    build.build()
    for name in names:
        if name == "shear2d_256_N3_long":
            if a.long_steps > 0:
                print(json.dumps(measure_long(a.long_steps)), flush=True)
        elif name == "batched2d_512":
            print(json.dumps(measure_batched(max(3, min(a.steps, 10)))), flush=True)
        else:
            make, desc = WORKLOADS[name]
            print(json.dumps(measure_gpu(name, make, desc, a.steps, a.budget_steps)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

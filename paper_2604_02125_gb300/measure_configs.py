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

from paper_2604_02125_gb300 import build, crkfr, inputs  # noqa: E402

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
}


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
        for prec in (("fp64", "fp32") if mesh.get("ncflux", "reduced") == "reduced" else ()):
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
    return {"workload": "batched2d_512", "description": "512 independent 2D Euler solves, sides 16..128, N 2..5",
            "nodes": nodes, "forms": {"fp32": {"dof_updates_per_s": nodes / (ms * 1e-3), "ms_per_step": ms}},
            "tuning": tuning}


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

"""Benchmark of the cRKFR hot path on one GB300 (DOF-updates/s).

A "step" is one cRKFR time step (volume kernel + face/update kernel) of the
2D Euler shear layer on 256 x 256 quads, N = 3 (1,048,576 nodes), with FP32
pair fluxes and the FP64 state update (the headline form).  Each timed step
is bracketed by CUDA events on the solver's stream; between timed steps a
256 MiB buffer is written to flush the 129 MB L2 (the step's working set,
about 110 MB, would otherwise stay L2-resident).

Also reported: the plain FP64 form on the same workload (fewer steps), the
end-to-end rate through the C ABI with host buffers (copies inside the timed
region), the volume kernel's roofline fraction, SM clocks sampled during the
timed region, and the FP64 CPU oracle timed on the host cores on a bounded
sample of the workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 (torchrun) every rank advances its own replica (the method needs
no exchange between independent replicas): weak scaling, max time over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cRKFR DOF-updates/s (FP32-flux & batched vs plain FP64, 1 GB300) at stated L2 error"
WORKLOAD = "2D compressible Euler shear layer, periodic [-1,1]^2, 256x256 quads, N=3, EC (Ranocha) flux, Rusanov"
CELLS = (256, 256)
N_DEG = 3


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# Algorithmic work of the volume kernel (flops counted from the formulas) and
# of the face / update kernel (bytes): paper_2604_02125_gb300/work.py.  2D
# Euler, EC flux: 75 flops per pair flux, 61 per node and stage.
def volume_flops_2d(E, N, stages):
    from paper_2604_02125_gb300 import work
    side = int(round(E ** 0.5))
    mesh = {"eq": "euler", "dim": 2, "N": N, "cells": [side, E // side], "vol": "ec"}
    return work.volume_flops(mesh, stages)


class ClockSampler:
    """nvidia-smi clock/throttle sampling (200 ms) around a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self, wait_s=3.0):
        """Start sampling; returns once the first sample is in (or after wait_s)."""
        try:
            self.out = open(os.path.join(ROOT, ".clocks_%d.csv" % os.getpid()), "w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < wait_s and self.proc.poll() is None:
            self.out.flush()
            if os.path.getsize(self.out.name) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        name = self.out.name
        self.out.close()
        os.remove(name)
        sm, mx, reasons = [], [], set()
        keys = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, v in zip(keys, r[5:9]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(k)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def job_time_ms(local_ms, world, dist=None, device="cuda"):
    """Whole-job time of a timed region: the maximum over ranks."""
    if world <= 1:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(nodes_per_rank, steps, world, job_ms):
    """DOF-updates/s of the whole job: every rank advances its own replica."""
    return world * nodes_per_rank * steps / (job_ms * 1e-3)


VOLUME_PROFILE = os.path.join(ROOT, "profiles", "k_volume_lanes_shear2d_256x256_N3_fp32.md")
FACE_PROFILE = os.path.join(ROOT, "profiles", "k_face_update_lanes_shear2d_256x256_N3_fp32.md")


def time_steps(solver, steps, stream, flush):
    """Per-step CUDA-event time (ms) of `steps` solver steps, L2 flushed between."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        solver.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def cpu_baseline(sample_cells=(128, 128), steps=6):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    from paper_2604_02125_gb300 import inputs
    oracle.build()
    mesh, U = inputs.shear_layer_2d(cells=sample_cells, N=N_DEG)
    t0 = time.perf_counter()
    for _ in range(steps):
        U = oracle.step(mesh, U, oracle.cfl_dt(mesh, U))
    dtw = time.perf_counter() - t0
    nodes = inputs.num_elems(mesh) * inputs.nodes_per_elem(mesh)
    return {"value": nodes * steps / dtw, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle",
            "sample": "%d steps of the same shear layer on %dx%d quads, N=%d (%d nodes), single thread, %.1f s"
                      % (steps, sample_cells[0], sample_cells[1], N_DEG, nodes, dtw)}


def _oracle_part(args):
    """Worker of the all-cores oracle timing: the oracle's restricted step
    (or_step_elements, the full step's routines on the selected elements and
    their neighbours) for elements [e_lo, e_hi), read from and written to
    shared memory."""
    from multiprocessing import shared_memory
    import oracle
    name_in, name_out, shape, mesh, dt, e_lo, e_hi = args
    si, so = shared_memory.SharedMemory(name=name_in), shared_memory.SharedMemory(name=name_out)
    try:
        U = np.ndarray(shape, dtype=np.float64, buffer=si.buf)
        out = np.ndarray(shape, dtype=np.float64, buffer=so.buf)
        out[:, e_lo:e_hi, :] = oracle.step_elements(mesh, U, dt, np.arange(e_lo, e_hi))
    finally:
        si.close()
        so.close()
    return e_hi - e_lo


def oracle_parallel_steps(mesh, U, steps, workers):
    """`steps` oracle steps of (mesh, U) on `workers` processes (spawned: safe
    after CUDA use), each advancing a contiguous range of elements with the
    unchanged oracle; dt from the oracle's CFL rule on each step's state.
    Returns (U after the steps, seconds of the steps without the pool start)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle
    oracle.build()
    E = U.shape[1]
    bounds = np.linspace(0, E, workers + 1).astype(int)
    bufs = [shared_memory.SharedMemory(create=True, size=U.nbytes) for _ in range(2)]
    try:
        arrs = [np.ndarray(U.shape, dtype=np.float64, buffer=b.buf) for b in bufs]
        arrs[0][...] = U
        with mp.get_context("spawn").Pool(workers) as pool:
            pool.map(_oracle_part, [(bufs[0].name, bufs[1].name, U.shape, mesh, 0.0, 0, 1)])   # start the workers
            t0 = time.perf_counter()
            cur = 0
            for _ in range(steps):
                dt = oracle.cfl_dt(mesh, arrs[cur])
                pool.map(_oracle_part, [(bufs[cur].name, bufs[1 - cur].name, U.shape, mesh, dt, int(bounds[k]),
                                         int(bounds[k + 1])) for k in range(workers) if bounds[k + 1] > bounds[k]])
                cur = 1 - cur
            el = time.perf_counter() - t0
        return arrs[cur].copy(), el
    finally:
        for b in bufs:
            b.close()
            b.unlink()


def cpu_baseline_all_cores(steps=4):
    """The oracle, as it stands, on every host core: the full 256^2 workload,
    elements split into contiguous ranges across worker processes."""
    from paper_2604_02125_gb300 import inputs
    workers = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    mesh, U = inputs.shear_layer_2d(cells=CELLS, N=N_DEG)
    _, el = oracle_parallel_steps(mesh, U, steps, workers)
    nodes = inputs.num_elems(mesh) * inputs.nodes_per_elem(mesh)
    return {"value": nodes * steps / el, "unit": "DOF-updates/s", "cores": workers, "kind": "oracle",
            "sample": "%d steps of the full %dx%d N=%d workload (%d nodes) on %d processes, each the unchanged "
                      "oracle's restricted step on a contiguous range of elements, %.1f s"
                      % (steps, CELLS[0], CELLS[1], N_DEG, nodes, workers, el)}


def run_batched(crkfr, inputs, stream, steps):
    """512 independent 2D Euler solves (sides 16..128, N in 2..5, FP32 pair
    fluxes, FP64 update) advanced together; per-step CUDA events on the
    stream.  The 2.3 GB state is far larger than L2."""
    import torch
    specs = inputs.batched_2d_specs()
    solves = [inputs.batched_2d_solve(sp) for sp in specs]
    meshes = [m for m, _ in solves]
    nodes = sum(inputs.num_elems(m) * inputs.nodes_per_elem(m) for m in meshes)
    b = crkfr.Solver(meshes, prec="fp32", stream=stream)
    for k, (_, U) in enumerate(solves):
        b.set_state(U, solve=k)
    b.step(2)                      # autotune + graph capture happen here
    b.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        ev[k][0].record(stream)
        b.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(c) for a, c in ev) / steps
    info = b.tuning_info()
    status = b.info(solve=0)["status"]
    b.close()
    # the same solves one after another through single-solve contexts: what
    # the persistent per-degree kernels and their autotuning gain
    from paper_2604_02125_gb300.measure_configs import sequential_batch
    seq = sequential_batch(meshes, [U for _, U in solves], steps, stream)
    # roofline of the per-degree volume kernels: counted FP32 flops of every
    # solve of that degree / the kernel's autotuned launch time
    stages = {1: 2, 2: 3, 3: 4, 4: 6, 5: 7}
    flops = {}
    for m in meshes:
        flops[m["N"]] = flops.get(m["N"], 0) + volume_flops_2d(inputs.num_elems(m), m["N"], stages[m["N"]])
    peaks = _peaks()
    fp32_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    vol_roof = {}
    for N, f in sorted(flops.items()):
        t = info.get("N%d_volume" % N, {}).get("ms")
        if t:
            vol_roof["N%d" % N] = {"tflops": f / (t * 1e-3) / 1e12, "frac": f / (t * 1e-3) / 1e12 / fp32_peak,
                                   "gflop_per_launch": f / 1e9, "ms_per_launch": t}
    return {"value": nodes / (ms * 1e-3), "ms_per_step": ms, "steps": steps, "solves": len(meshes),
            "nodes": nodes, "status": crkfr.status_string(status), "tuning": info,
            "vs_sequential": seq["ms_per_step"] / ms, "sequential": seq,
            "volume_roofline": dict(vol_roof, bound="alu", peak_tflops=fp32_peak,
                                    note="launch times from the autotuner (best of two, warm L2)"),
            "workload": "512 independent 2D Euler solves, sides 16..128 quads, N in {2,3,4,5}, seeded smooth "
                        "densities (amplitude 0.1-0.5) and shear, FP32 pair fluxes, FP64 update"}


# reduced meshes of every workload for single-threaded oracle timings (a few
# seconds each); the GPU side of the same workloads is measured by
# paper_2604_02125_gb300/measure_configs.py
ORACLE_SAMPLES = {
    "wave1d_64_N3": ("density_wave_1d", dict(cells=64, N=3), 2000),
    "shear2d_256_N3": ("shear_layer_2d", dict(cells=(32, 32), N=3), 40),
    "shear2d_256_N3_kep": ("shear_layer_2d", dict(cells=(32, 32), N=3, vol="kep"), 40),
    "shear2d_256_N3_central": ("shear_layer_2d", dict(cells=(32, 32), N=3, vol="central"), 40),
    "mhd2d_128_N4": ("mhd_vortex_2d", dict(cells=(16, 16), N=4), 40),
    "tgv3d_64_N3": ("tgv_3d", dict(cells=(8, 8, 8), N=3), 20),
    # the multi-stage RKFR scheme and the stage-wise non-conservative flux
    "shear2d_256_N3_rkfr": ("shear_layer_2d", dict(cells=(32, 32), N=3), 40, "rkfr"),
    "mhd2d_128_N4_ncstages": ("mhd_vortex_2d", dict(cells=(16, 16), N=4), 40, "ncstages"),
}


def cpu_baseline_configs():
    """The FP64 oracle, single thread, on a reduced mesh of every workload."""
    import oracle
    from paper_2604_02125_gb300 import inputs
    oracle.build()
    for name, (fn, kw, steps, *variant) in ORACLE_SAMPLES.items():
        mesh, U = getattr(inputs, fn)(**kw)
        step = oracle.step
        if variant == ["rkfr"]:
            step = oracle.rkfr_step
        elif variant == ["ncstages"]:
            mesh = dict(mesh, ncflux="stages")
        t0 = time.perf_counter()
        for _ in range(steps):
            U = step(mesh, U, oracle.cfl_dt(mesh, U))
        el = time.perf_counter() - t0
        nodes = inputs.num_elems(mesh) * inputs.nodes_per_elem(mesh)
        print(json.dumps({"workload": name, "kind": "oracle", "cores": 1, "dof_updates_per_s": nodes * steps / el,
                          "sample": "%s%s, %d steps, %d nodes, %.2f s" % (fn, kw, steps, nodes, el)}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_2604_02125_gb300 import inputs
    oracle.build()
    cells = (24, 24)
    mesh, U = inputs.shear_layer_2d(cells=cells, N=N_DEG)
    for _ in range(args.warmup):
        U = oracle.step(mesh, U, oracle.cfl_dt(mesh, U))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = oracle.step(mesh, U, oracle.cfl_dt(mesh, U))
    el = time.perf_counter() - t0
    nodes = inputs.num_elems(mesh) * inputs.nodes_per_elem(mesh)
    value = nodes * args.steps / el
    sample = ("each step: one oracle step of the shear layer on %dx%d quads, N=%d (%d nodes), FP64, single thread"
              % (cells[0], cells[1], N_DEG, nodes))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (bounded CPU sample, %dx%d quads)" % cells, "form": "fp64 oracle"},
        "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--cpu-baseline-configs", action="store_true",
                    help="only time the FP64 oracle on reduced meshes of every workload")
    args = ap.parse_args()
    if args.cpu_baseline_configs:
        return cpu_baseline_configs()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2604_02125_gb300 import build, crkfr, inputs
    build.build()
    mesh, U = inputs.shear_layer_2d(cells=CELLS, N=N_DEG)
    E = inputs.num_elems(mesh)
    nodes = E * inputs.nodes_per_elem(mesh)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        s32 = crkfr.Solver(mesh, prec="fp32", stream=stream)
        s32.set_state(U)
        s32.step(args.warmup)
        s32.sync()
        # clocks are sampled from just before the first timed region to the
        # end of the last one (headline, FP64 form, batched form, per kernel)
        clk = ClockSampler(local)
        clk.start()
        barrier()
        times = time_steps(s32, args.steps, stream, flush)
        barrier()
        status = s32.info()["status"]
        total_ms = job_time_ms(sum(times), world, dist)
        value = job_value(nodes, args.steps, world, total_ms)

        # plain FP64 form, same workload, a few steps
        k64 = max(3, min(30, args.steps))
        s64 = crkfr.Solver(mesh, prec="fp64", stream=stream)
        s64.set_state(U)
        s64.step(2)
        s64.sync()
        t64 = time_steps(s64, k64, stream, flush)
        s64.close()

        # error of the FP32 pair-flux form against the FP64 path (itself pinned to
        # the FP64 oracle at 1e-12 per step) after 100 steps from the same state
        e32 = crkfr.Solver(mesh, prec="fp32", stream=stream)
        e64 = crkfr.Solver(mesh, prec="fp64", stream=stream)
        e32.set_state(U)
        e64.set_state(U)
        e32.step(100)
        e64.step(100)
        a32, a64 = e32.get_state(), e64.get_state()
        err100 = float(np.linalg.norm(a32 - a64) / np.linalg.norm(a64))
        time32, time64 = e32.info()["t"], e64.info()["t"]
        e32.close()
        e64.close()

        batched = None if args.no_batched else run_batched(crkfr, inputs, stream, max(3, min(10, args.steps)))

        # the subcell blending limiter with the paper's Kelvin-Helmholtz
        # setting (KEP volume flux, alpha_max = 0.008) on the same mesh,
        # against the unlimited step with the same flux
        mk, Uk = inputs.shear_layer_2d(cells=CELLS, N=N_DEG, vol="kep")
        lim = {}
        kl = max(3, min(200, args.steps))
        for tag, m in (("limited", dict(mk, limiter=True, alpha_max=0.008)), ("unlimited", mk)):
            r = crkfr.Solver(m, prec="fp32", stream=stream)
            r.set_state(Uk)
            r.step(2)
            r.sync()
            tl = time_steps(r, kl, stream, flush)
            lim[tag] = {"ms_per_step": sum(tl) / kl, "value": nodes * kl / (sum(tl) * 1e-3), "steps": kl,
                        "status": crkfr.status_string(r.info()["status"])}
            r.close()
        lim["cost"] = lim["limited"]["ms_per_step"] / lim["unlimited"]["ms_per_step"]

        # the multi-stage RKFR scheme (eq. rkfr.non.cons) on the same workload
        # and kernels: s volume and s face exchanges per step, against one
        # each -- the single-stage advantage the compact scheme is built for
        rkfr = {}
        for prec, krk in (("fp32", max(3, min(200, args.steps))), ("fp64", k64)):
            r = crkfr.Solver(mesh, prec=prec, stream=stream, scheme="rkfr")
            r.set_state(U)
            r.step(2)
            r.sync()
            trk = time_steps(r, krk, stream, flush)
            rv, rf = r.time_kernels(max(3, min(20, args.steps)), flush)
            r.close()
            rkfr[prec] = {"value": nodes * krk / (sum(trk) * 1e-3), "ms_per_step": sum(trk) / krk, "steps": krk,
                          "volume_ms_per_step": rv, "face_update_ms_per_step": rf}

        # volume-kernel duration, CUDA events on the solver's stream, same L2 flush
        kv = max(3, min(50, args.steps))
        vol_ms, face_ms = s32.time_kernels(kv, flush)
        clocks = clk.stop()

        # end to end through the C ABI with host buffers: every step uploads
        # the full state from pinned host memory, advances it one step and
        # downloads the full result.  Pipelined: three contexts on their own
        # streams take the steps in turn with the asynchronous copies, so one
        # step's upload and another's download overlap a third's compute.
        Uh = torch.from_numpy(U).pin_memory()
        ke = max(6, min(60, args.steps))
        ctxs = [crkfr.Solver(mesh, prec="fp32", stream=torch.cuda.Stream()) for _ in range(3)]
        outs = [torch.empty_like(Uh).pin_memory() for _ in range(3)]
        for c in ctxs:   # warm-up of every context
            c.set_state(Uh)
            c.step(1)
            c.sync()
        barrier()
        t0 = time.perf_counter()
        for k in range(ke):
            c = ctxs[k % 3]
            c.set_state(Uh, sync=False)
            c.step(1)
            c.get_state(outs[k % 3], sync=False)
        for c in ctxs:
            c.sync()
        barrier()
        e2e_s = job_time_ms((time.perf_counter() - t0) * 1e3, world, dist) * 1e-3
        # the result of every pipelined step equals the device-side step
        s32.set_state(U)
        s32.step(1)
        ref = s32.get_state()
        e2e_ok = all(np.array_equal(o.numpy(), ref) for o in outs)
        link = crkfr.probe_peaks(["h2d_bytes", "d2h_bytes", "duplex_bytes_per_direction"])
        for c in ctxs:
            c.close()
        # the same, one context, synchronous copies (set_state / get_state wait)
        Oh = outs[0]
        kq = max(3, min(20, args.steps))
        barrier()
        t0 = time.perf_counter()
        for _ in range(kq):
            s32.set_state(Uh)
            s32.step(1)
            s32.get_state(Oh)
        barrier()
        seq_s = job_time_ms((time.perf_counter() - t0) * 1e3, world, dist) * 1e-3
        s32.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    stages = 4
    vflops = volume_flops_2d(E, N_DEG, stages)
    peaks = _peaks()
    sm_mhz_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_mhz_max * 1e6 / 1e12     # TFLOP/s, FP32 FMA lanes x clock
    ms_step = total_ms / args.steps
    roofline = None
    if vol_ms:
        from paper_2604_02125_gb300 import profile_summary
        prof = profile_summary.read_profile_traffic(VOLUME_PROFILE)
        ach = vflops / (vol_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                    "peak_source": "FP32 lanes x max SM clock: 152 SMs x 128 lanes x 2 flops x %.0f MHz" % sm_mhz_max,
                    "traffic": prof[1] if prof else None,
                    "traffic_source": os.path.relpath(VOLUME_PROFILE, ROOT) if prof else "no capture of these sources",
                    "kernel": "k_volume_lanes<Euler<2>,3,float>", "flops_per_launch": vflops,
                    "ms_per_launch": vol_ms, "face_update_ms_per_launch": face_ms}
        if face_ms:
            # face/update kernel against HBM: algorithmic bytes per DOF-update
            # (2D Euler, FP32 form) = u read 32 + Rbar read 16 + own face
            # records 2 dirs x 2 sides x (N+1) face nodes x C comps x 4 B / (N+1)^2
            # nodes + u written 32 (the neighbours' records are the same data)
            C = 2 * 4 + 1
            rec = 2 * 2 * (N_DEG + 1) * C * 4 / (N_DEG + 1) ** 2
            fbytes = nodes * (32 + 16 + rec + 32)
            hbm = peaks.get("hbm_gbs")
            fprof = profile_summary.read_profile_traffic(FACE_PROFILE)
            roofline["face_update"] = {
                "bound": "hbm", "achieved": fbytes / (face_ms * 1e-3) / 1e9, "unit": "GB/s",
                "peak": hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs" if hbm else None,
                "frac": (fbytes / (face_ms * 1e-3) / 1e9 / hbm) if hbm else None,
                "bytes_per_launch": fbytes, "traffic": fprof[1] if fprof else None}
    # multi-stage RKFR, FP32 form: the face/update stages against HBM, the
    # single-stage volume launches against the FP32 peak (same flops as the
    # cRKFR volume kernel: every stage's flux differencing).  Algorithmic bytes
    # per DOF-update of the face stages with RK4 (A subdiagonal, every b_q
    # non-zero): per stage u^n 32 + Rbar 16 + own records + output state 32,
    # plus the kept increments K_0..K_2 written once (16 each) and read once by
    # the last stage (16 each); the inner stages read no earlier K.
    if rkfr.get("fp32", {}).get("face_update_ms_per_step"):
        C = 2 * 4 + 1
        rec = 2 * 2 * (N_DEG + 1) * C * 4 / (N_DEG + 1) ** 2
        rk_bytes = nodes * (stages * (32 + 16 + rec + 32) + 16 * (stages - 1) * 2)
        hbm = peaks.get("hbm_gbs")
        fms, vms = rkfr["fp32"]["face_update_ms_per_step"], rkfr["fp32"]["volume_ms_per_step"]
        rkfr["fp32"]["face_roofline"] = {"bound": "hbm", "achieved": rk_bytes / (fms * 1e-3) / 1e9, "unit": "GB/s",
                                         "peak": hbm, "frac": (rk_bytes / (fms * 1e-3) / 1e9 / hbm) if hbm else None,
                                         "bytes_per_step": rk_bytes}
        rkfr["fp32"]["volume_roofline"] = {"bound": "alu", "achieved": vflops / (vms * 1e-3) / 1e12,
                                           "unit": "TFLOP/s", "peak": fp32_peak,
                                           "frac": vflops / (vms * 1e-3) / 1e12 / fp32_peak}
    out = {
        "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "fp32 pair fluxes, fp64 update", "elements": E, "nodes": nodes,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "gpu_launches": 2 * args.steps,
        "status": crkfr.status_string(status),
        "forms": {"fp32_pairflux": {"value": value, "ms_per_step": ms_step,
                                    "rel_l2_vs_fp64_after_100_steps": err100,
                                    "rel_t_vs_fp64_after_100_steps": abs(time32 - time64) / time64,
                                    "dt": "FP64 maximum and division, FP32 wave speeds of the FP64 state (reading "
                                          "R15): dt within 1e-6 of the oracle's per step"},
                  "limiter": dict(lim, setting="KEP volume flux, subcell blending limiter alpha_max = 0.008 (the "
                                               "paper's Kelvin-Helmholtz runs), FP32 form; per step the coefficient "
                                               "kernel, the volume kernel and the limited per-node face / update kernel",
                                  rel_l2_vs_oracle="<= 1e-12 per step (FP64), tests/test_gpu_limiter.py"),
                  "fp64": {"value": nodes * k64 / (sum(t64) * 1e-3), "ms_per_step": sum(t64) / k64, "steps": k64,
                           "rel_l2_vs_oracle_per_step": "<= 1e-12 (tests/test_gpu_parity.py)"},
                  "batched": batched,
                  "rkfr": dict(rkfr, scheme="multi-stage RKFR, %d stages: per stage one single-stage volume launch "
                               "and one face/update launch" % stages,
                               crkfr_speedup={"fp32": rkfr["fp32"]["ms_per_step"] / ms_step,
                                              "fp64": rkfr["fp64"]["ms_per_step"] / (sum(t64) / k64)},
                               rel_l2_vs_oracle="<= 1e-12 per step (FP64), <= 1e-5 after 100 steps (FP32): "
                                                "tests/test_gpu_rkfr.py")},
        "e2e": {"value": world * nodes * ke / e2e_s, "unit": "DOF-updates/s",
                "h2d_bytes_per_step": int(U.nbytes), "d2h_bytes_per_step": int(U.nbytes),
                "mode": "per step: full state H2D from pinned memory, one step, full state D2H; 3 contexts "
                        "pipelined with cr_set_state_async / cr_get_state_async; %d steps" % ke,
                "results_match_device_step": e2e_ok,
                # the host link bounds it: per step one state each way, both directions at once
                "link_roofline": {"duplex_gbs_per_direction": link["duplex_bytes_per_direction"] / 1e9,
                                  "h2d_gbs": link["h2d_bytes"] / 1e9, "d2h_gbs": link["d2h_bytes"] / 1e9,
                                  "floor_ms_per_step": 1e3 * U.nbytes / link["duplex_bytes_per_direction"],
                                  "frac": (U.nbytes / link["duplex_bytes_per_direction"]) / (e2e_s / ke)},
                "sequential": {"value": world * nodes * kq / seq_s, "steps": kq,
                               "mode": "one context, cr_set_state / cr_step / cr_get_state (synchronous)"}},
        "roofline": roofline,
        "clocks": dict(clocks, window="headline, fp64, batched, limiter, rkfr and per-kernel timed regions") if clocks else None,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
        out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores()
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Run one cRKFR workload through the C ABI (used for profiling and by users).

  python -m paper_2604_02125_gb300.run_case --case shear2d --cells 256 256 --N 3 --prec fp32 --steps 3

Cases: wave1d, shear2d, mhd2d, tgv3d, fronts2d (a steep density / pressure slab
across x on [0,1]^2); --scheme rkfr runs the multi-stage RKFR scheme instead of
the single-stage cRKFR step, --ncflux stages (mhd2d) the stage-wise
non-conservative flux, --limiter [--alpha-max A] the subcell blending limiter
(Euler).  Prints the step count, time and dt.
"""
import argparse
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2604_02125_gb300 import build, crkfr, inputs  # noqa: E402

CASES = {
    "wave1d": lambda c, N, vol: inputs.density_wave_1d(cells=c[0], N=N, vol=vol),
    "shear2d": lambda c, N, vol: inputs.shear_layer_2d(cells=tuple(c[:2]), N=N, vol=vol),
    "mhd2d": lambda c, N, vol: inputs.mhd_vortex_2d(cells=tuple(c[:2]), N=N, vol=vol),
    "tgv3d": lambda c, N, vol: inputs.tgv_3d(cells=tuple(c[:3]), N=N, vol=vol),
    "fronts2d": lambda c, N, vol: _fronts(c, N, vol),
}


def _fronts(c, N, vol):
    import numpy as np
    mesh = inputs.mesh_dict("euler", 2, N, list(c[:2]), [0.0, 0.0], [1.0, 1.0], 1.4, vol=vol)
    X = inputs.node_coords(mesh)
    slab = 1.0 + (np.tanh(300.0 * (X[0] - 0.3)) - np.tanh(300.0 * (X[0] - 0.65)))
    one = np.ones_like(X[0])
    return mesh, inputs.euler_cons(1.4, slab * (1.0 + 0.1 * np.sin(2 * np.pi * X[1])), [0.4 * one, 0.1 * one], slab)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="shear2d", choices=sorted(CASES))
    ap.add_argument("--cells", type=int, nargs="+", default=[256, 256])
    ap.add_argument("--N", type=int, default=3)
    ap.add_argument("--vol", default="ec")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--scheme", default="crkfr", choices=["crkfr", "rkfr"])
    ap.add_argument("--ncflux", default="reduced", choices=["reduced", "stages"])
    ap.add_argument("--limiter", action="store_true")
    ap.add_argument("--alpha-max", type=float, default=0.7)
    a = ap.parse_args(argv)
    build.build()
    mesh, U = CASES[a.case](a.cells, a.N, a.vol)
    mesh = dict(mesh, ncflux=a.ncflux)
    if a.limiter:
        mesh = dict(mesh, limiter=True, alpha_max=a.alpha_max)
    with crkfr.Solver(mesh, prec=a.prec, scheme=a.scheme) as s:
        s.set_state(U)
        t0 = time.perf_counter()
        s.step(a.steps)
        s.sync()
        el = time.perf_counter() - t0
        info = s.info()
    print("%s cells=%s N=%d %s %s: %d steps in %.3f s, t=%.6g dt=%.6g status=%d"
          % (a.case, a.cells, a.N, a.prec, a.scheme, info["steps"], el, info["t"], info["dt"], info["status"]))
    return 0 if info["status"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())

"""Algorithmic work of one cRKFR step, for roofline fractions.

Counted from the formulas the kernels evaluate (an add, multiply or
reciprocal is one flop, a fused multiply-add two, a compare none), every pair
of a line once (the two-point fluxes are symmetric):

Volume kernel (flux differencing, eq. entropy.cons.flux.dev, per stage):
  pairs per element and stage  d n^(d-1) n(n-1)/2   (n = N+1)
  Euler, d dimensions, M = d+2 variables, per pair flux:
    EC (Ranocha): both logarithmic means 35 (one reciprocal for the two),
      averages and the flux 6d+10, accumulation into the two nodes
      (2 D_pq, 2 D_qp and an FMA per variable and node) 2+4M    -> 10d+55
    KEP (Kennedy-Gruber): averages of v, p, rho, e and the flux 4d+11,
      accumulation 2+4M                                          -> 8d+21
    central: two physical fluxes 2(2d+4), their mean 2M,
      accumulation 2+4M                                          -> 10d+22
  GLM-MHD (M = 9), per pair flux:
    EC: averages of v, B, psi 14, both logarithmic means 35, p~ 5, the
      averaged squares and products 14, mass and momentum 12, induction and
      GLM 8, energy 24, accumulation 2+4M                        -> 150
    central: two physical fluxes 2x40, their mean 2M, accumulation 2+4M -> 136
  per node and stage: pair data (Euler 3d+5, GLM-MHD 39), stage combination
  and R-bar 6M, residual scaling dM, the end-point fluxes and face sums of
  every line 36d/n (Euler) or 200d/n (GLM-MHD), and for GLM-MHD the
  non-conservative term B(u_p) (D g)_p per direction d(4n+20).
  In 2D Euler with the EC flux at N = 3 this gives 75 flops per pair and 61
  per node and stage: 1,144 flops per DOF-update.

Face / update kernel (eq. numflux.cons, eq. crkfr.non.cons.final), bytes per
DOF-update: u^n read and u^{n+1} written (FP64, 8M each), R-bar read (M in
the path's arithmetic R), and the element's own face records, 2d faces x
(NP/n) face nodes x C components x R per element, C = 2M+1 (GLM-MHD 4M+1);
the neighbour's copy of a record is the same data, served by L2.
"""


def stages(N):
    return {1: 2, 2: 3, 3: 4, 4: 6, 5: 7}[N]


def nvars(mesh):
    return mesh["dim"] + 2 if mesh.get("eq", "euler") == "euler" else 9


def flops_per_pair(mesh):
    d, M = mesh["dim"], nvars(mesh)
    vol = mesh.get("vol", "ec")
    if mesh.get("eq", "euler") == "euler":
        return {"ec": 10 * d + 55, "kep": 8 * d + 21, "central": 10 * d + 22}[vol]
    return {"ec": 150, "central": 136}[vol]


def flops_per_node_stage(mesh):
    d, M, n = mesh["dim"], nvars(mesh), mesh["N"] + 1
    if mesh.get("eq", "euler") == "euler":
        return (3 * d + 5) + 6 * M + d * M + 36.0 * d / n
    return 39 + 6 * M + d * M + 200.0 * d / n + d * (4 * n + 20)


def volume_flops(mesh, n_stages=None):
    """Counted flops of one step's volume kernel (n_stages: stages per step,
    default the degree's tableau; 1 for a single-stage RKFR volume launch)."""
    d, N = mesh["dim"], mesh["N"]
    n = N + 1
    E = 1
    for k in range(d):
        E *= mesh["cells"][k]
    s = stages(N) if n_stages is None else n_stages
    pairs = E * s * d * n ** (d - 1) * (n * (n - 1) // 2)
    nodes = E * n ** d
    return pairs * flops_per_pair(mesh) + nodes * s * flops_per_node_stage(mesh)


def face_bytes(mesh, real_bytes):
    """Algorithmic bytes of one face / update launch (see above)."""
    d, N, M = mesh["dim"], mesh["N"], nvars(mesh)
    n = N + 1
    E = 1
    for k in range(d):
        E *= mesh["cells"][k]
    C = 4 * M + 1 if mesh.get("eq", "euler") != "euler" else 2 * M + 1
    nodes = E * n ** d
    per_node = 8 * M + real_bytes * M + 8 * M + 2.0 * d * C * real_bytes / n
    return nodes * per_node

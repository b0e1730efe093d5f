"""Comparison helpers shared by the GPU parity tests.

check_close: relative L2 over the whole block and, per variable, the largest
nodal difference against that variable's largest magnitude (at least a tenth
of the largest magnitude of any variable, so that a field that starts at zero
and stays at round-off level -- the GLM field psi on div-free data, a velocity
component of the Taylor-Green vortex -- is measured against the flow's
scale).  A single wrong face node on a small mesh moves the nodal maximum by
the size of its error even where the L2 norm over all nodes hides it.

check_increment: the same two measures on the increments u^{n+1} - u^n of a
step, which a one-step comparison of the states alone dilutes by ||u|| /
||du|| (about 1e3 at the CFL numbers used).
"""
import numpy as np


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def check_close(G, O, tol, what=""):
    assert np.all(np.isfinite(G)), what
    rel = rel_l2(G, O)
    assert rel <= tol, (what, "rel L2", rel)
    floor = 0.1 * np.max(np.abs(O))
    for v in range(O.shape[0]):
        scale = max(np.max(np.abs(O[v])), floor)
        err = np.max(np.abs(G[v] - O[v])) / scale
        assert err <= tol, (what, "var", v, "nodal max", err)


def check_increment(G, O, U0, tol, what=""):
    check_close(G - U0, O - U0, tol, what + " increment")

"""Writes gll_closed_form.txt: the Gauss-Lobatto-Legendre nodes and weights
of degree N = 1..5 on [0, 1] from their definition, in exact arithmetic
(sympy): the nodes are -1, 1 and the roots of P_N'(x); the weights are
2 / (N (N + 1) P_N(x_i)^2); both mapped from [-1, 1] to [0, 1].  Neither the
oracle nor the CUDA path is involved.  Run from the repository root:

    python tests/golden/make_gll_closed_form.py
"""
import os

import sympy as sp


def gll(N):
    x = sp.symbols("x")
    P = sp.legendre(N, x)
    inner = sp.solve(sp.diff(P, x), x)
    nodes = sorted([sp.Integer(-1), sp.Integer(1)] + [sp.nsimplify(r) for r in inner], key=lambda r: float(r))
    weights = [sp.Rational(2, N * (N + 1)) / P.subs(x, r) ** 2 for r in nodes]
    return [(r + 1) / 2 for r in nodes], [w / 2 for w in weights]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gll_closed_form.txt")
    with open(out, "w") as f:
        f.write("# Gauss-Lobatto-Legendre rule on [0,1]: N, i, node x_i, weight w_i (exact values to 20 digits)\n")
        f.write("# nodes: 0, 1 and the roots of P_N' mapped from [-1,1]; weights 1/(N(N+1) P_N(x_i)^2)\n")
        for N in range(1, 6):
            xs, ws = gll(N)
            for i, (xi, wi) in enumerate(zip(xs, ws)):
                f.write("%d %d %s %s\n" % (N, i, sp.N(sp.simplify(xi), 20), sp.N(sp.simplify(wi), 20)))
    print(out)


if __name__ == "__main__":
    main()

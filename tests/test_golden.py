"""The oracle's reference element against the stored closed-form GLL rule
(tests/golden/gll_closed_form.txt, the solution points of Sec. 2.1): an
independent check of the oracle's node and weight computation, which the other
pins compare with a numerical root finder.  CPU only."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gll_closed_form.txt")


def _load():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            N, i, x, w = line.split()
            rows.setdefault(int(N), []).append((int(i), float(x), float(w)))
    return rows


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_gll_rule_matches_closed_form(orc, N):
    rows = sorted(_load()[N])
    assert [r[0] for r in rows] == list(range(N + 1))
    xi, w, D, dgL, dgR = orc.tables(N)
    np.testing.assert_allclose(xi, [r[1] for r in rows], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [r[2] for r in rows], rtol=1e-15, atol=1e-16)

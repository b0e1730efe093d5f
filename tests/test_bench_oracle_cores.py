"""The all-cores oracle timing of bench.py: worker processes (spawned) each run
the unchanged oracle's restricted step on a contiguous range of elements; the
result must equal the serial oracle step bit for bit."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

from paper_2604_02125_gb300 import inputs  # noqa: E402


def test_partitioned_oracle_steps_equal_serial_steps(orc):
    mesh, U = inputs.shear_layer_2d(cells=(6, 5), N=3)
    par, seconds = bench.oracle_parallel_steps(mesh, U, 2, workers=3)
    ser, _ = orc.run(mesh, U, 2)
    assert seconds > 0
    np.testing.assert_array_equal(par, ser)

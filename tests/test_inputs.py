"""The seeded synthetic inputs (CPU): layout, determinism, the stated initial
data, and the sizes of the workloads."""
import numpy as np

from paper_2604_02125_gb300 import inputs


def test_shear_layer_layout_values_and_seed():
    mesh, U = inputs.shear_layer_2d(cells=(4, 3), N=2)
    assert U.shape == (4, 12, 9) and U.dtype == np.float64
    mesh2, U2 = inputs.shear_layer_2d(cells=(4, 3), N=2)
    np.testing.assert_array_equal(U, U2)                       # seeded
    _, U3 = inputs.shear_layer_2d(cells=(4, 3), N=2, seed=7)
    assert not np.array_equal(U[2], U3[2]) and np.array_equal(U[0], U3[0])   # noise only on v_y
    x, y = inputs.node_coords(mesh)
    # node i fastest within an element, elements x fastest, GLL points inside each element
    xi = inputs.gll_points01(2)
    np.testing.assert_allclose(x[0, :3], -1.0 + 0.5 * xi, atol=1e-15)
    np.testing.assert_allclose(x[1, :3], -0.5 + 0.5 * xi, atol=1e-15)
    B = np.tanh(15 * y + 7.5) - np.tanh(15 * y - 7.5)
    rho = 0.5 + 0.75 * B
    np.testing.assert_allclose(U[0], rho, rtol=1e-15)
    np.testing.assert_allclose(U[1] / U[0], 0.5 * (B - 1), atol=1e-15)
    vy = U[2] / U[0]
    assert np.max(np.abs(vy - 0.1 * np.sin(np.pi * x))) < 6e-3          # 1e-3 N(0,1) noise
    p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
    np.testing.assert_allclose(p, 1.0, rtol=1e-13)


def test_workload_sizes():
    mesh, U = inputs.shear_layer_2d()
    assert U.shape == (4, 65536, 16)
    specs = inputs.batched_2d_specs()
    assert len(specs) == 512 and {s["N"] for s in specs} == {2, 3, 4, 5}
    assert all(16 <= s["side"] <= 128 for s in specs)
    nodes = sum(s["side"] ** 2 * (s["N"] + 1) ** 2 for s in specs)
    assert nodes == 71936205
    assert specs == inputs.batched_2d_specs()


def test_mhd_cleaning_speed_bounds_the_fast_speed(orc):
    mesh, U = inputs.mhd_vortex_2d(cells=(6, 5), N=3)
    fast = max(orc.wave_speed(dict(mesh, c_h=0.0), d, U[:, e, p])
               for d in range(2) for e in range(U.shape[1]) for p in range(U.shape[2]))
    assert mesh["c_h"] >= fast

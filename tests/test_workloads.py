"""Input generators: the counter-based generator and the workload shapes."""
import numpy as np

from paper_2503_04428_gb300 import workloads as wl


def test_splitmix64_published_sequence():
    # first outputs of SplitMix64 from state 0 (Steele, Lea & Flood 2014;
    # the reference C code of Vigna)
    z = wl.splitmix64(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform01_range_and_mean():
    u = wl.uniform01(1, 100000)
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005


def test_tube_workload_shape_and_no_vacuum():
    lengths = wl.tube_lengths(4096, 2)
    assert lengths.min() >= 256 and lengths.max() <= 8192
    assert abs(lengths.sum() / 1.73e7 - 1) < 0.03
    WL, WR = wl.tube_states(4096, 2)
    g = 5.0 / 3.0
    cL = np.sqrt(g * WL[:, 2] / WL[:, 0])
    cR = np.sqrt(g * WR[:, 2] / WR[:, 0])
    assert np.allclose(cL * cR, g)  # normalisation c_L c_R = gamma
    assert np.all(2 * (cL + cR) / (g - 1) > WR[:, 1] - WL[:, 1])  # never vacuum
    r_rho = WL[:, 0] / WR[:, 0]
    assert r_rho.min() >= 1e-3 * 0.999 and r_rho.max() <= 1e3 * 1.001


def test_small_cases_are_physical():
    for case in (wl.sod(50), wl.rt2d(16, 48), wl.sedov3d(8), wl.wedge(32, 8, 8), wl.kh2d(8, 16),
                 wl.smooth_random(3, [5, 4, 3], 3), wl.liska_wendroff(8), wl.sedov1d_spherical(20)):
        U = case["U"]
        dim = case["dim"]
        rho = U[0]
        ke = 0.5 * sum(U[1 + d] ** 2 for d in range(dim)) / rho
        p = (case["gamma"] - 1) * (U[1 + dim] - ke)
        assert np.all(rho > 0) and np.all(p > 0), case["name"]
        assert U.shape == (2 + dim + case["n_scalars"], case["n"][2], case["n"][1], case["n"][0])

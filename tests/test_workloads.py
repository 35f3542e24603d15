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


def test_rt_single_mode_input():
    """App. C.2 initial state: densities 1 and 2, the scalar in [0, 1], P > 0,
    hydrostatic balance dP/dz = rho g wherever rho is flat, and the interface
    (scalar 1/2) at h0 cos(kappa x)."""
    case = wl.rt2d_single_mode(64, 256)
    U = case["U"][:, 0]  # (nv, nz, nx)
    rho, p = U[0], 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
    f = U[4] / rho
    assert rho.min() >= 1.0 - 1e-15 and rho.max() <= 2.0 + 1e-15
    assert f.min() >= 0.0 and f.max() <= 1.0 and p.min() > 0.0
    zc = 0.5 * (case["faces"][1][1:] + case["faces"][1][:-1])
    dz = zc[1] - zc[0]
    xc = 0.5 * (case["faces"][0][1:] + case["faces"][0][:-1])
    h = 0.01 * np.cos(4 * np.pi * xc)
    far = np.abs(zc[:, None] - h[None, :]) > 0.1
    both = far[1:] & far[:-1]
    dpdz = np.diff(p, axis=0) / dz
    assert np.max(np.abs(dpdz - (-0.5) * rho[1:])[both]) < 1e-11
    # the scalar crosses 1/2 between the two cells around z = h(x)
    for i in range(0, 64, 8):
        k = np.searchsorted(zc, h[i])
        assert f[k - 1, i] < 0.5 + 1e-12 and f[k, i] > 0.5 - 1e-12

"""Host-side helpers of bench.py's roller fingering report (Sec. IV, Eq. charac_time), on the CPU:
the front's band power read in cycles per micrometre (an FFT of the binned positions) equals the
exact sum over spheres and modes; both readings are periodic in y with the strip's length; the
half-maximum time interpolates between samples."""
import math

import numpy as np

import bench


def _front(N=3000, seed=0):
    rng = np.random.default_rng(seed)
    p = np.zeros((N, 3))
    p[:, 0] = rng.uniform(0.0, 60.0, N)
    p[:, 1] = rng.uniform(0.0, bench.FING_LY, N)
    p[:, 1] += 25.0 * np.sin(2.0 * math.pi * 60.0 * p[:, 1] / bench.FING_LY)  # a modulation inside the band
    p[:, 2] = 1.5
    return p


def test_cycles_band_power_equals_exact_sum():
    p = _front()
    y = p[np.argsort(p[:, 0])[int(0.3 * len(p)):], 1]
    L_um = bench.FING_LY * bench.FING_A_M * 1e6
    n = np.arange(1, 1 << 16)
    modes = n[(n / L_um >= bench.FING_KMIN_UM) & (n / L_um <= bench.FING_KMAX_UM)]
    assert modes[0] == 7 and modes[-1] == 838
    exact = float(np.sum(np.abs(np.exp(-2j * math.pi * np.outer(modes, y) / bench.FING_LY).sum(axis=1)) ** 2))
    assert abs(bench.front_band_power_cycles(p) / exact - 1.0) <= 1e-3


def test_band_powers_periodic_in_y():
    p = _front(seed=1)
    q = p.copy()
    q[:, 1] += bench.FING_LY
    assert math.isclose(bench.front_band_power(q), bench.front_band_power(p), rel_tol=1e-6)
    assert math.isclose(bench.front_band_power_cycles(q), bench.front_band_power_cycles(p), rel_tol=1e-6)


def test_half_time_interpolates():
    t = [0.0, 1.0, 2.0, 3.0]
    assert bench._half_time(t, [0.0, 2.0, 6.0, 10.0]) == 1.75  # half of 10 between 2 (t=1) and 6 (t=2)
    assert bench._half_time(t, [8.0, 9.0, 10.0, 7.0]) == 0.0


def test_workload_defaults():
    """Each workload gets its own suspension size unless --N is given (the accuracy comparison runs the
    FP64 oracle step by step, which at the monolayer's 65536 spheres would take hours), and the RFD
    length follows the pair precision (Sec. II.A's delta ~ eps^(1/3) a)."""
    r = bench.resolve_defaults
    assert r(bench.parse([])).N == 65536
    assert r(bench.parse(["--workload", "accuracy"])).N == 4096
    assert r(bench.parse(["--workload", "fingering"])).N == 32768
    assert r(bench.parse(["--workload", "accuracy", "--N", "1024"])).N == 1024
    assert r(bench.parse(["--impl", "reference"])).N == 65536
    assert r(bench.parse([])).delta == 5e-3
    assert r(bench.parse(["--precision", "fp64"])).delta == 1e-6
    assert r(bench.parse(["--delta", "1e-4"])).delta == 1e-4

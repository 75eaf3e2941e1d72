"""Host-side helpers of the Sec. IV.A checks, against closed forms (CPU)."""
import math

import numpy as np

from paper_1609_08146_gb300 import numerical_checks as nc


def test_cube_spacing_and_extent():
    pts, h = nc.cube(12.5, 0.4)
    n = round(len(pts) ** (1 / 3))
    assert n ** 3 == len(pts) and abs(h - 25.0 / (n - 1)) < 1e-15
    assert np.allclose(pts.min(axis=0), -12.5) and np.allclose(pts.max(axis=0), 12.5)
    x = np.unique(pts[:, 0])
    assert np.allclose(np.diff(x), h)


def test_mean_cell_length_matches_the_cell_sum():
    # <A>_N = dtheta dr^2 / 2 * sum_{n=0}^{N} (2n + 1) / N over the N annuli
    r_max, N, Nt = 1000.0, 37, 53
    dr, dth = r_max / N, 2 * math.pi / Nt
    A = dth * dr * dr / 2 * sum(2 * n + 1 for n in range(N + 1)) / N
    assert abs(nc.mean_cell_length(r_max, N, Nt) - math.sqrt(A)) < 1e-12 * math.sqrt(A)


def test_incident_power_closed_forms():
    cfg = nc.config(n_nodes=16)
    w0, r_max = cfg["beam"]["w0"], cfg["mirror"]["r_max"]
    X2 = 2 * (r_max / w0) ** 2
    # radial: |A|^2 = (rho / w0)^2 e^{-2 rho^2 / w0^2}, clipped at r_max
    rad = math.pi * w0 ** 2 / 4 * (1 - (1 + X2) * math.exp(-X2))
    assert abs(nc.incident_power(cfg) - rad) < 1e-6 * rad
    cfg["beam"]["pol"] = "linear"
    lin = math.pi * w0 ** 2 / 2 * (1 - math.exp(-X2))
    assert abs(nc.incident_power(cfg) - lin) < 1e-6 * lin


def test_pulse_energy_parseval():
    # over one period T = 2 pi / dk the cross terms of different k_n vanish:
    # INT e^2 dt = 2 T dk^2 sum |a_n|^2, up to the k_n + k_m terms (relative
    # size about 1 / (k_0 T))
    om = np.linspace(0.9, 1.1, 41)
    rng = np.random.default_rng(5)
    a = rng.normal(size=41) * np.exp(-((om - 1) / 0.05) ** 2) + 0j
    k = 2 * math.pi * om
    dk = k[1] - k[0]
    T = 2 * math.pi / dk
    ref = 2 * T * dk * dk * np.sum(np.abs(a) ** 2)
    assert abs(nc.pulse_energy_1d(a, om) - ref) < 2e-3 * ref

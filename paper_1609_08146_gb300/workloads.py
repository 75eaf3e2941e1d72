"""Seeded synthetic workloads shaped like the paper's (Sec. IV, Table 1).

Inputs only: mirror and beam parameters, frequency grids, observation
points, time samples.  Nothing here evaluates any part of the method, so
both the CUDA path and the CPU oracle consume these definitions.  Lengths in
lambda0, omega in units of omega0, time in lambda0/c (2.6685 fs at 800 nm).

  small     f = 20, NA = 1 (r_max = 2f), x-polarised Gaussian w0 = 20,
            64 Gauss-Legendre x 64 trapezoid nodes + rim, 32 x 32 focal-plane
            grid over +-2, one frequency (omega0).
  broadband f = 62,500 (5 cm at 800 nm), r_max = 2f, w0 = 0.6 f, 512 x 512
            nodes, Gaussian 10 fs pulse (intensity FWHM 3.7474), 256 uniform
            omegas over [0.5, 1.5], 64 x 64 focal-plane grid over +-3 plus 64
            points on the axis over +-5, 512 time samples t = (m - 256)/8.
  sweep     the broadband pulse with f in {1e2, 1e3, 1e4, 1e5}, r_max = 2f,
            w0 = 0.6 f, N x N nodes, 4096 uniform random points in [-2, 2]^3.
  full_range_requests  uneven requests, each its own mirror and beam, 128^2 to
            1024^2 nodes, 1k to 262k points, 1 to 512 omegas.
"""
from __future__ import annotations

import numpy as np

FS_PER_UNIT_800NM = 800e-9 / 299792458.0 * 1e15  # lambda0 / c at 800 nm, in fs


def focal_plane_grid(n: int, half: float) -> np.ndarray:
    """Inclusive n x n grid over [-half, half]^2 at z = 0, [n*n, 3]."""
    x = np.linspace(-half, half, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)


def axis_points(n: int, half: float) -> np.ndarray:
    z = np.linspace(-half, half, n)
    return np.stack([np.zeros(n), np.zeros(n), z], axis=1)


def random_cube(n: int, half: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-half, half, size=(n, 3))


def uniform_omegas(n: int, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    return np.array([1.0]) if n == 1 else np.linspace(lo, hi, n)


def small():
    return dict(
        name="mono f=20 lambda, NA=1, 64x64 nodes, 32x32 focal-plane points",
        mirror=dict(f=20.0, r_min=0.0, r_max=40.0, n_r=64, n_theta=64, rim=True),
        beam=dict(profile="gauss", w0=20.0, pol="linear", pol_angle=0.0, zernike=[]),
        spectrum=dict(kind="mono"),
        omegas=np.array([1.0]),
        points=focal_plane_grid(32, 2.0),
    )


def broadband(n_nodes: int = 512, n_omega: int = 256):
    pts = np.vstack([focal_plane_grid(64, 3.0), axis_points(64, 5.0)])
    f = 62500.0
    return dict(
        name="broadband 10 fs, f=62500 lambda0, NA=1, %dx%d nodes, 4160 points, %d omegas"
        % (n_nodes, n_nodes, n_omega),
        mirror=dict(f=f, r_min=0.0, r_max=2 * f, n_r=n_nodes, n_theta=n_nodes, rim=True),
        beam=dict(profile="gauss", w0=0.6 * f, pol="linear", pol_angle=0.0, zernike=[]),
        spectrum=dict(kind="gauss_time", fwhm_t=10.0 / FS_PER_UNIT_800NM, lambda_c=1.0, energy=1.0),
        omegas=uniform_omegas(n_omega),
        points=pts,
        times=(np.arange(512) - 256) / 8.0,
    )


def sweep(f: float, n_nodes: int, n_points: int = 4096, seed: int = 1609):
    return dict(
        name="sweep f=%g, %dx%d nodes, %d random points" % (f, n_nodes, n_nodes, n_points),
        mirror=dict(f=f, r_min=0.0, r_max=2 * f, n_r=n_nodes, n_theta=n_nodes, rim=True),
        beam=dict(profile="gauss", w0=0.6 * f, pol="linear", pol_angle=0.0, zernike=[]),
        spectrum=dict(kind="gauss_time", fwhm_t=10.0 / FS_PER_UNIT_800NM, lambda_c=1.0, energy=1.0),
        omegas=uniform_omegas(256),
        points=random_cube(n_points, 2.0, seed),
    )


def uneven_requests(n: int, seed: int, max_nodes: int = 256, max_points: int = 8192,
                    max_omega: int = 256, n_configs: int = 8):
    """Seeded uneven requests shaped like a serving mix: a pool of n_configs
    mirror/beam configurations (f log-uniform in [1e3, 1e5], r_max = 2f,
    w0 = 0.6 f, N x N nodes with N in {64, 128, ..., max_nodes}, Gaussian or
    super-Gaussian N=4, x-linear / radial / azimuthal, Zernike j = 2..15 with
    N(0, 0.1) waves); each request picks a configuration, a log-uniform point
    count in [256, max_points] (uniform in the +-2 cube) and a log-uniform
    omega count in [1, max_omega] on [0.5, 1.5] (omega0 alone if 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [s for s in (64, 128, 256, 512, 1024) if s <= max_nodes]
    configs = []
    for _ in range(n_configs):
        f = float(10 ** rng.uniform(3, 5))
        N = int(rng.choice(sizes))
        configs.append(dict(
            mirror=dict(f=f, r_min=0.0, r_max=2 * f, n_r=N, n_theta=N, rim=True),
            beam=dict(profile=str(rng.choice(["gauss", "supergauss"])), sg_order=4, w0=0.6 * f,
                      pol=str(rng.choice(["linear", "radial", "azimuthal"])), pol_angle=0.0,
                      zernike=list(rng.normal(0.0, 0.1, size=14))),
            spectrum=dict(kind="gauss_time", fwhm_t=10.0 / FS_PER_UNIT_800NM, lambda_c=1.0,
                          energy=1.0)))
    reqs = []
    for _ in range(n):
        c = int(rng.integers(n_configs))
        npts = int(round(10 ** rng.uniform(np.log10(256), np.log10(max_points))))
        nom = int(round(10 ** rng.uniform(0, np.log10(max_omega))))
        reqs.append(dict(config=c, omegas=uniform_omegas(nom),
                         points=rng.uniform(-2.0, 2.0, size=(npts, 3))))
    return configs, reqs


def full_range_requests(n: int, seed: int):
    """Seeded uneven requests at the batched workload's full ranges, each with
    its own mirror and beam: f log-uniform in [1e3, 1e5], r_max = 2f,
    w0 = 0.6 f, N x N nodes with N = 2^U{7..10} (128^2 to 1024^2), Gaussian
    or super-Gaussian N=4 beam, x-linear / radial / azimuthal polarisation,
    Zernike j = 2..15 with N(0, 0.1) waves, the broadband 10 fs pulse; a
    log-uniform point count in [1024, 262144] uniform in the +-2 cube and a
    log-uniform omega count in [1, 512] on [0.5, 1.5] (omega0 alone if 1).
    Returns (configs, reqs) with request i using configs[i]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    configs, reqs = [], []
    for i in range(n):
        f = float(10 ** rng.uniform(3, 5))
        N = int(2 ** rng.integers(7, 11))
        profile = str(rng.choice(["gauss", "supergauss"]))
        pol = str(rng.choice(["linear", "radial", "azimuthal"]))
        zern = list(rng.normal(0.0, 0.1, size=14))
        npts = int(round(10 ** rng.uniform(np.log10(1024), np.log10(262144))))
        nom = int(round(10 ** rng.uniform(0, np.log10(512))))
        configs.append(dict(
            mirror=dict(f=f, r_min=0.0, r_max=2 * f, n_r=N, n_theta=N, rim=True),
            beam=dict(profile=profile, sg_order=4, w0=0.6 * f, pol=pol, pol_angle=0.0, zernike=zern),
            spectrum=dict(kind="gauss_time", fwhm_t=10.0 / FS_PER_UNIT_800NM, lambda_c=1.0, energy=1.0)))
        reqs.append(dict(config=i, omegas=uniform_omegas(nom),
                         points=rng.uniform(-2.0, 2.0, size=(npts, 3))))
    return configs, reqs


def oracle_args(w):
    """The same workload in the oracle's parameter format."""
    m = dict(w["mirror"])
    m["rim"] = 1 if m.get("rim", True) else 0
    b = dict(w["beam"])
    b["r_norm"] = m["r_max"]
    return m, b

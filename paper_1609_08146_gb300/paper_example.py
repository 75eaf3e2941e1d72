"""The paper's worked example (Sec. IV.B, Table 1) on the GPU path.

A linearly (x) polarised Gaussian beam, w0 = 0.100 m, on a parabola with
f = 0.0675 m and r_max = 0.125 m (NA about 1), with the super-Gaussian power
spectrum of Eq. 27 (centre 820 nm, width parameter 70 nm, order 3) sampled at
100 frequencies and normalised to E_tot = 150 J.  The spectral field on a
focal-plane grid comes from sc_eval, the time-domain field from
sc_time_domain; this module only post-processes the results (peak time,
intensity map, cuts) on the host.

Units: lambda0 = 820 nm, c = 1.  SI scale (the paper's Eq. 16 leaves it open,
reading R12): the real field E(t) of the incident pulse carries the energy
E_tot = eps0 c * SS |A|^2 dA * INT e(t)^2 dt over the whole transverse plane,
e(t) = 2 Re sum_n a_n exp(-i k_n t) dk, which fixes one factor s (V/m per
field unit); the intensity is I_E = 1/2 c eps0 (s E)^2 (Sec. IV.B, Eq. 28).
"""
from __future__ import annotations

import math

import numpy as np

from .workloads import focal_plane_grid

LAMBDA0_M = 820e-9
C_M_S = 299792458.0
EPS0 = 8.8541878128e-12
FS_PER_UNIT = LAMBDA0_M / C_M_S * 1e15


def config(n_nodes: int = 512, n_grid: int = 65, half: float = 2.0, n_omega: int = 100,
           r_max_m: float = 0.125):
    """Table 1's configuration; r_max_m = 0.0551 gives the NA 0.7 mirror of
    the comparison in Sec. IV.B (r / (f + r^2 / 4f) = 0.7)."""
    f = 0.0675 / LAMBDA0_M
    dl = 70.0 / 820.0
    lam_lo, lam_hi = 1.0 - 1.6 * dl, 1.0 + 1.6 * dl
    omegas = np.linspace(1.0 / lam_hi, 1.0 / lam_lo, n_omega)  # uniform in k
    return dict(
        name="paper example (Table 1): f=0.0675 m, r_max=0.125 m, w0=0.100 m, 820 nm, 150 J",
        mirror=dict(f=f, r_min=0.0, r_max=r_max_m / LAMBDA0_M, n_r=n_nodes, n_theta=n_nodes, rim=True),
        beam=dict(profile="gauss", w0=0.100 / LAMBDA0_M, pol="linear", pol_angle=0.0, zernike=[]),
        spectrum=dict(kind="supergauss_lambda", lambda_c=1.0, dlambda=dl, sg_n=3, energy=1.0),
        omegas=omegas,
        points=focal_plane_grid(n_grid, half),
        times=np.linspace(-8.0, 8.0, 321),
        energy_J=150.0,
    )


def si_scale(amp, omegas, beam_w0):
    """V/m per field unit for the configured pulse energy of 1 J (scale by
    sqrt(E_tot) for another energy): E_tot = eps0 * lambda0^3 * P_A * INT e^2 dt
    with P_A = pi w0^2 / 2 (lambda0^2) and t in lambda0 / c."""
    k = 2 * math.pi * np.asarray(omegas)
    dk = k[1] - k[0]
    period = 2 * math.pi / dk
    t = np.linspace(0.0, period, 200001)[:-1]
    e = 2 * np.real(np.exp(-1j * np.outer(t, k)) @ np.asarray(amp)) * dk
    int_e2 = np.sum(e * e) * (t[1] - t[0])
    P_A = math.pi * beam_w0 ** 2 / 2
    return math.sqrt(1.0 / (EPS0 * LAMBDA0_M ** 3 * P_A * int_e2))


def fwhm_1d(x, y):
    """Full width at half maximum of a sampled peak (linear interpolation)."""
    y = np.asarray(y, float)
    i = int(np.argmax(y))
    h = y[i] / 2

    def cross(rng):
        prev = i
        for j in rng:
            if y[j] < h:
                return x[j] + (h - y[j]) * (x[prev] - x[j]) / (y[prev] - y[j])
            prev = j
        return x[rng[-1]] if len(rng) else x[i]

    return cross(range(i + 1, len(y))) - cross(range(i - 1, -1, -1))


def analyse(Et, Bt, times, n_grid, half, scale_vm, energy_J, E_focus=None, omegas=None):
    """Focal-plane quantities of Sec. IV.B from E(t), B(t) [n_t, n_grid^2, 3]."""
    x = np.linspace(-half, half, n_grid)
    I_E = 0.5 * C_M_S * EPS0 * (scale_vm ** 2 * energy_J) * np.sum(Et ** 2, axis=2)  # W/m^2
    m, p = np.unravel_index(np.argmax(I_E), I_E.shape)
    c = n_grid // 2
    Imap = I_E[m].reshape(n_grid, n_grid)
    i0, j0 = np.unravel_index(np.argmax(Imap), Imap.shape)
    wx = fwhm_1d(x, Imap[:, j0])
    wy = fwhm_1d(x, Imap[i0, :])
    a, b = max(wx, wy), min(wx, wy)
    # component magnitudes over the whole pulse: the longitudinal fields are
    # in quadrature with E_x, so at the instant of peak intensity they sit
    # near a zero crossing
    Ex = np.abs(Et[:, :, 0]).max()
    Bz = np.abs(Bt[:, :, 2]).max()
    Ez = np.abs(Et[:, :, 2]).max()
    focus = int(np.argmin(np.sum((focal_plane_grid(n_grid, half)[:, :2]) ** 2, axis=1)))
    out = dict(
        peak_intensity_W_cm2=float(I_E.max() * 1e-4),
        peak_time_fs=float(times[m] * FS_PER_UNIT),
        fwhm_x_um=float(wx * LAMBDA0_M * 1e6),
        fwhm_y_um=float(wy * LAMBDA0_M * 1e6),
        eccentricity=float(math.sqrt(max(0.0, 1 - (b / a) ** 2))),
        Bz_over_Ex=float(Bz / Ex),
        Ez_over_Ex=float(Ez / Ex),
        focus_index=focus,
        center_index=c,
    )
    if E_focus is not None:
        # duration of the main pulse at the focus: FWHM of the envelope of E_x,
        # |sum_n E_n exp(-i k_n t)| (the analytic signal of Eq. 13)
        k = 2 * math.pi * np.asarray(omegas)
        t = np.linspace(times[0], times[-1], 4001)
        env = np.abs(np.exp(-1j * np.outer(t, k)) @ np.asarray(E_focus))
        out["pulse_fwhm_fs"] = float(fwhm_1d(t, env) * FS_PER_UNIT)
    return out


def run(ctx, n_nodes: int = 512, n_grid: int = 65, half: float = 2.0, r_max_m: float = 0.125):
    """Evaluate the example on the GPU; returns (metrics, E, B, Et, Bt, cfg)."""
    import torch

    cfg = config(n_nodes, n_grid, half, r_max_m=r_max_m)
    mc, b = cfg["mirror"], cfg["beam"]
    m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"])
    inc = ctx.incident(profile=b["profile"], w0=b["w0"], pol=b["pol"], spectrum=cfg["spectrum"])
    om = cfg["omegas"]
    P = torch.tensor(cfg["points"], device="cuda")
    E, B = ctx.eval(m, inc, om, P)
    Et, Bt = ctx.time_domain(E, B, om, cfg["times"])
    torch.cuda.synchronize()
    amp = ctx.spectrum(inc, om)
    s = si_scale(amp, om, b["w0"])
    focus = int(np.argmin(np.sum(cfg["points"][:, :2] ** 2, axis=1)))
    metrics = analyse(Et.cpu().numpy().astype(np.float64), Bt.cpu().numpy().astype(np.float64),
                      cfg["times"], n_grid, half, s, cfg["energy_J"],
                      E_focus=E[:, focus, 0].cpu().numpy().astype(np.complex128), omegas=om)
    return metrics, E, B, Et, Bt, cfg


def maxwell_time_residual(ctx, cfg, p0, t0, h=0.01, dt=0.01):
    """Eq. 26b at one space-time point: central differences of the GPU's
    time-domain fields, e_t = 2|curl E + dB/dt| / (|curl E| + |dB/dt|) +
    2|curl B - dE/dt| / (|curl B| + |dE/dt|) (the paper normalises by maxima
    over the region; here by the values at the point)."""
    import torch

    mc, b = cfg["mirror"], cfg["beam"]
    m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"])
    inc = ctx.incident(profile=b["profile"], w0=b["w0"], pol=b["pol"], spectrum=cfg["spectrum"])
    p0 = np.asarray(p0, float)
    pts = [p0]
    for ax in range(3):
        for sgn in (-1.0, 1.0):
            q = p0.copy()
            q[ax] += sgn * h
            pts.append(q)
    P = torch.tensor(np.array(pts), device="cuda")
    om = cfg["omegas"]
    E, B = ctx.eval(m, inc, om, P)
    Et, Bt = ctx.time_domain(E, B, om, np.array([t0 - dt, t0, t0 + dt]))
    torch.cuda.synchronize()
    Et = Et.cpu().numpy().astype(np.float64)
    Bt = Bt.cpu().numpy().astype(np.float64)

    def d(F, ax, c):  # spatial derivative at t0
        return (F[1, 2 + 2 * ax, c] - F[1, 1 + 2 * ax, c]) / (2 * h)

    def curl(F):
        return np.array([d(F, 1, 2) - d(F, 2, 1), d(F, 2, 0) - d(F, 0, 2), d(F, 0, 1) - d(F, 1, 0)])

    dEdt = (Et[2, 0] - Et[0, 0]) / (2 * dt)
    dBdt = (Bt[2, 0] - Bt[0, 0]) / (2 * dt)
    cE, cB = curl(Et), curl(Bt)
    far = 2 * np.linalg.norm(cE + dBdt) / (np.linalg.norm(cE) + np.linalg.norm(dBdt))
    amp = 2 * np.linalg.norm(cB - dEdt) / (np.linalg.norm(cB) + np.linalg.norm(dEdt))
    return float(far), float(amp)

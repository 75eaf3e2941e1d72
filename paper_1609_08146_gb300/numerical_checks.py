"""The numerical checks of Sec. IV.A on the GPU path.

A radially polarised Gaussian beam with the super-Gaussian power spectrum of
Table 1 (820 nm, 70 nm, order 3: an 18 fs pulse) on an NA = 1 paraboloid
(r_max = 2f, f = 0.0675 m).  The text asks for a beam that the rim does not
clip and prints no waist; w0 = 0.05 m leaves 7e-6 of the power outside
r_max.  Three checks, each computed from sc_eval / sc_time_domain results
with host post-processing only:

  convergence   e_rel = max|F_N - F_Nmax| / max|F_Nmax| per field component
                over a focal region, against the average polar cell length
                sqrt(<A>_N), <A>_N = dtheta dr^2 (N+1)^2 / (2N) (Sec. IV.A);
  energy        the energy 1/2 INT (E^2 + B^2) dV of the time-domain field in
                a cube around the focus, against the energy of the incident
                pulse P_A INT e(t)^2 dt (Eqs. 15-17 in the units of Eq. 13:
                c = 1, so a travelling wave carries E^2 per unit area and
                time);
  maxwell_freq  e_f of Eq. 26a on a cube of points: curls by central
                differences, normalised by the maxima over the region.

Lengths in lambda0 = 820 nm, omega in omega0, t in lambda0 / c.
"""
from __future__ import annotations

import math

import numpy as np

from . import paper_example as pe

F_M = 0.0675
W0_M = 0.05


def config(n_nodes: int = 384, n_omega: int = 100, w0_m: float = W0_M, pol: str = "radial",
           order: int = 0):
    """Sec. IV.A's set-up: Table 1's spectrum and focal length, NA = 1.  order 1
    adds the first-order longitudinal terms to the collimated beam."""
    base = pe.config(n_nodes=n_nodes, n_grid=3, half=1.0, n_omega=n_omega)
    f = F_M / pe.LAMBDA0_M
    base["name"] = ("Sec. IV.A checks: %s Gaussian w0=%g m, f=0.0675 m, NA=1, %dx%d nodes"
                    % (pol, w0_m, n_nodes, n_nodes))
    base["mirror"] = dict(f=f, r_min=0.0, r_max=2 * f, n_r=n_nodes, n_theta=n_nodes, rim=True)
    base["beam"] = dict(profile="gauss", w0=w0_m / pe.LAMBDA0_M, pol=pol, pol_angle=0.0, zernike=[],
                        order=order)
    return base


def cube(half: float, h: float):
    """Uniform grid over [-half, half]^3 (inclusive) with the spacing nearest
    to h that divides the edge: (points [n^3, 3], actual spacing)."""
    n = int(round(2 * half / h)) + 1
    x = np.linspace(-half, half, n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1), 2 * half / (n - 1)


def _handles(ctx, cfg, n_r=None, n_theta=None):
    mc, b = cfg["mirror"], cfg["beam"]
    m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], n_r or mc["n_r"], n_theta or mc["n_theta"])
    inc = ctx.incident(profile=b["profile"], w0=b["w0"], pol=b["pol"], spectrum=cfg["spectrum"],
                       order=b.get("order", 0))
    return m, inc


def mean_cell_length(r_max: float, n_r: int, n_theta: int) -> float:
    """sqrt(<A>_N) of Sec. IV.A with dr = r_max / N and dtheta = 2 pi / n_theta."""
    dr, dth = r_max / n_r, 2 * math.pi / n_theta
    return math.sqrt(dth * dr * dr / 2 * (n_r + 1) ** 2 / n_r)


COMPONENTS = ("E_x", "E_y", "E_z", "B_x", "B_y", "B_z")


def convergence(ctx, cfg, sizes, points, omega_index=None, precision: str = "fp64"):
    """e_rel per component for each N x N mesh in sizes against the largest.

    Returns a list of dicts {n, cell_lambda, e_rel: {component: value}} in the
    order of sizes (the last one, the reference, has zeros).  Components that
    vanish identically by symmetry (reference maximum below 1e-9 of the
    largest component, e.g. B_z of a radial beam) are left out.  The field is
    taken at one frequency (the centre sample by default), as the
    convergence is per spectral component; the FP64 path shows it below the
    FP32 path's rounding floor."""
    import torch

    om = cfg["omegas"]
    j = len(om) // 2 if omega_index is None else omega_index
    P = torch.tensor(points, device="cuda")
    fields = []
    for n in sizes:
        m, inc = _handles(ctx, cfg, n, n)
        E, B = ctx.eval(m, inc, om[j:j + 1], P, precision=precision)
        torch.cuda.synchronize()
        F = np.concatenate([E[0].cpu().numpy(), B[0].cpu().numpy()], axis=1).astype(np.complex128)
        fields.append(F)
    ref = fields[-1]
    peak = np.max(np.abs(ref), axis=0)
    keep = [c for c in range(6) if peak[c] > 1e-9 * peak.max()]
    out = []
    r_max = cfg["mirror"]["r_max"]
    for n, F in zip(sizes, fields):
        e = {COMPONENTS[c]: float(np.max(np.abs(F[:, c] - ref[:, c])) / peak[c]) for c in keep}
        out.append(dict(n=n, cell_lambda=mean_cell_length(r_max, n, n), e_rel=e))
    return out


def incident_power(cfg, n_quad: int = 20000) -> float:
    """P_A = INT_{rho < r_max} |A p^|^2 dA of the configured beam (midpoint rule)."""
    b, mc = cfg["beam"], cfg["mirror"]
    w0 = b["w0"]
    rho = (np.arange(n_quad) + 0.5) * (mc["r_max"] / n_quad)
    if b["profile"] == "gauss":
        a2 = np.exp(-2 * (rho / w0) ** 2)
    elif b["profile"] == "supergauss":
        a2 = np.exp(-2 * (rho / w0) ** (2 * b.get("sg_order", 4)))
    else:
        a2 = (rho <= w0).astype(float)
    if b["pol"] in ("radial", "azimuthal"):
        a2 = a2 * (rho / w0) ** 2
    return float(np.sum(a2 * 2 * math.pi * rho) * (mc["r_max"] / n_quad))


def pulse_energy_1d(amp, omegas, n_t: int = 200001) -> float:
    """INT e(t)^2 dt over one period of the grid, e(t) = 2 Re sum a_n e^{-i k_n t} dk."""
    k = 2 * math.pi * np.asarray(omegas)
    dk = k[1] - k[0]
    period = 2 * math.pi / dk
    t = np.linspace(-period / 2, period / 2, n_t)[:-1]
    e = 2 * np.real(np.exp(-1j * np.outer(t, k)) @ np.asarray(amp)) * dk
    return float(np.sum(e * e) * (t[1] - t[0]))


def energy(ctx, cfg, half: float, h: float, times=(0.0,), chunk: int = 1 << 18):
    """U(t) = 1/2 SUM (E^2 + B^2) h^3 over the cube [-half, half]^3 at each time
    (h: the grid's actual spacing), divided by the incident energy P_A INT e^2 dt.  Points are evaluated in
    chunks of `chunk` so the spectra stay within a few GB."""
    import torch

    pts, h = cube(half, h)
    m, inc = _handles(ctx, cfg)
    om = cfg["omegas"]
    U = np.zeros(len(times))
    for s in range(0, len(pts), chunk):
        P = torch.tensor(pts[s:s + chunk], device="cuda")
        E, B = ctx.eval(m, inc, om, P)
        Et, Bt = ctx.time_domain(E, B, om, np.asarray(times, dtype=np.float64))
        torch.cuda.synchronize()
        e2 = (Et.double() ** 2).sum(dim=(1, 2)) + (Bt.double() ** 2).sum(dim=(1, 2))
        U += 0.5 * e2.cpu().numpy() * h ** 3
        del E, B, Et, Bt
    amp = ctx.spectrum(inc, om)
    U_inc = incident_power(cfg) * pulse_energy_1d(amp, om)
    return dict(n_points=len(pts), half=half, h=h, times=list(times),
                ratio=[float(u / U_inc) for u in U], U_inc=U_inc)


def maxwell_freq(ctx, cfg, half: float = 1.0, n: int = 9, dx: float = 0.01, omega_indices=None,
                 precision: str = "fp32"):
    """max over the points of |e_f| (Eq. 26a) on an n^3 grid over [-half, half]^3,
    for each selected frequency.  Derivatives by central differences of step
    dx (truncation error about (k dx)^2 / 6); the maxima in the denominators
    run over the grid, as in the paper."""
    import torch

    om = cfg["omegas"]
    sel = [len(om) // 2] if omega_indices is None else list(omega_indices)
    base, _ = cube(half, 2 * half / (n - 1))
    offs = [np.zeros(3)]
    for ax in range(3):
        for sg in (-1.0, 1.0):
            d = np.zeros(3)
            d[ax] = sg * dx
            offs.append(d)
    pts = np.concatenate([base + d for d in offs], axis=0)
    m, inc = _handles(ctx, cfg)
    out = []
    for j in sel:
        E, B = ctx.eval(m, inc, om[j:j + 1], torch.tensor(pts, device="cuda"), precision=precision)
        torch.cuda.synchronize()
        E = E[0].cpu().numpy().astype(np.complex128).reshape(7, -1, 3)
        B = B[0].cpu().numpy().astype(np.complex128).reshape(7, -1, 3)
        k = 2 * math.pi * om[j]

        def curl(F):
            def d(ax, c):
                return (F[2 + 2 * ax, :, c] - F[1 + 2 * ax, :, c]) / (2 * dx)
            return np.stack([d(1, 2) - d(2, 1), d(2, 0) - d(0, 2), d(0, 1) - d(1, 0)], axis=1)

        cE, cB = curl(E), curl(B)
        ikB, ikE = 1j * k * B[0], 1j * k * E[0]
        nrm = lambda v: np.sqrt(np.sum(np.abs(v) ** 2, axis=1))  # noqa: E731
        ef = (2 * nrm(cE - ikB) / (nrm(cE).max() + nrm(ikB).max())
              + 2 * nrm(cB + ikE) / (nrm(cB).max() + nrm(ikE).max()))
        out.append(dict(omega=float(om[j]), max_e_f=float(ef.max())))
    return out

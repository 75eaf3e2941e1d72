"""Seeded random configurations against the FP64 oracle on both GPU paths.

Each case draws a mirror (paraboloid or ellipsoid, inner rim or none, rim term
on or off, ragged node counts), a beam (every collimated profile and
polarisation with Zernike aberrations and order 0 or 1, a Laguerre-Gauss mode,
or the ellipsoid's dipole), an omega count from 1 to 300 (every kernel class)
and points around the focus.  Both paths are judged by the gate metric of
reading R11.  The FP32 path must meet the parity gate, 1e-5.  The FP64 path
must agree to 2e-10: its phases round to about 2e-16 k R (k R up to about
3e3 here), and a component built from terms that cancel (the radial beam's B
near the axis) magnifies that by up to a few hundred.  Fitted envelopes are
held to 5e-8, five times the fit tolerance, since the truncated Chebyshev terms
cancel in the same way.  A beam that misses the mirror (a top-hat inside an
inner rim) must give exactly zero on both paths.
"""
import numpy as np
import pytest

import oracle
from paper_1609_08146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_08146_gb300 as sc  # noqa: E402

N_CASES = 40


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    yield c
    c.close()


def _gate(F, R):
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def _draw(seed):
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    n_r, n_t = int(rng.integers(5, 70)), int(rng.integers(3, 70))
    rim = bool(rng.integers(0, 2))
    n_om = int(rng.choice([1, 2, 3, 5, 8, 9, 13, 16, 17, 23, 28, 32, 33, 47, 64, 100, 129, 256, 300]))
    lo = float(rng.uniform(0.6, 0.95))
    om = np.array([1.0]) if n_om == 1 else np.linspace(lo, lo + float(rng.uniform(0.05, 0.6)), n_om)
    kind = rng.choice(["collimated", "collimated", "collimated", "lg", "dipole"])
    if kind == "dipole":
        e = float(rng.uniform(3.0, 10.0))
        c = e + float(rng.uniform(5.0, 12.0))
        a = np.sqrt(c * c - e * e)
        mirror = dict(surface="ellipsoid", c=c, e=e, r_min=0.0, r_max=float(rng.uniform(0.3, 0.9)) * a,
                      n_r=n_r, n_theta=n_t, rim=int(rim))
        p = rng.normal(size=3)
        beam = dict(profile="dipole", dipole=tuple(p / np.linalg.norm(p)))
    else:
        f = float(10 ** rng.uniform(0.9, 2.0))
        r_max = f * float(rng.uniform(0.8, 2.0))
        r_min = float(rng.choice([0.0, 0.0, rng.uniform(0.05, 0.3) * r_max]))
        mirror = dict(f=f, r_min=r_min, r_max=r_max, n_r=n_r, n_theta=n_t, rim=int(rim))
        pol = str(rng.choice(["linear", "radial", "azimuthal"]))
        w0 = float(rng.uniform(0.2, 0.7)) * r_max
        if kind == "lg":
            beam = dict(profile="laguerre_gauss", pol=pol, w0=w0, lg_p=int(rng.integers(0, 3)),
                        lg_l=int(rng.integers(-2, 3)) if pol == "linear" else 1,
                        z_waist=-float(rng.uniform(0.5, 3.0)) * f, pol_angle=float(rng.uniform(0, 3)))
        else:
            prof = str(rng.choice(["gauss", "supergauss", "tophat"]))
            beam = dict(profile=prof, sg_order=int(rng.integers(2, 6)), pol=pol, w0=w0,
                        pol_angle=float(rng.uniform(0, 3)),
                        zernike=list(rng.normal(0, 0.1, size=int(rng.integers(0, 8)))),
                        order=int(rng.integers(0, 2)) if prof != "tophat" else 0)
    pts = np.vstack([np.zeros((1, 3)), rng.uniform(-1.5, 1.5, size=(int(rng.integers(2, 12)), 3))])
    return mirror, beam, om, pts


@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_configuration(ctx, seed):
    mirror, beam, om, pts = _draw(seed)
    if mirror.get("surface") == "ellipsoid":
        m = ctx.ellipsoid(mirror["c"], mirror["e"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"],
                          rim=bool(mirror["rim"]))
        ob = oracle.dipole_beam(mirror, beam["dipole"])
    else:
        m = ctx.mirror(mirror["f"], mirror["r_min"], mirror["r_max"], mirror["n_r"], mirror["n_theta"],
                       rim=bool(mirror["rim"]))
        ob = dict(beam, r_norm=mirror["r_max"])
    kw = {k: v for k, v in beam.items() if k in ("profile", "w0", "sg_order", "pol", "pol_angle", "zernike",
                                                 "order", "lg_p", "lg_l", "z_waist", "dipole")}
    if beam["profile"] == "laguerre_gauss":
        kw["omega_band"] = (float(om[0]), float(om[-1]) + 1e-9)
        if om.size == 1:
            kw["omega_band"] = (0.99, 1.01)
    inc = ctx.incident(spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)), **kw)
    E0, B0 = oracle.field(mirror, ob, om, pts)
    fitted = beam["profile"] == "laguerre_gauss"
    for prec, tol in (("fp32", 1e-5), ("fp64", 5e-8 if fitted else 2e-10)):
        E, B = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"), precision=prec)
        torch.cuda.synchronize()
        E, B = E.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128)
        if not np.any(E0) and not np.any(B0):
            assert not np.any(E) and not np.any(B), (seed, prec)
            continue
        e = max(_gate(E, E0), _gate(B, B0))
        assert e <= tol, (seed, prec, e, mirror, beam, om.size)

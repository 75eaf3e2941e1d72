"""The first correction beyond physical optics (Sec. II: the MFIE's
Liouville-Neumann series) on the GPU against the FP64 oracle on the same
rules: the polar rule about every surface node for dJ, and the mirror's own
nodes for the field of dJ.

The correction itself (MFIE order 1 minus order 0) is compared as well, so a
mistake in it cannot hide under the tolerance of the whole field: on these
mirrors of tens of wavelengths it is about 1e-3 of the field.
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

N_RHO, N_PHI = 48, 96


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    c.set_option(sc.SC_OPT_MFIE_RHO, N_RHO)
    c.set_option(sc.SC_OPT_MFIE_PHI, N_PHI)
    yield c
    c.close()


def rel_err(F, R):
    F = np.asarray(F, dtype=np.complex128)
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def gpu(ctx, mirror, beam, om, pts, order, precision):
    if "c" in mirror:
        m = ctx.ellipsoid(mirror["c"], mirror["e"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    else:
        m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    inc = ctx.incident(profile=beam["profile"], w0=beam["w0"], sg_order=beam.get("sg_order", 4),
                       pol=beam.get("pol", "linear"), pol_angle=beam.get("pol_angle", 0.0),
                       zernike=beam.get("zernike", []),
                       spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
    ctx.set_option(sc.SC_OPT_MFIE_ORDER, order)
    try:
        E, B = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"), precision=precision)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(sc.SC_OPT_MFIE_ORDER, 0)
    return E.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128)


def oracle_fields(mirror, beam, om, pts):
    mo = dict(mirror, rim=1)
    if "c" in mirror:
        mo["surface"] = "ellipsoid"
    bo = dict(beam, r_norm=mirror["r_max"])
    E0, B0 = oracle.field(mo, bo, om, pts)
    E1, B1 = oracle.field_mfie(mo, bo, om, pts, N_RHO, N_PHI)
    return E0, B0, E1, B1


CASES = [
    (dict(f=5.0, r_max=10.0, n_r=24, n_theta=24),
     dict(profile="gauss", w0=5.0, pol="linear", pol_angle=0.3, zernike=[0.05, -0.1, 0.08, 0.02])),
    (dict(f=4.0, r_max=8.0, n_r=20, n_theta=28),
     dict(profile="supergauss", sg_order=4, w0=5.0, pol="radial")),
    (dict(f=6.0, r_max=9.0, n_r=22, n_theta=24),
     dict(profile="gauss", w0=4.0, pol="azimuthal", zernike=[0.0, 0.1, 0.0, -0.05, 0.07])),
    (dict(c=14.0, e=6.0, r_max=11.0, n_r=20, n_theta=24),
     dict(profile="gauss", w0=6.0, pol="linear")),
]


@pytest.mark.parametrize("mirror,beam", CASES)
def test_mfie_correction_matches_oracle(ctx, mirror, beam):
    om = np.linspace(0.9, 1.1, 3)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(7, 1.0, seed=17)])
    E0o, B0o, E1o, B1o = oracle_fields(mirror, beam, om, pts)
    dEo, dBo = E1o - E0o, B1o - B0o
    # the correction is visible: 1e-4 to 1e-2 of the field here
    assert np.max(np.abs(dEo)) > 1e-5 * np.max(np.abs(E0o))
    # FP64: the whole field and the correction alone
    E1, B1 = gpu(ctx, mirror, beam, om, pts, 1, "fp64")
    E0, B0 = gpu(ctx, mirror, beam, om, pts, 0, "fp64")
    assert max(rel_err(E1, E1o), rel_err(B1, B1o)) <= 1e-11
    scale_d = max(np.max(np.abs(dEo)), np.max(np.abs(dBo)))
    assert np.max(np.abs((E1 - E0) - dEo)) <= 1e-9 * scale_d
    assert np.max(np.abs((B1 - B0) - dBo)) <= 1e-9 * scale_d
    if "c" in mirror:
        return  # a collimated beam on an ellipsoid is FP64-only
    # FP32 path plus the FP64 correction: the R11 gate, and the correction to FP32 rounding
    E1f, B1f = gpu(ctx, mirror, beam, om, pts, 1, "fp32")
    assert max(rel_err(E1f, E1o), rel_err(B1f, B1o)) <= 1e-5
    E0f, _ = gpu(ctx, mirror, beam, om, pts, 0, "fp32")
    assert np.max(np.abs((E1f - E0f) - dEo)) <= 1e-3 * np.max(np.abs(dEo)) + 2e-6 * np.max(np.abs(E0o))


def test_mfie_time_domain_and_host_buffers(ctx):
    mirror, beam = CASES[0]
    om = np.linspace(0.9, 1.1, 5)
    t = np.linspace(-3.0, 3.0, 9)
    pts = wl.random_cube(5, 0.8, seed=3)
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    inc = ctx.incident(profile=beam["profile"], w0=beam["w0"], pol=beam["pol"], pol_angle=beam["pol_angle"],
                       zernike=beam["zernike"], spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
    ctx.set_option(sc.SC_OPT_MFIE_ORDER, 1)
    try:
        Eh, Bh = ctx.eval(m, inc, om, pts, precision="fp64")  # host buffers
        Et, Bt = ctx.eval_time_domain(m, inc, om, pts, t, precision="fp64")
    finally:
        ctx.set_option(sc.SC_OPT_MFIE_ORDER, 0)
    _, _, E1o, B1o = oracle_fields(mirror, beam, om, pts)
    assert max(rel_err(Eh, E1o), rel_err(Bh, B1o)) <= 1e-11
    Rt = oracle.time_domain(E1o, om, t)
    assert np.max(np.abs(np.asarray(Et) - Rt)) <= 2e-6 * np.max(np.abs(Rt))


def test_mfie_refusals(ctx):
    om = np.array([1.0])
    ann = ctx.mirror(5.0, 1.0, 10.0, 12, 12)
    inc = ctx.incident(profile="gauss", w0=5.0)
    lg = ctx.incident(profile="laguerre_gauss", w0=5.0, omega_band=(0.9, 1.1),
                      spectrum=dict(kind="sampled", omega=om, amp=np.ones(1)))
    disk = ctx.mirror(5.0, 0.0, 10.0, 12, 12)
    P = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    ctx.set_option(sc.SC_OPT_MFIE_ORDER, 1)
    try:
        for m, i in ((ann, inc), (disk, lg)):
            with pytest.raises(sc.ScError) as e:
                ctx.eval(m, i, om, P, precision="fp64")
            assert e.value.status == sc.SC_ERR_INVALID
        with pytest.raises(sc.ScError) as e:
            ctx.eval_batch([(disk, inc, om, P)])
        assert e.value.status == sc.SC_ERR_INVALID
    finally:
        ctx.set_option(sc.SC_OPT_MFIE_ORDER, 0)
    with pytest.raises(sc.ScError):
        ctx.set_option(sc.SC_OPT_MFIE_ORDER, 2)

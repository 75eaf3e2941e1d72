"""Frequency-dependent incident envelopes on the GPU paths against the FP64
oracle: Laguerre-Gauss beams with a finite Rayleigh range (width, wavefront
curvature and Gouy phase depend on k) and a caller's envelope with a
spatio-temporal coupling (a spatially chirped beam).  The library expands
the envelope in Chebyshev polynomials of k over the beam's band, one node
table per real or imaginary part of each kept term; the oracle samples the
exact envelope at every (frequency, node).
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

MIRROR = dict(f=20.0, r_max=40.0, n_r=96, n_theta=96)
BAND = (0.8, 1.2)


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    yield c
    c.close()


def _rel(F, R):
    return float(np.max(np.abs(F - R)) / np.max(np.abs(R)))


def _gate(F, R):
    """The parity gate's metric (reading R11): per omega, the RMS over points of
    |F - R| over the peak |R|, maximised over omega.  The FP32 path's error is
    largest at coherent points such as the focus, where it grows with the
    length of the FP32 runs between compensated folds (2048 nodes by default;
    SC_OPT_FLUSH_NODES shortens them)."""
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def _chirp(xyz, k, w0=7.0, beta=4.0, k0=2 * np.pi):
    """Spatially chirped x-polarised Gaussian: its centre moves with k."""
    x, y = xyz[:, 0], xyz[:, 1]
    e = np.zeros((len(xyz), 2), dtype=np.complex128)
    e[:, 0] = np.exp(-((x - beta * (k - k0)) ** 2 + y ** 2) / w0 ** 2) * np.exp(0.3j * (k - k0) * x)
    return e


def _gpu(ctx, beam, om, pts, precision, mirror=MIRROR):
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    inc = ctx.incident(omega_band=BAND, spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)), **beam)
    E, B, st = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"), precision=precision, stats=True)
    torch.cuda.synchronize()
    return E.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128), st


LG_BEAMS = [
    dict(profile="laguerre_gauss", pol="linear", w0=6.0, lg_p=0, lg_l=0, z_waist=-30.0),
    dict(profile="laguerre_gauss", pol="linear", w0=6.0, lg_p=1, lg_l=2, z_waist=-35.0, pol_angle=0.4),
    dict(profile="laguerre_gauss", pol="radial", w0=7.0, lg_p=0, lg_l=1, z_waist=-28.0),
    dict(profile="laguerre_gauss", pol="azimuthal", w0=7.0, lg_p=1, lg_l=1, z_waist=-40.0),
]


@pytest.mark.parametrize("beam", LG_BEAMS)
def test_laguerre_gauss_parity(ctx, beam):
    om = np.linspace(BAND[0], BAND[1], 11)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(9, 1.5, 5)])
    ob = dict(beam, r_norm=MIRROR["r_max"])
    E0, B0 = oracle.field(dict(MIRROR, rim=1), ob, om, pts)
    for prec, err, tol in (("fp32", _gate, 1e-5), ("fp64", _rel, 2e-8)):
        E, B, st = _gpu(ctx, beam, om, pts, prec)
        assert max(err(E, E0), err(B, B0)) <= tol, (prec, st)
        assert 2 <= st["tables"] <= 40
    # the finite Rayleigh range is visible: the collimated beam differs
    col = dict(profile="gauss", pol=beam["pol"], w0=beam["w0"], pol_angle=beam.get("pol_angle", 0.0),
               r_norm=MIRROR["r_max"])
    if beam["lg_p"] == 0 and (beam["pol"] != "linear" or beam["lg_l"] == 0):
        Ec, _ = oracle.field(dict(MIRROR, rim=1), col, om, pts)
        assert _rel(Ec, E0) > 1e-3


def test_spatially_chirped_envelope_parity(ctx):
    om = np.linspace(BAND[0], BAND[1], 9)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(7, 1.5, 6)])
    cb = oracle.envelope_callback(_chirp)
    E0, B0 = oracle.field(dict(MIRROR, rim=1), dict(profile="envelope", w0=7.0, env_fn=cb, r_norm=40.0), om, pts)
    for prec, err, tol in (("fp32", _gate, 1e-5), ("fp64", _rel, 2e-8)):
        E, B, st = _gpu(ctx, dict(profile="envelope", w0=7.0, envelope=_chirp), om, pts, prec)
        assert max(err(E, E0), err(B, B0)) <= tol, (prec, st)


def _tilt(xyz, k, alpha=3.0):
    """Pulse-front tilt: a Gaussian whose phase alpha k x is linear in k."""
    x, y = xyz[:, 0], xyz[:, 1]
    e = np.zeros((len(xyz), 2), dtype=np.complex128)
    e[:, 1] = np.exp(-(x * x + y * y) / 49.0) * np.exp(1j * alpha * k * x)
    return e


def test_pulse_front_tilt_is_one_table(ctx):
    """A phase linear in k goes into the nodes' optical path before the fit,
    so a tilt of hundreds of radians across the band costs one table."""
    om = np.linspace(BAND[0], BAND[1], 7)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(5, 1.5, 8)])
    cb = oracle.envelope_callback(_tilt)
    E0, B0 = oracle.field(dict(MIRROR, rim=1), dict(profile="envelope", w0=7.0, env_fn=cb, r_norm=40.0), om, pts)
    for prec, err, tol in (("fp32", _gate, 1e-5), ("fp64", _rel, 2e-8)):
        E, B, st = _gpu(ctx, dict(profile="envelope", w0=7.0, envelope=_tilt), om, pts, prec)
        assert st["tables"] == 1
        assert max(err(E, E0), err(B, B0)) <= tol, (prec, st)


def test_envelope_beams_alone_equal_mixed(ctx):
    reqs = []
    m = ctx.mirror(MIRROR["f"], 0.0, MIRROR["r_max"], 48, 48)
    for i, beam in enumerate([LG_BEAMS[0], dict(profile="gauss", w0=8.0), dict(profile="envelope", w0=7.0,
                                                                                envelope=_chirp)]):
        om = np.linspace(0.85, 1.15, (5, 17, 40)[i])
        inc = ctx.incident(omega_band=BAND, spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)), **beam)
        reqs.append((m, inc, om, torch.tensor(wl.random_cube(20 + 7 * i, 1.5, 30 + i), device="cuda")))
    alone = [ctx.eval(*r) for r in reqs]
    torch.cuda.synchronize()
    mixed = ctx.eval_batch(reqs)
    torch.cuda.synchronize()
    for (Ea, Ba), (Em, Bm) in zip(alone, mixed):
        assert torch.equal(Ea, Em) and torch.equal(Ba, Bm)


def test_envelope_errors(ctx):
    m = ctx.mirror(MIRROR["f"], 0.0, MIRROR["r_max"], 24, 24)
    pts = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    inc = ctx.incident(omega_band=BAND, **LG_BEAMS[0])
    with pytest.raises(RuntimeError):  # outside the band of the fit
        ctx.eval(m, inc, [1.3], pts)
    # a phase quadratic in k (the linear part is factored out before the fit)
    rough = lambda xyz, k: np.column_stack([np.exp(3j * k * k * xyz[:, 0]), 0 * xyz[:, 0]])  # noqa: E731
    inc = ctx.incident(omega_band=BAND, profile="envelope", w0=5.0, envelope=rough,
                       spectrum=dict(kind="mono"))
    with pytest.raises(RuntimeError):  # needs far more than 20 terms in k
        ctx.eval(m, inc, [1.0], pts)

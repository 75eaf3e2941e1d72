"""First-order incident beam (beam order 1, the O(eps) longitudinal terms of
the collimated beam) on the GPU paths against the FP64 oracle.

The correction itself (order 1 minus order 0) is compared as well, so that a
mistake in it cannot hide under the tolerance of the whole field: it is
O(eps) of the field, eps = lambda / (pi w0), and the cases use eps of a few
per cent.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1609_08146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_08146_gb300 as sc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    yield c
    c.close()


BEAMS = [
    dict(profile="gauss", pol="linear", w0=8.0, pol_angle=0.3),
    dict(profile="supergauss", sg_order=4, pol="radial", w0=10.0),
    dict(profile="gauss", pol="azimuthal", w0=8.0, zernike=[0.1, -0.05, 0.2, 0.03, 0.07]),
    dict(profile="gauss", pol="linear", w0=6.0, zernike=[0.0, 0.3, 0.0, 0.0, -0.2, 0.1]),
]


def _run(ctx, mirror, beam, order, om, pts, precision):
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    inc = ctx.incident(profile=beam["profile"], w0=beam["w0"], sg_order=beam.get("sg_order", 4),
                       pol=beam["pol"], pol_angle=beam.get("pol_angle", 0.0),
                       zernike=beam.get("zernike", []), order=order,
                       spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
    E, B = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"), precision=precision)
    torch.cuda.synchronize()
    return E.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128)


def _oracle(mirror, beam, order, om, pts):
    mo = dict(mirror, rim=1)
    bo = dict(beam, order=order, r_norm=mirror["r_max"])
    return oracle.field(mo, bo, om, pts)


def _rel(F, R):
    return float(np.max(np.abs(F - R)) / np.max(np.abs(R)))


def _check_correction(D, Do, Fo, tol_d, tol_f):
    """GPU correction D against the oracle's Do; where the correction vanishes
    (B of a radial beam: div b_perp = 0), D must vanish to the field tolerance."""
    if np.max(np.abs(Do)) > 1e-6 * np.max(np.abs(Fo)):
        return _rel(D, Do) <= tol_d
    return np.max(np.abs(D)) <= 2 * tol_f * np.max(np.abs(Fo))


@pytest.mark.parametrize("beam", BEAMS)
def test_first_order_parity_and_correction(ctx, beam):
    mirror = dict(f=20.0, r_max=40.0, n_r=96, n_theta=96)
    om = np.linspace(0.8, 1.2, 11)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(9, 1.5, 77)])
    E1o, B1o = _oracle(mirror, beam, 1, om, pts)
    E0o, B0o = _oracle(mirror, beam, 0, om, pts)
    dEo, dBo = E1o - E0o, B1o - B0o
    # the correction is visible at this eps (about 1% of the field)
    assert np.max(np.abs(dEo)) > 1e-3 * np.max(np.abs(E0o))
    for prec, tol_f, tol_d in (("fp32", 1e-5, 3e-3), ("fp64", 1e-11, 1e-8)):
        E1, B1 = _run(ctx, mirror, beam, 1, om, pts, prec)
        E0, B0 = _run(ctx, mirror, beam, 0, om, pts, prec)
        assert max(_rel(E1, E1o), _rel(B1, B1o)) <= tol_f, prec
        assert _check_correction(E1 - E0, dEo, E0o, tol_d, tol_f), prec
        assert _check_correction(B1 - B0, dBo, B0o, tol_d, tol_f), prec


def test_first_order_alone_equals_mixed_batch(ctx):
    mirror = dict(f=1e3, r_max=2e3, n_r=48, n_theta=40)
    reqs = []
    for i, order in enumerate((0, 1, 1, 0)):
        m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
        om = wl.uniform_omegas((3, 37, 8, 100)[i])
        inc = ctx.incident(profile="gauss", w0=100.0 * (i + 1), pol="radial", order=order,
                           spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
        reqs.append((m, inc, om, torch.tensor(wl.random_cube(50 + 13 * i, 2.0, i), device="cuda")))
    alone = [ctx.eval(*r) for r in reqs]
    torch.cuda.synchronize()
    mixed = ctx.eval_batch(reqs)
    torch.cuda.synchronize()
    for (Ea, Ba), (Em, Bm) in zip(alone, mixed):
        assert torch.equal(Ea, Em) and torch.equal(Ba, Bm)


def test_static_path_rejects_first_order(ctx):
    m = ctx.mirror(20.0, 0.0, 40.0, 16, 16)
    inc = ctx.incident(profile="gauss", w0=8.0, order=1)
    pts = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    ctx.eval(m, inc, [1.0], pts)  # makes the tables resident
    E = torch.empty((1, 4, 3), dtype=torch.complex64, device="cuda")
    amp = torch.tensor([1.0, 0.0], dtype=torch.float64, device="cuda")
    st = ctx._lib.sc_eval_fp32_static(ctx._h, m._h, inc._h, 1.0, 0.0, 1,
                                      ctypes.cast(amp.data_ptr(), sc._DP),
                                      sc._VP(pts.data_ptr()), 4, sc._VP(E.data_ptr()), None)
    assert st == sc.SC_ERR_INVALID
    assert b"node tables" in ctx._lib.sc_last_error(ctx._h)

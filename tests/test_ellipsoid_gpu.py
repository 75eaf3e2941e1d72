"""Beyond paraboloids (reading R16): an ellipsoidal mirror with an electric
dipole at its upper focus F1, on the GPU paths against the FP64 oracle.

Every ray from F1 reaches the lower focus F2 (the origin) over the same
path, so the FP32 path's compensated phase R - |P| stays exact; the dipole's
k-dependence is three node tables with weights (ik)^m.  A collimated beam on
the ellipsoid does not focus on the origin (the case where the paraboloid's
phase cancellation fails): the FP64 path takes it, the FP32 path refuses it.
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


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    yield c
    c.close()


def _gate(F, R):
    """Reading R11: per omega the RMS over points of |F - R| over the peak |R|."""
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def _rel(F, R):
    return float(np.max(np.abs(F - R)) / np.max(np.abs(R)))


def _run(ctx, ell, beam, om, pts, precision):
    m = ctx.ellipsoid(ell["c"], ell["e"], 0.0, ell["r_max"], ell["n_r"], ell["n_theta"])
    inc = ctx.incident(spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)), **beam)
    E, B, st = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"), precision=precision, stats=True)
    torch.cuda.synchronize()
    return E.cpu().numpy().astype(np.complex128), B.cpu().numpy().astype(np.complex128), st


ELL = dict(surface="ellipsoid", c=14.0, e=6.0, r_max=12.0, n_r=96, n_theta=96)


@pytest.mark.parametrize("p", [(1.0, 0.0, 0.0), (0.0, 0.0, 1.0), (0.3, -0.5, 0.8)])
def test_dipole_on_ellipsoid_parity(ctx, p):
    om = np.linspace(0.8, 1.2, 9)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(9, 1.5, 12)])
    E0, B0 = oracle.field(dict(ELL, rim=1), oracle.dipole_beam(ELL, p), om, pts)
    for prec, err, tol in (("fp32", _gate, 1e-5), ("fp64", _rel, 1e-11)):
        E, B, st = _run(ctx, ELL, dict(profile="dipole", dipole=p), om, pts, prec)
        assert st["tables"] == 3
        assert max(err(E, E0), err(B, B0)) <= tol, prec


def test_large_ellipsoid_fp32_against_fp64(ctx):
    """f = c - e = 1000 lambda, F1 10^4 lambda away: the compensated FP32 phase
    holds at scale (the FP64 path is the reference)."""
    ell = dict(c=6000.0, e=5000.0, r_max=3000.0, n_r=256, n_theta=256)
    om = np.linspace(0.9, 1.1, 32)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(63, 2.0, 13)])
    beam = dict(profile="dipole", dipole=(1.0, 0.0, 0.0))
    E32, B32, _ = _run(ctx, ell, beam, om, pts, "fp32")
    E64, B64, _ = _run(ctx, ell, beam, om, pts, "fp64")
    assert max(_gate(E32, E64), _gate(B32, B64)) <= 1e-5
    # spot check of the FP64 path against the oracle
    E0, B0 = oracle.field(dict(ell, surface="ellipsoid", rim=1), oracle.dipole_beam(dict(ell), (1.0, 0.0, 0.0)),
                          om[::31], pts[:3])
    assert _rel(E64[::31, :3], E0) < 1e-10


def test_collimated_beam_on_ellipsoid_needs_fp64(ctx):
    om = np.linspace(0.9, 1.1, 5)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(5, 1.5, 14)])
    beam = dict(profile="gauss", pol="linear", w0=5.0)
    E0, B0 = oracle.field(dict(ELL, rim=1), dict(beam, r_norm=ELL["r_max"]), om, pts)
    E, B, _ = _run(ctx, ELL, beam, om, pts, "fp64")
    assert max(_rel(E, E0), _rel(B, B0)) <= 1e-11
    with pytest.raises(RuntimeError):
        _run(ctx, ELL, beam, om, pts, "fp32")


def test_dipole_needs_an_ellipsoid(ctx):
    m = ctx.mirror(8.0, 0.0, 16.0, 16, 16)
    inc = ctx.incident(profile="dipole", dipole=(1.0, 0.0, 0.0))
    with pytest.raises(RuntimeError):
        ctx.eval(m, inc, [1.0], torch.zeros((2, 3), dtype=torch.float64, device="cuda"))

"""sc_eval_time_domain: the time-domain field straight from the mirror
integrals, one chunk of omegas at a time (Sec. III.B Eq. 13 applied to the
spectra of Eq. 11).  It must equal sc_eval followed by sc_time_domain: bitwise
in one chunk, to the FP32 rounding of the chunk sums otherwise; and the
oracle's own inverse transform of its own spectra at sampled points.
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


def _setup(ctx, n_omega=37, n_pts=300):
    w = wl.sweep(2e3, 48, n_points=n_pts, seed=21)
    mc = w["mirror"]
    m = ctx.mirror(mc["f"], 0.0, mc["r_max"], mc["n_r"], mc["n_theta"])
    inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"], spectrum=w["spectrum"])
    om = np.linspace(0.7, 1.3, n_omega)
    times = np.linspace(-6.0, 6.0, 41)
    return w, m, inc, om, times


def _rel(F, R):
    F, R = np.asarray(F, dtype=np.float64), np.asarray(R, dtype=np.float64)
    return float(np.max(np.abs(F - R)) / np.max(np.abs(R)))


def test_fused_equals_eval_then_transform(ctx):
    w, m, inc, om, times = _setup(ctx)
    P = torch.tensor(w["points"], device="cuda")
    E, B = ctx.eval(m, inc, om, P)
    Et0, Bt0 = ctx.time_domain(E, B, om, times)
    torch.cuda.synchronize()
    Et0, Bt0 = Et0.cpu().numpy(), Bt0.cpu().numpy()
    # one chunk: the same spectra through the same transform, bitwise
    Et, Bt = ctx.eval_time_domain(m, inc, om, P, times)
    torch.cuda.synchronize()
    assert np.array_equal(Et.cpu().numpy(), Et0) and np.array_equal(Bt.cpu().numpy(), Bt0)
    # several chunks: FP32 sums of partial sums
    for chunk in (1, 7, 36):
        Et, Bt, st = ctx.eval_time_domain(m, inc, om, P, times, omega_chunk=chunk, stats=True)
        torch.cuda.synchronize()
        assert max(_rel(Et.cpu().numpy(), Et0), _rel(Bt.cpu().numpy(), Bt0)) < 2e-6, chunk
        assert st["evals"] == P.shape[0] * 48 * 48 * om.size


def test_fused_host_buffers_fp64_and_no_B(ctx):
    w, m, inc, om, times = _setup(ctx, n_omega=12, n_pts=40)
    P = torch.tensor(w["points"], device="cuda")
    Etd, Btd = ctx.eval_time_domain(m, inc, om, P, times, omega_chunk=5)
    Eth, Bth = ctx.eval_time_domain(m, inc, om, w["points"], times, omega_chunk=5)
    torch.cuda.synchronize()
    assert np.array_equal(Etd.cpu().numpy(), Eth) and np.array_equal(Btd.cpu().numpy(), Bth)
    Et_only, none = ctx.eval_time_domain(m, inc, om, P, times, omega_chunk=5, with_B=False)
    torch.cuda.synchronize()
    assert none is None and np.array_equal(Et_only.cpu().numpy(), Eth)
    E64, B64 = ctx.eval(m, inc, om, P, precision="fp64")
    Et64_0, _ = ctx.time_domain(E64, B64, om, times, precision="fp64")
    Et64, _ = ctx.eval_time_domain(m, inc, om, P, times, precision="fp64", omega_chunk=4)
    torch.cuda.synchronize()
    assert _rel(Et64.cpu().numpy(), Et64_0.cpu().numpy()) < 2e-6


def test_fused_matches_the_oracle_transform(ctx):
    w, m, inc, om, times = _setup(ctx, n_omega=24, n_pts=64)
    idx = np.array([0, 17, 40, 63])
    mo, bo = wl.oracle_args(w)
    amp = oracle.spectrum(w["spectrum"], om, bo)
    E0, B0 = oracle.field(mo, bo, om, w["points"][idx], amp=amp)
    Et0 = oracle.time_domain(E0, om, times)
    Et, _ = ctx.eval_time_domain(m, inc, om, torch.tensor(w["points"], device="cuda"), times, omega_chunk=5)
    torch.cuda.synchronize()
    assert _rel(Et.cpu().numpy()[:, idx], Et0) < 1e-5

"""Serving and batched evaluation of beams that need several node tables.

A first-order beam (two tables), a Laguerre-Gauss mode (a Chebyshev fit in k)
and the ellipsoid's dipole (three tables) are served next to a collimated
beam: each result is bitwise the request evaluated alone, through sc_submit
and through sc_eval_batch.  A request that cannot run fails by itself: a pair
whose wavefront does not focus on the origin is refused at submission, and an
envelope too rough to fit fails its own ticket while the others in flight
finish.
"""
import numpy as np
import pytest

from paper_1609_08146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_08146_gb300 as sc  # noqa: E402


def _sampled(om):
    return dict(kind="sampled", omega=om, amp=np.ones(om.size))


def _requests(ctx):
    reqs = []
    om = np.linspace(0.8, 1.2, 40)
    m = ctx.mirror(20.0, 0.0, 40.0, 48, 40)
    reqs.append((m, ctx.incident(profile="gauss", w0=12.0, pol="radial", order=1, spectrum=_sampled(om)),
                 om, 70, 1))
    om = np.linspace(0.9, 1.1, 12)
    reqs.append((m, ctx.incident(profile="laguerre_gauss", w0=12.0, pol="linear", lg_p=1, lg_l=2,
                                 z_waist=-30.0, omega_band=(0.9, 1.1 + 1e-9), spectrum=_sampled(om)),
                 om, 33, 2))
    om = np.linspace(0.85, 1.15, 100)
    e = ctx.ellipsoid(14.0, 6.0, 0.0, 9.0, 40, 36)
    reqs.append((e, ctx.incident(profile="dipole", dipole=(0.6, 0.0, 0.8), spectrum=_sampled(om)),
                 om, 41, 3))
    om = wl.uniform_omegas(8)
    reqs.append((m, ctx.incident(profile="gauss", w0=12.0, pol="linear", spectrum=_sampled(om)), om, 120, 4))
    return [(mm, inc, om, torch.tensor(wl.random_cube(n, 1.5, seed), device="cuda"))
            for (mm, inc, om, n, seed) in reqs]


def test_multi_table_requests_served_and_batched_bitwise():
    ctx = sc.Context(0)
    try:
        reqs = _requests(ctx)
        alone = [ctx.eval(m, inc, om, pts) for (m, inc, om, pts) in reqs]
        torch.cuda.synchronize()
        tickets = [ctx.submit(m, inc, om, pts) for (m, inc, om, pts) in reqs]
        for t in tickets:
            ctx.wait(t, 120.0)
        for t, (Ea, Ba) in zip(tickets, alone):
            E, B = ctx.fetch(t)
            assert torch.equal(E, Ea) and torch.equal(B, Ba)
            ctx.release(t)
        mixed = ctx.eval_batch(reqs)
        torch.cuda.synchronize()
        for (Ea, Ba), (Em, Bm) in zip(alone, mixed):
            assert torch.equal(Ea, Em) and torch.equal(Ba, Bm)
    finally:
        ctx.close()


def test_a_failing_request_fails_alone():
    ctx = sc.Context(0)
    try:
        reqs = _requests(ctx)
        alone = [ctx.eval(m, inc, om, pts) for (m, inc, om, pts) in reqs]
        torch.cuda.synchronize()
        # a collimated beam on the ellipsoid needs the FP64 path: refused at once
        e = reqs[2][0]
        om = wl.uniform_omegas(8)
        flat = ctx.incident(profile="gauss", w0=4.0, pol="linear", spectrum=_sampled(om))
        pts = torch.tensor(wl.random_cube(10, 1.0, 9), device="cuda")
        with pytest.raises(sc.ScError) as err:
            ctx.submit(e, flat, om, pts)
        assert err.value.status == sc.SC_ERR_INVALID
        with pytest.raises(sc.ScError) as err:
            ctx.eval_batch([reqs[3], (e, flat, om, pts)])
        assert err.value.status == sc.SC_ERR_INVALID
        # an envelope too rough for the Chebyshev fit fails its own ticket only
        band = (0.9, 1.1 + 1e-9)
        rough = ctx.incident(profile="envelope", w0=5.0, omega_band=band, spectrum=_sampled(om),
                             envelope=lambda xyz, k: np.column_stack([np.exp(3j * k * k * xyz[:, 0]),
                                                                      0 * xyz[:, 0]]))
        m = reqs[0][0]
        om_r = np.linspace(0.9, 1.1, 8)
        tickets = [ctx.submit(*reqs[0]), ctx.submit(m, rough, om_r, pts), ctx.submit(*reqs[3])]
        with pytest.raises(sc.ScError) as err:
            ctx.wait(tickets[1], 120.0)
        assert err.value.status == sc.SC_ERR_INVALID
        for t, i in ((tickets[0], 0), (tickets[2], 3)):
            ctx.wait(t, 120.0)
            E, B = ctx.fetch(t)
            assert torch.equal(E, alone[i][0]) and torch.equal(B, alone[i][1])
        for t in tickets:
            ctx.release(t)
    finally:
        ctx.close()

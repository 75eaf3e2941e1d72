"""Serving: continuous batching of submitted requests (sc_submit/poll/wait).

Requests submitted while others run are admitted as memory frees up, run in
overlapping batches on several lanes, and each result is bitwise the same as
the request evaluated alone.  Short requests pass a long one that runs in
bounded launches on a low-priority lane.  Admission respects the HBM budget,
a request that can never fit is refused, and cancellation is honoured.
"""
import time

import numpy as np
import pytest

from paper_1609_08146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_08146_gb300 as sc  # noqa: E402


def make(ctx, f, nr, nt, nom, npts, seed, pol="linear"):
    m = ctx.mirror(f, 0.0, 2 * f, nr, nt)
    om = wl.uniform_omegas(nom)
    inc = ctx.incident(profile="gauss", w0=0.6 * f, pol=pol,
                       spectrum=dict(kind="gauss_time", fwhm_t=3.7474, lambda_c=1.0))
    return m, inc, om, wl.random_cube(npts, 2.0, seed)


def test_served_results_equal_alone_and_overlap():
    ctx = sc.Context(0)
    try:
        big = make(ctx, 6.25e4, 256, 256, 256, 4160, 1)
        small = [make(ctx, 1e3 * (1 + i % 4), 32, 32, 8 + 17 * i, 50 + 40 * i, 10 + i,
                      pol=("linear", "radial", "azimuthal")[i % 3]) for i in range(8)]
        # alone first (this also fixes each shape's tuned split count)
        alone = [ctx.eval(m, inc, om, torch.tensor(p, device="cuda")) for (m, inc, om, p) in [big] + small]
        torch.cuda.synchronize()
        # the big request first, the small ones while it runs (host and device points mixed)
        tb = ctx.submit(big[0], big[1], big[2], big[3])
        ts = []
        for i, (m, inc, om, p) in enumerate(small):
            pts = torch.tensor(p, device="cuda") if i % 2 else p
            ts.append(ctx.submit(m, inc, om, pts))
        for t in [tb] + ts:
            ctx.wait(t, 120.0)
        for t, (Ea, Ba) in zip([tb] + ts, alone):
            E, B = ctx.fetch(t)
            assert torch.equal(E, Ea) and torch.equal(B, Ba)
        times = {t: ctx.ticket_times(t) for t in [tb] + ts}
        for t, (s0, s1, s2) in times.items():
            assert 0.0 <= s0 <= s1 <= s2
        # some small request started on the other lane while the big one was on the GPU
        assert any(times[t][1] < times[tb][2] for t in ts)
        for t in [tb] + ts:
            ctx.release(t)
    finally:
        ctx.close()


def test_caller_owned_outputs_and_cancel():
    ctx = sc.Context(0)
    try:
        m, inc, om, p = make(ctx, 2e3, 32, 40, 40, 300, 5)
        P = torch.tensor(p, device="cuda")
        Ea, Ba = ctx.eval(m, inc, om, P)
        E = torch.empty_like(Ea)
        B = torch.empty_like(Ba)
        t = ctx.submit(m, inc, om, P, out=(E, B))
        ctx.wait(t, 60.0)
        torch.cuda.synchronize()
        assert torch.equal(E, Ea) and torch.equal(B, Ba)
        ctx.release(t)
        # cancel: queued requests are dropped, running ones discarded
        ts = [ctx.submit(m, inc, om, p) for _ in range(6)]
        ctx.cancel(ts[-1])
        with pytest.raises(sc.ScError) as e:
            ctx.wait(ts[-1], 60.0)
        assert e.value.status == sc.SC_ERR_CANCELLED
        for t in ts[:-1]:
            ctx.wait(t, 60.0)
        for t in ts:
            ctx.release(t)
        with pytest.raises(sc.ScError) as e:
            ctx.poll(12345678)
        assert e.value.status == sc.SC_ERR_NOT_FOUND
    finally:
        ctx.close()


def test_admission_by_budget():
    # 96 MiB budget, 8 MiB workspace cap per lane: about four 6 MB requests fit
    ctx = sc.Context(0, budget_bytes=96 << 20)
    try:
        ctx.set_option(sc.SC_OPT_WORKSPACE_CAP, 8 << 20)
        m, inc, om, p = make(ctx, 1e3, 24, 24, 64, 2000, 7)
        ts = [ctx.submit(m, inc, om, p) for _ in range(12)]
        done = []
        deadline = time.time() + 120
        while len(done) < len(ts) and time.time() < deadline:
            for t in ts:
                if t not in done and ctx.poll(t):
                    done.append(t)
                    E, _ = ctx.fetch(t)
                    assert torch.isfinite(torch.view_as_real(E)).all()
                    ctx.release(t)  # frees its memory: admits the next
            time.sleep(0.002)
        assert len(done) == len(ts)
        # a request larger than the whole budget can never be admitted
        big = wl.random_cube(50000, 2.0, 9)
        with pytest.raises(sc.ScError) as e:
            ctx.submit(m, inc, np.linspace(0.5, 1.5, 256), big)
        assert e.value.status == sc.SC_ERR_BUSY
    finally:
        ctx.close()


def test_short_requests_pass_a_long_one():
    # a long request (512^2 nodes x 4160 points x 256 omegas = 2.8e11
    # evaluations, above the 1e11 bound; about 0.24 s) runs on a low-priority
    # lane in launches of about 6e10 evaluations; short requests submitted
    # after it run on the high-priority lanes between those launches and
    # finish first
    ctx = sc.Context(0)
    try:
        long_req = make(ctx, 6.25e4, 512, 512, 256, 4160, 3)
        small = [make(ctx, 1e3 * (1 + i), 64, 64, 16 + 8 * i, 500 + 100 * i, 20 + i,
                      pol=("linear", "radial", "azimuthal")[i % 3]) for i in range(4)]
        reqs = [long_req] + small
        alone = [ctx.eval(m, inc, om, torch.tensor(p, device="cuda")) for (m, inc, om, p) in reqs]
        torch.cuda.synchronize()
        for priority in (1, 0):
            ctx.set_option(sc.SC_OPT_SERVE_PRIORITY, priority)
            ts = [ctx.submit(m, inc, om, p) for (m, inc, om, p) in reqs]
            for t in ts:
                ctx.wait(t, 120.0)
            for t, (Ea, Ba) in zip(ts, alone):
                E, B = ctx.fetch(t)
                assert torch.equal(E, Ea) and torch.equal(B, Ba)
            times = [ctx.ticket_times(t) for t in ts]
            done = [x[2] for x in times]
            if priority:
                assert all(d < done[0] for d in done[1:]), times
            for t in ts:
                ctx.release(t)
        # the policy changes only while no ticket is outstanding
        t = ctx.submit(*small[0])
        with pytest.raises(sc.ScError) as e:
            ctx.set_option(sc.SC_OPT_SERVE_PRIORITY, 1)
        assert e.value.status == sc.SC_ERR_BUSY
        ctx.wait(t, 60.0)
        ctx.release(t)
        ctx.set_option(sc.SC_OPT_SERVE_PRIORITY, 1)
    finally:
        ctx.close()

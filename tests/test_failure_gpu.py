"""Failure detection without a GPU fault: a bounded device wait that runs out
reports SC_ERR_TIMEOUT through the context's error word, and the context
keeps working (the next evaluation matches one from a fresh context)."""
import time

import numpy as np
import pytest

from paper_1609_08146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_08146_gb300 as sc  # noqa: E402


def test_bounded_wait_times_out_and_context_survives():
    ctx = sc.Context(0)
    try:
        w = wl.sweep(1e3, 32, n_points=40)
        mc = w["mirror"]
        m = ctx.mirror(mc["f"], 0.0, mc["r_max"], mc["n_r"], mc["n_theta"])
        inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"], spectrum=w["spectrum"])
        P = torch.tensor(w["points"], device="cuda")
        E1, B1 = ctx.eval(m, inc, w["omegas"], P)
        t0 = time.time()
        st = ctx._lib.sc_selftest_wait(ctx._h)
        dt = time.time() - t0
        assert st == sc.SC_ERR_TIMEOUT
        assert b"bounded device wait" in ctx._lib.sc_last_error(ctx._h)
        assert 0.5 < dt < 30.0
        # the error word was cleared and the context still evaluates correctly
        E2, B2 = ctx.eval(m, inc, w["omegas"], P, stats=True)[:2]
        torch.cuda.synchronize()
        assert torch.equal(E1, E2) and torch.equal(B1, B2)
    finally:
        ctx.close()


@pytest.mark.parametrize("n_omega,tile", [(256, 0), (256, 7), (8, 1), (8, 9), (300, 0), (300, 7)])
def test_lost_copy_ends_the_launch_after_one_wait(n_omega, tile):
    """A node-tile copy that never lands (SC_OPT_FAIL_COPY leaves it
    unissued: no fault, no copy in flight) makes its wait run out once; the
    CTA and then the whole launch stop instead of spending a wait limit on
    every later tile of the item (hundreds here).  The call reports
    SC_ERR_TIMEOUT within a few seconds, and the next call on the context is
    bitwise equal to one made before.  The direct kernel (256 and 8 omegas)
    and, with chunk planning off, the grouped kernel (300 omegas in one
    chunk); the lost copy is one of the first two or a refill."""
    ctx = sc.Context(0)
    if n_omega > 256:
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
    try:
        w = wl.sweep(1e4, 256, n_points=2048)
        mc = w["mirror"]
        m = ctx.mirror(mc["f"], 0.0, mc["r_max"], mc["n_r"], mc["n_theta"])
        om = wl.uniform_omegas(n_omega)
        inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"],
                           spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
        P = torch.tensor(w["points"], device="cuda")
        E1, B1 = ctx.eval(m, inc, om, P, stats=True)[:2]  # tunes and caches this shape
        ctx.set_option(sc.SC_OPT_FAIL_COPY, tile)
        try:
            t0 = time.time()
            with pytest.raises(sc.ScError) as e:
                ctx.eval(m, inc, om, P, stats=True)
            dt = time.time() - t0
        finally:
            ctx.set_option(sc.SC_OPT_FAIL_COPY, -1)
        assert e.value.status == sc.SC_ERR_TIMEOUT
        assert 0.5 < dt < 5.0, dt
        E2, B2 = ctx.eval(m, inc, om, P, stats=True)[:2]
        torch.cuda.synchronize()
        assert torch.equal(E1, E2) and torch.equal(B1, B2)
    finally:
        ctx.close()

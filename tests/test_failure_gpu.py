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

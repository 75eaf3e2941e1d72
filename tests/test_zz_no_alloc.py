"""The allocation-free entry point sc_eval_fp32_static.

Some callers cannot call cudaMalloc while they evaluate: services that hand
all device memory to their own pools at start-up, and real-time loops that
forbid cudaMalloc and cudaFree because those calls can block on the whole
device.  They use this entry point, whose k_n and split partials live in the
library's fixed static device scratch; a_n, the points and the outputs are
the caller's device buffers.  This file checks, through the C-ABI, that two
calls in a row give the field of Eq. 11 within the FP32 parity tolerance of
the other GPU tests, against the FP64 oracle and against sc_eval, that the
second call leaves free device memory unchanged, and that host pointers and
an oversized request are refused.  It is named to be collected last and sets
up everything it needs itself, so it passes both alone in a fresh process and
after the rest of the suite.
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

TOL32 = 1e-5


def rel_err(F, R):
    F = np.asarray(F, dtype=np.complex128)
    R = np.asarray(R, dtype=np.complex128)
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def static_eval(ctx, m, inc, om, amp, P, E, B):
    """amp: a_n as a device tensor of [n_omega][2] doubles (or a host array,
    which the call must refuse)."""
    lib = ctx._lib
    d = float(om[1] - om[0]) if om.size > 1 else 0.0
    a_ptr = amp.data_ptr() if isinstance(amp, torch.Tensor) else amp.ctypes.data
    return lib.sc_eval_fp32_static(ctx._h, m._h, inc._h, float(om[0]), d, int(om.size),
                                   ctypes.cast(a_ptr, ctypes.POINTER(ctypes.c_double)),
                                   P.data_ptr() if isinstance(P, torch.Tensor) else P.ctypes.data,
                                   int(P.shape[0]), E.data_ptr(),
                                   B.data_ptr() if B is not None else None)


def test_static_scratch_entry_point_matches_oracle_and_sc_eval():
    ctx = sc.Context(0)
    try:
        w = wl.sweep(1e4, 64, n_points=300)
        mc, beam = w["mirror"], w["beam"]
        m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"])
        inc = ctx.incident(profile="gauss", w0=beam["w0"], spectrum=w["spectrum"])
        cases = [(w["omegas"][:96], w["points"][:300]), (w["omegas"][40:57], w["points"][100:220])]
        # reference through the allocating entry point (also makes the table resident)
        refs = []
        for om, pts in cases:
            E, B = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"))
            refs.append((E, B))
        torch.cuda.synchronize()
        for i, (om, pts) in enumerate(cases):
            a_host = ctx.spectrum(inc, om)  # a_n, uploaded by the caller before the call
            amp = torch.tensor(np.ascontiguousarray(a_host.view(np.float64)), device="cuda")
            P = torch.tensor(pts, device="cuda")
            E = torch.full((om.size, P.shape[0], 3), float("nan"), dtype=torch.complex64, device="cuda")
            B = torch.full_like(E, float("nan"))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            st = static_eval(ctx, m, inc, om, amp, P, E, B)
            assert st == sc.SC_OK, ctx._lib.sc_last_error(ctx._h)
            torch.cuda.synchronize()
            if i == 1:  # set-up happened on the first call; later calls allocate nothing
                assert torch.cuda.mem_get_info()[0] == free0
            Es, Bs = E.cpu().numpy(), B.cpu().numpy()
            # the field of Eq. 11 itself, from the FP64 oracle (R11 metric on a_n x sums)
            E0, B0 = oracle.field(dict(mc, rim=1), dict(beam, r_norm=mc["r_max"]), om, pts, amp=a_host)
            assert rel_err(Es, E0) <= TOL32
            assert rel_err(Bs, B0) <= TOL32
            Er, Br = refs[i]
            assert rel_err(Es, Er.cpu().numpy()) <= TOL32
            assert rel_err(Bs, Br.cpu().numpy()) <= TOL32
        # host pointers are refused (this path copies nothing from the host)
        om, pts = cases[1]
        a_host = np.ascontiguousarray(ctx.spectrum(inc, om).view(np.float64))
        P = torch.tensor(pts, device="cuda")
        E = torch.empty((om.size, P.shape[0], 3), dtype=torch.complex64, device="cuda")
        st = static_eval(ctx, m, inc, om, a_host, P, E, None)
        assert st == sc.SC_ERR_INVALID
        assert b"device memory" in ctx._lib.sc_last_error(ctx._h)
        amp = torch.tensor(a_host, device="cuda")
        st = static_eval(ctx, m, inc, om, amp, np.ascontiguousarray(pts), E, None)
        assert st == sc.SC_ERR_INVALID
        # a request larger than the static scratch is refused with a clear message
        om = np.linspace(0.5, 1.5, 2048)
        amp = torch.zeros((2048, 2), dtype=torch.float64, device="cuda")
        P = torch.zeros((200, 3), dtype=torch.float64, device="cuda")
        E = torch.empty((1, 1, 3), dtype=torch.complex64, device="cuda")
        st = static_eval(ctx, m, inc, om, amp, P, E, None)
        assert st == sc.SC_ERR_INVALID
        assert b"static scratch" in ctx._lib.sc_last_error(ctx._h)
    finally:
        ctx.close()

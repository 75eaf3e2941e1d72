"""Batched evaluation (persistent scheduler over requests of uneven size).

A request's result must be bitwise the same alone (sc_eval) and inside a
mixed batch (sc_eval_batch): its tiling depends only on its own shape and
the reduction order is fixed.  Batches span both kernel families (up to 48
omegas: the direct kernel with 1, 2, 4 or 8 threads per point; more: grouped
kernels of 8..256 threads per point), several mirrors and beams, ragged point
counts, and match the FP64 oracle.
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


def rel_err(F, R):
    F = np.asarray(F, dtype=np.complex128)
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


SPECS = [
    # (f, n_r, n_theta, w0 / f, beam, pol, zernike, n_omega, n_points, seed)
    (1e3, 40, 36, 0.6, "gauss", "linear", [], 1, 300, 1),
    (5e3, 32, 40, 0.5, "supergauss", "radial", [], 3, 97, 2),
    (2e4, 48, 32, 0.6, "gauss", "azimuthal", [0.1, -0.05, 0.02], 8, 260, 3),
    (1e3, 40, 36, 0.6, "gauss", "linear", [], 12, 33, 4),
    (1e4, 24, 64, 0.6, "gauss", "linear", [0.05], 37, 130, 5),
    (6.25e4, 64, 64, 0.6, "gauss", "linear", [], 100, 64, 6),
    (3e3, 32, 32, 0.55, "supergauss", "linear", [], 256, 41, 7),
    (1e5, 32, 48, 0.6, "gauss", "radial", [], 520, 9, 8),
]


def make(ctx, spec):
    f, nr, nt, wr, prof, pol, zern, nom, npts, seed = spec
    m = ctx.mirror(f, 0.0, 2 * f, nr, nt)
    om = wl.uniform_omegas(nom)
    inc = ctx.incident(profile=prof, w0=wr * f, pol=pol, zernike=zern,
                       spectrum=dict(kind="sampled", omega=om, amp=np.ones(om.size)))
    pts = torch.tensor(wl.random_cube(npts, 2.0, seed), device="cuda")
    return m, inc, om, pts


def test_alone_equals_mixed_bitwise():
    ctx = sc.Context(0)
    try:
        reqs = [make(ctx, s) for s in SPECS]
        alone = [ctx.eval(m, inc, om, pts) for (m, inc, om, pts) in reqs]  # also tunes each shape
        torch.cuda.synchronize()
        mixed = ctx.eval_batch(reqs)
        torch.cuda.synchronize()
        for (Ea, Ba), (Em, Bm) in zip(alone, mixed):
            assert torch.equal(Ea, Em) and torch.equal(Ba, Bm)
        # a different mix and order gives the same bits again
        order = [5, 0, 7, 2]
        mixed2 = ctx.eval_batch([reqs[i] for i in order])
        torch.cuda.synchronize()
        for i, (Em, Bm) in zip(order, mixed2):
            assert torch.equal(alone[i][0], Em) and torch.equal(alone[i][1], Bm)
    finally:
        ctx.close()


def test_batch_matches_oracle():
    ctx = sc.Context(0)
    try:
        reqs = [make(ctx, s) for s in SPECS]
        outs = ctx.eval_batch(reqs)
        torch.cuda.synchronize()
        for spec, (m, inc, om, pts), (E, B) in zip(SPECS, reqs, outs):
            f, nr, nt, wr, prof, pol, zern, nom, npts, seed = spec
            idx = np.arange(0, npts, max(1, npts // 6))
            mo = dict(f=f, r_max=2 * f, n_r=nr, n_theta=nt, rim=1)
            bo = dict(profile=prof, w0=wr * f, pol=pol, zernike=zern, r_norm=2 * f)
            E0, B0 = oracle.field(mo, bo, om, pts.cpu().numpy()[idx])
            e = max(rel_err(E.cpu().numpy()[:, idx], E0), rel_err(B.cpu().numpy()[:, idx], B0))
            assert e <= 1e-5, (spec, e)
    finally:
        ctx.close()


def test_graph_replay_and_many_small_requests():
    ctx = sc.Context(0)
    try:
        rng = np.random.default_rng(3)
        reqs = []
        for i in range(24):
            spec = (1e3 * (1 + i % 3), 16 + 8 * (i % 3), 24, 0.6, "gauss", "linear", [],
                    int(rng.integers(1, 40)), int(rng.integers(5, 90)), 100 + i)
            reqs.append(make(ctx, spec))
        ref = [ctx.eval(m, inc, om, pts) for (m, inc, om, pts) in reqs]
        c0 = ctx.counters()
        out1 = ctx.eval_batch(reqs)
        out2 = ctx.eval_batch(reqs)
        torch.cuda.synchronize()
        c1 = ctx.counters()
        assert c1["graph_captures"] >= c0["graph_captures"] + 1
        assert c1["graph_replays"] >= c0["graph_replays"] + 1
        for (Er, Br), (E1, B1), (E2, B2) in zip(ref, out1, out2):
            assert torch.equal(Er, E1) and torch.equal(Er, E2)
            assert torch.equal(Br, B1) and torch.equal(Br, B2)
    finally:
        ctx.close()


def test_batch_rejects_host_buffers_and_bad_grids():
    ctx = sc.Context(0)
    try:
        m, inc, om, pts = make(ctx, SPECS[0])
        arr = (sc.sc_request * 1)()
        om2 = np.array([1.0, 1.1, 1.3])
        E = torch.empty((3, pts.shape[0], 3), dtype=torch.complex64, device="cuda")
        arr[0] = sc.sc_request(m._h, inc._h, om2.ctypes.data_as(sc._DP), 3,
                               sc._VP(pts.data_ptr()), pts.shape[0], sc._VP(E.data_ptr()), None)
        assert ctx._lib.sc_eval_batch(ctx._h, arr, 1, None) == sc.SC_ERR_INVALID
        host = np.zeros((pts.shape[0], 3))
        om1 = np.array([1.0])
        arr[0] = sc.sc_request(m._h, inc._h, om1.ctypes.data_as(sc._DP), 1,
                               sc._VP(host.ctypes.data), pts.shape[0], sc._VP(E.data_ptr()), None)
        assert ctx._lib.sc_eval_batch(ctx._h, arr, 1, None) == sc.SC_ERR_INVALID
    finally:
        ctx.close()

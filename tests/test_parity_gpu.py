"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on
identical seeded inputs.

Error metric (per frequency, on the spatial sums, i.e. unit amplitudes):
    err(omega) = sqrt(mean_points sum_c |F_gpu - F_oracle|^2) / max_points |F_oracle|
gated at 1e-5 for the FP32 compensated-phase path and, for the plain FP64
path, at 1e-12 plus the FP64 phase floor 2e-16 k r_max of the oracle itself.
Cases span several node tiles, several node splits with a ragged last split,
ragged omega groups and point blocks, the rim term (outer and inner), chunked
omegas and points, every beam model, and the full-size broadband workload in
the launch configuration the benchmark times (sampled points).
"""
import math

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


def tol64(mirror, omegas):
    return 1e-12 + 2e-16 * 2 * math.pi * max(omegas) * mirror["r_max"]


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    yield c
    c.close()


def rel_err(F, R):
    """max over omega of sqrt(mean_pts sum_c |F-R|^2) / max_pts |R|."""
    F = np.asarray(F, dtype=np.complex128)
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def unit_spectrum(omegas):
    return dict(kind="sampled", omega=np.asarray(omegas, float), amp=np.ones(len(omegas)))


def run_gpu(ctx, mirror, beam, omegas, pts, precision="fp32", spectrum=None):
    m = ctx.mirror(mirror["f"], mirror.get("r_min", 0.0), mirror["r_max"], mirror["n_r"],
                   mirror["n_theta"], rim=bool(mirror.get("rim", True)),
                   radial=mirror.get("radial", "gauss_legendre"))
    inc = ctx.incident(profile=beam["profile"], w0=beam["w0"], sg_order=beam.get("sg_order", 4),
                       zernike=beam.get("zernike", []), pol=beam.get("pol", "linear"),
                       pol_angle=beam.get("pol_angle", 0.0), order=beam.get("order", 0),
                       spectrum=spectrum or unit_spectrum(omegas))
    P = torch.tensor(np.asarray(pts, float), device="cuda")
    E, B = ctx.eval(m, inc, omegas, P, precision=precision)
    torch.cuda.synchronize()
    return E.cpu().numpy(), B.cpu().numpy()


def run_oracle(mirror, beam, omegas, pts, amp=None):
    m = dict(mirror)
    m["rim"] = 1 if m.get("rim", True) else 0
    b = dict(beam)
    b["r_norm"] = m["r_max"]
    return oracle.field(m, b, omegas, pts, amp=amp)


def check(ctx, mirror, beam, omegas, pts, fp64=True):
    E0, B0 = run_oracle(mirror, beam, omegas, pts)
    E, B = run_gpu(ctx, mirror, beam, omegas, pts, "fp32")
    e32 = max(rel_err(E, E0), rel_err(B, B0))
    assert e32 <= TOL32, e32
    if fp64:
        E, B = run_gpu(ctx, mirror, beam, omegas, pts, "fp64")
        e64 = max(rel_err(E, E0), rel_err(B, B0))
        assert e64 <= tol64(mirror, omegas), e64
    return e32


def test_small_monochromatic_workload(ctx):
    w = wl.small()
    check(ctx, w["mirror"], w["beam"], w["omegas"], w["points"])


@pytest.mark.parametrize(
    "beam",
    [
        dict(profile="gauss", w0=1200.0, pol="linear", pol_angle=0.3),
        dict(profile="supergauss", sg_order=4, w0=1500.0, pol="radial"),
        dict(profile="gauss", w0=1200.0, pol="azimuthal", zernike=[0.1, -0.05, 0.2, 0.03, -0.1, 0.04]),
        dict(profile="tophat", w0=1900.0, pol="linear"),
    ],
)
def test_ragged_tiles_splits_groups(ctx, beam):
    # 48 x 40 nodes = 60 tiles; 512 nodes per split -> 4 splits, last ragged;
    # 2 tiles per FP32 run -> several compensated folds per split;
    # 37 omegas -> 5 groups of 8 (ragged); 50 points (ragged point block)
    ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, 512)
    ctx.set_option(sc.SC_OPT_FLUSH_NODES, 64)
    try:
        mirror = dict(f=1000.0, r_max=2000.0, n_r=48, n_theta=40, rim=True)
        om = np.linspace(0.7, 1.3, 37)
        pts = wl.random_cube(50, 2.0, seed=11)
        check(ctx, mirror, beam, om, pts)
    finally:
        ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, 0)
        ctx.set_option(sc.SC_OPT_FLUSH_NODES, 2048)


@pytest.mark.parametrize("n_omega", [1, 2, 3, 4, 5, 6, 7, 8, 9, 11, 13, 16, 17, 21, 25, 32, 33, 40, 41, 48, 49, 64, 65,
                                     80, 100, 129, 200, 256, 600])
def test_omega_counts(ctx, n_omega):
    # every kernel class: direct (<= 48 omegas; 1, 2, 4 or 8 threads per point
    # with 1..8 omegas each) and grouped (8..256 threads per point), and
    # requests cut into a full grouped chunk and a rest (65, 80, 129, 200, 600)
    mirror = dict(f=62500.0, r_max=125000.0, n_r=24, n_theta=32, rim=True)
    beam = dict(profile="gauss", w0=37500.0, pol="linear")
    om = wl.uniform_omegas(n_omega)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(12, 2.0, seed=n_omega)])
    check(ctx, mirror, beam, om, pts, fp64=n_omega <= 64)


def test_omega_chunks_beyond_2048(ctx):
    mirror = dict(f=100.0, r_max=200.0, n_r=16, n_theta=16, rim=True)
    beam = dict(profile="gauss", w0=60.0, pol="linear")
    om = np.linspace(0.6, 1.4, 2600)
    pts = wl.random_cube(3, 1.0, seed=5)
    check(ctx, mirror, beam, om, pts, fp64=False)


def test_chunk_planning_on_and_off(ctx):
    # 65 omegas: planned as 64 + 1 (grouped and direct kernels), or one chunk
    # on 16 threads per point with SC_OPT_OMEGA_CHUNKS = 0; both within the
    # gate against the oracle, and the plan reported for the context follows
    # the option
    mirror = dict(f=1000.0, r_max=2000.0, n_r=40, n_theta=48, rim=True)
    beam = dict(profile="gauss", w0=600.0, pol="radial")
    om = wl.uniform_omegas(65)
    pts = wl.random_cube(30, 1.5, seed=65)
    assert sorted(ctx.plan_omega_chunks(65, 1000)) == [1, 64]
    e_on = check(ctx, mirror, beam, om, pts, fp64=False)
    ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
    try:
        assert ctx.plan_omega_chunks(65, 1000) == [65]
        assert ctx.plan_omega_chunks(5000, 1000) == [2048, 2048, 904]
        e_off = check(ctx, mirror, beam, om, pts, fp64=False)
    finally:
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 1)
    assert max(e_on, e_off) <= TOL32


@pytest.mark.parametrize("n_omega", [300, 600, 1100])
def test_grouped_kernel_classes(ctx, n_omega):
    # chunk planning off: chunks above 256 omegas run on the grouped kernel
    # (64, 128 and 256 threads per point), the classes planning never reaches;
    # ragged splits and folds
    mirror = dict(f=500.0, r_max=1000.0, n_r=40, n_theta=44, rim=True)
    beam = dict(profile="gauss", w0=500.0, pol="radial", zernike=[0.05, -0.1, 0.03])
    om = wl.uniform_omegas(n_omega)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(9, 1.5, seed=n_omega)])
    ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
    ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, 640)
    ctx.set_option(sc.SC_OPT_FLUSH_NODES, 256)
    try:
        assert ctx.plan_omega_chunks(n_omega, 1000) == [n_omega]
        check(ctx, mirror, beam, om, pts, fp64=False)
    finally:
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 1)
        ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, 0)
        ctx.set_option(sc.SC_OPT_FLUSH_NODES, 2048)


# (omega count, default layout, alternative layout) as (class, threads per
# point, omegas per thread)
LAYOUTS = [(8, (7, 2, 4), (24, 1, 8)), (11, (9, 2, 6), (25, 4, 3)), (15, (11, 2, 8), (26, 4, 4)),
           (40, (15, 8, 5), (27, 16, 3)), (57, (18, 8, 8), (28, 16, 4)),
           (100, (19, 16, 8), (29, 32, 4))]


@pytest.mark.parametrize("n_omega,default,alt", LAYOUTS)
def test_tile_layouts(ctx, n_omega, default, alt):
    # both tile shapes of the omega counts that have two, pinned with
    # SC_OPT_TILE_LAYOUT, each against the oracle (ragged omega groups and
    # point blocks, several splits); the shape the call took is reported
    mirror = dict(f=700.0, r_max=1400.0, n_r=36, n_theta=40, rim=True)
    beam = dict(profile="gauss", w0=600.0, pol="linear", zernike=[0.0, 0.05, -0.02])
    om = wl.uniform_omegas(n_omega)
    pts = wl.random_cube(37, 1.5, seed=n_omega)
    E0, B0 = run_oracle(mirror, beam, om, pts)
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"], rim=True)
    inc = ctx.incident(profile="gauss", w0=beam["w0"], pol="linear", zernike=beam["zernike"],
                       spectrum=unit_spectrum(om))
    P = torch.tensor(pts, device="cuda")
    ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
    ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, 320)
    try:
        for layout, want in ((0, default), (1, alt), (-1, None)):
            ctx.set_option(sc.SC_OPT_TILE_LAYOUT, layout)
            E, B, st = ctx.eval(m, inc, om, P, stats=True)
            torch.cuda.synchronize()
            got = (st["kernel_class"], st["threads_per_point"], st["omegas_per_thread"])
            if want is None:
                assert got in (default, alt)
            else:
                assert got == want
            assert st["splits"] == -(-mirror["n_r"] * mirror["n_theta"] // 320)
            err = max(rel_err(E.cpu().numpy(), E0), rel_err(B.cpu().numpy(), B0))
            assert err <= TOL32, (layout, err)
    finally:
        ctx.set_option(sc.SC_OPT_TILE_LAYOUT, -1)
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 1)
        ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, 0)


def test_tile_layout_autotuned_and_reported(ctx):
    # with the autotuner on, an omega count with two layouts takes one of them
    # (timed once, then cached: a second call reports the same shape); the
    # FP64 path reports no shape; out-of-range values are refused
    mirror = dict(f=700.0, r_max=1400.0, n_r=48, n_theta=48, rim=True)
    om = wl.uniform_omegas(100)
    pts = wl.random_cube(300, 1.5, seed=100)
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"], rim=True)
    inc = ctx.incident(profile="gauss", w0=600.0, pol="radial", spectrum=unit_spectrum(om))
    P = torch.tensor(pts, device="cuda")
    ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 0)
    try:
        shapes = []
        for _ in range(2):
            E, B, st = ctx.eval(m, inc, om, P, stats=True)
            torch.cuda.synchronize()
            shapes.append((st["kernel_class"], st["threads_per_point"], st["omegas_per_thread"],
                           st["splits"]))
        assert shapes[0] == shapes[1]
        assert shapes[0][:3] in ((19, 16, 8), (29, 32, 4))
        assert shapes[0][3] >= 1
        sel = np.arange(0, 300, 10)
        E0, B0 = run_oracle(mirror, dict(profile="gauss", w0=600.0, pol="radial"), om, pts[sel])
        assert max(rel_err(E.cpu().numpy()[:, sel], E0), rel_err(B.cpu().numpy()[:, sel], B0)) <= TOL32
        _, _, st = ctx.eval(m, inc, om, P, precision="fp64", stats=True)
        assert st["kernel_class"] == -1 and st["threads_per_point"] == -1
    finally:
        ctx.set_option(sc.SC_OPT_OMEGA_CHUNKS, 1)
    for bad in (-2, 2):
        with pytest.raises(sc.ScError):
            ctx.set_option(sc.SC_OPT_TILE_LAYOUT, bad)


@pytest.mark.parametrize("n_omega", [25, 33, 41, 49])
def test_small_count_cuts_on_a_large_request(ctx, n_omega):
    # 64 x 64 nodes and 1030 points: above 4M pairs per omega, so small counts
    # are cut too (e.g. 33 as 1 + 32, 41 as 10 + 31 under the measured tables);
    # a sample of the points against the oracle
    mirror = dict(f=1000.0, r_max=2000.0, n_r=64, n_theta=64, rim=True)
    beam = dict(profile="supergauss", w0=1200.0, pol="azimuthal")
    om = wl.uniform_omegas(n_omega)
    pts = wl.random_cube(1030, 1.5, seed=n_omega)
    assert len(ctx.plan_omega_chunks(n_omega, 1030 * 64 * 64)) > 1
    E, B = run_gpu(ctx, mirror, beam, om, pts)
    sel = np.arange(0, 1030, 26)
    E0, B0 = run_oracle(mirror, beam, om, pts[sel])
    assert max(rel_err(E[:, sel], E0), rel_err(B[:, sel], B0)) <= TOL32


def test_inner_rim_and_no_rim(ctx):
    beam = dict(profile="gauss", w0=300.0, pol="radial")
    om = np.linspace(0.8, 1.2, 20)
    pts = wl.random_cube(20, 1.5, seed=3)
    check(ctx, dict(f=500.0, r_min=150.0, r_max=900.0, n_r=32, n_theta=48, rim=True), beam, om, pts)
    check(ctx, dict(f=500.0, r_min=150.0, r_max=900.0, n_r=32, n_theta=48, rim=False), beam, om, pts)


@pytest.mark.parametrize(
    "mirror,beam",
    [
        # disk: the node row at r = 0 has zero weight
        (dict(f=500.0, r_max=900.0, n_r=41, n_theta=48, rim=True, radial="simpson"),
         dict(profile="gauss", w0=400.0, pol="linear", pol_angle=0.2)),
        # annulus, both rims, aberrated radial beam
        (dict(f=500.0, r_min=150.0, r_max=900.0, n_r=33, n_theta=48, rim=True, radial="simpson"),
         dict(profile="supergauss", sg_order=4, w0=500.0, pol="radial", zernike=[0.1, -0.2, 0.05, 0.1])),
        # first-order beam (second node table) through r = 0
        (dict(f=40.0, r_max=60.0, n_r=45, n_theta=40, rim=True, radial="simpson"),
         dict(profile="gauss", w0=12.0, pol="azimuthal", order=1)),
    ],
)
def test_simpson_radial_rule(ctx, mirror, beam):
    """Composite Simpson in r (Sec. III.C.1 names Simpson or Gauss-Legendre):
    the same sum on both sides, FP32 and FP64 against the oracle, over
    ragged tiles and omega groups (13 omegas)."""
    om = wl.uniform_omegas(13)
    pts = np.vstack([np.zeros((1, 3)), wl.random_cube(20, 1.5, seed=41)])
    check(ctx, mirror, beam, om, pts, fp64=False)
    E0, B0 = run_oracle(mirror, beam, om, pts)
    E, B = run_gpu(ctx, mirror, beam, om, pts, "fp64")
    # the first-order oracle takes its divergences by finite differences (1e-11)
    tol = 1e-11 if beam.get("order", 0) else tol64(mirror, om)
    assert max(rel_err(E, E0), rel_err(B, B0)) <= tol


def test_simpson_focus_closed_form_on_gpu(ctx):
    """Simpson in r on the GPU tends to the hand-derived focal value of Eq. 11
    at fourth order: the FP64 path's error falls 16x per halving of h."""
    f, a, om = 20.0, 30.0, np.array([1.0])
    k = 2 * math.pi
    Ra = f + a * a / (4 * f)
    Ex = 2 * (1j * k * f + 1) * (1 - f / Ra) - (1 - f * f / Ra ** 2) - (a * a / (2 * Ra ** 2)) * (
        1 + 1j / (k * Ra))
    errs = []
    for n in (9, 17, 33):
        E, _ = run_gpu(ctx, dict(f=f, r_max=a, n_r=n, n_theta=16, rim=True, radial="simpson"),
                       dict(profile="tophat", w0=1.01 * a, pol="linear"), om, np.zeros((1, 3)), "fp64")
        errs.append(abs(E[0, 0, 0] - Ex) / abs(Ex))
    assert 14.0 < errs[0] / errs[1] < 18.5 and 14.0 < errs[1] / errs[2] < 18.5, errs


def test_point_chunking_small_workspace(ctx):
    ctx.set_option(sc.SC_OPT_WORKSPACE_CAP, 1 << 20)
    try:
        mirror = dict(f=2000.0, r_max=4000.0, n_r=32, n_theta=32, rim=True)
        beam = dict(profile="gauss", w0=2400.0, pol="linear")
        om = wl.uniform_omegas(40)
        pts = wl.random_cube(700, 2.0, seed=9)
        check(ctx, mirror, beam, om, pts, fp64=False)
    finally:
        ctx.set_option(sc.SC_OPT_WORKSPACE_CAP, 2 << 30)


def test_tophat_focus_closed_form_on_gpu(ctx):
    """GPU against the hand-derived focal value of Eq. 11 (no oracle)."""
    f, a = 20.0, 30.0
    om = np.array([0.9, 1.0, 1.1])
    E, B = run_gpu(ctx, dict(f=f, r_max=a, n_r=160, n_theta=64, rim=True),
                   dict(profile="tophat", w0=1.01 * a, pol="linear"), om, np.zeros((1, 3)))
    Ra = f + a * a / (4 * f)
    for i, o in enumerate(om):
        k = 2 * math.pi * o
        Ex = 2 * (1j * k * f + 1) * (1 - f / Ra) - (1 - f * f / Ra ** 2) - (a * a / (2 * Ra ** 2)) * (
            1 + 1j / (k * Ra))
        By = 2j * k * f * (1 - f / Ra) - (1 - f * f / Ra ** 2)
        assert abs(E[i, 0, 0] - Ex) < 1e-5 * abs(Ex)
        assert abs(B[i, 0, 1] - By) < 1e-5 * abs(Ex)


def test_host_buffers_equal_device_buffers(ctx):
    w = wl.sweep(1000.0, 32, n_points=64)
    m = ctx.mirror(**{k: w["mirror"][k] for k in ("f", "r_min", "r_max", "n_r", "n_theta")})
    inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"], spectrum=w["spectrum"])
    om = w["omegas"][:40]
    Eh, Bh = ctx.eval(m, inc, om, w["points"])  # numpy in, numpy out (staged)
    Ed, Bd = ctx.eval(m, inc, om, torch.tensor(w["points"], device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(Eh, Ed.cpu().numpy())
    assert np.array_equal(Bh, Bd.cpu().numpy())


def test_deterministic(ctx):
    w = wl.sweep(1e4, 64, n_points=128)
    m = ctx.mirror(**{k: w["mirror"][k] for k in ("f", "r_min", "r_max", "n_r", "n_theta")})
    inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"], spectrum=w["spectrum"])
    P = torch.tensor(w["points"], device="cuda")
    E1, B1 = ctx.eval(m, inc, w["omegas"], P)
    E2, B2 = ctx.eval(m, inc, w["omegas"], P)
    torch.cuda.synchronize()
    assert torch.equal(E1, E2) and torch.equal(B1, B2)


def test_spectrum_applied(ctx):
    # with the physical spectrum, E_n = a_n times the unit-amplitude field
    w = wl.sweep(1000.0, 24, n_points=16)
    mirror, beam = w["mirror"], w["beam"]
    om = w["omegas"][::8]
    spec = dict(w["spectrum"], phi=[0.0, 0.0, 1.5])
    a = oracle.spectrum(spec, om, beam)
    E0, B0 = run_oracle(mirror, beam, om, w["points"], amp=a)
    E, B = run_gpu(ctx, mirror, beam, om, w["points"], "fp32", spectrum=spec)
    assert max(rel_err(E, E0), rel_err(B, B0)) <= TOL32


def test_time_domain_matches_oracle(ctx):
    w = wl.sweep(1000.0, 32, n_points=40)
    om = w["omegas"]
    E, B = run_gpu(ctx, w["mirror"], w["beam"], om, w["points"], "fp32", spectrum=w["spectrum"])
    t = (np.arange(96) - 48) / 4.0
    Et, Bt = ctx.time_domain(torch.tensor(E, device="cuda"), torch.tensor(B, device="cuda"), om, t)
    torch.cuda.synchronize()
    Rt = oracle.time_domain(E.astype(np.complex128), om, t)
    RBt = oracle.time_domain(B.astype(np.complex128), om, t)
    assert np.max(np.abs(Et.cpu().numpy() - Rt)) <= 2e-6 * np.max(np.abs(Rt))
    assert np.max(np.abs(Bt.cpu().numpy() - RBt)) <= 2e-6 * np.max(np.abs(RBt))
    # FP64 spectra through the same stage
    E64, _ = run_gpu(ctx, w["mirror"], w["beam"], om, w["points"], "fp64", spectrum=w["spectrum"])
    Et64, _ = ctx.time_domain(torch.tensor(E64, device="cuda"), None, om, t, precision="fp64")
    torch.cuda.synchronize()
    R64 = oracle.time_domain(E64, om, t)
    assert np.max(np.abs(Et64.cpu().numpy() - R64)) <= 2e-6 * np.max(np.abs(R64))


def test_invalid_inputs(ctx):
    m = ctx.mirror(20.0, 0.0, 40.0, 8, 8)
    inc = ctx.incident(profile="gauss", w0=20.0)
    with pytest.raises(sc.ScError) as e:
        ctx.eval(m, inc, [1.0, 1.1, 1.3], np.zeros((2, 3)))  # non-uniform grid, FP32 path
    assert e.value.status == sc.SC_ERR_INVALID
    on_mirror = np.array([[10.0, 0.0, 100.0 / 80.0 - 20.0]])
    with pytest.raises(sc.ScError) as e:
        ctx.eval(m, inc, [1.0], on_mirror)
    assert e.value.status == sc.SC_ERR_INVALID
    with pytest.raises(sc.ScError):
        ctx.eval(m, inc, [-1.0], np.zeros((1, 3)))
    # a non-uniform grid is fine on the FP64 path
    E, _ = ctx.eval(m, inc, [1.0, 1.1, 1.3], np.zeros((2, 3)), precision="fp64")
    assert np.all(np.isfinite(E))


@pytest.mark.parametrize("f", [1e2, 1e3, 1e4, 1e5])
def test_precision_sweep_sampled(ctx, f):
    """Compensated phase at f/lambda0 up to 1e5 (256 x 256 nodes, 256 omegas,
    8 sampled points of the random focal cube)."""
    w = wl.sweep(f, 256, n_points=4096)
    pts = w["points"][::512]
    check(ctx, w["mirror"], w["beam"], w["omegas"], pts, fp64=False)


def test_precision_sweep_1024_nodes_at_f_1e5(ctx):
    """The largest precision-sweep case: f = 1e5 lambda0, 1024 x 1024 nodes,
    256 omegas, the 4096-point focal cube on the GPU in one call; the oracle
    checks 64 sampled points at 16 omegas spread over the band (both ends)."""
    w = wl.sweep(1e5, 1024, n_points=4096)
    mirror, beam = w["mirror"], w["beam"]
    om = w["omegas"]
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    inc = ctx.incident(profile="gauss", w0=beam["w0"], spectrum=unit_spectrum(om))
    E, B = ctx.eval(m, inc, om, torch.tensor(w["points"], device="cuda"))
    torch.cuda.synchronize()
    sel = np.arange(0, 4096, 64)
    so = np.round(np.linspace(0, 255, 16)).astype(int)
    E0, B0 = run_oracle(mirror, beam, om[so], w["points"][sel])
    Es = E.cpu().numpy()[so][:, sel]
    Bs = B.cpu().numpy()[so][:, sel]
    assert max(rel_err(Es, E0), rel_err(Bs, B0)) <= TOL32


def test_broadband_full_size_sampled(ctx):
    """The benchmark's workload (512 x 512 nodes, 256 omegas, 4160 points) in
    the benchmark's launch configuration; the oracle checks 10 sampled points
    (focus, plane and axis) at every omega."""
    w = wl.broadband()
    mirror, beam = w["mirror"], w["beam"]
    m = ctx.mirror(mirror["f"], 0.0, mirror["r_max"], mirror["n_r"], mirror["n_theta"])
    om = w["omegas"]
    inc = ctx.incident(profile="gauss", w0=beam["w0"], spectrum=unit_spectrum(om))
    P = torch.tensor(w["points"], device="cuda")
    E, B = ctx.eval(m, inc, om, P)
    torch.cuda.synchronize()
    idx = np.array([2080, 0, 63, 1000, 2047, 3000, 4095, 4096, 4127, 4159])
    E0, B0 = run_oracle(mirror, beam, om, w["points"][idx])
    Es, Bs = E.cpu().numpy()[:, idx], B.cpu().numpy()[:, idx]
    assert max(rel_err(Es, E0), rel_err(Bs, B0)) <= TOL32
    assert torch.isfinite(torch.view_as_real(E)).all()

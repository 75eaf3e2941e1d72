"""Sec. IV.A's numerical checks on the GPU path: a radially polarised,
unclipped Gaussian beam with Table 1's spectrum on an NA = 1 paraboloid.

  * parity with the FP64 oracle at sampled focal points;
  * the focal structure of a radial beam (E_z alone on the axis);
  * convergence of every non-vanishing component with the mesh, with mesh
    cells far larger than the wavelength (Sec. IV.A: more than 100 lambda);
  * the frequency-domain Maxwell residual e_f of Eq. 26a: it falls as the
    square of the finite-difference step until it meets the O(eps) error of
    the collimated incident beam (eps = lambda / (pi w0), Sec. III.A), and
    below that with the first-order beam;
  * energy: the time-domain field in a 25 lambda cube around the focus holds
    the energy of the incident pulse (Sec. IV.A).
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
from paper_1609_08146_gb300 import numerical_checks as nc  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = sc.Context(0)
    yield c
    c.close()


def rel_err(F, R):
    F = np.asarray(F, dtype=np.complex128)
    num = np.sqrt(np.mean(np.sum(np.abs(F - R) ** 2, axis=2), axis=1))
    den = np.max(np.sqrt(np.sum(np.abs(R) ** 2, axis=2)), axis=1)
    return float(np.max(num / den))


def test_radial_na1_parity_and_focus(ctx):
    cfg = nc.config(n_nodes=192, n_omega=100)
    pts = np.vstack([np.zeros((1, 3)), [[0.3, 0.0, 0.0], [0.0, -0.4, 0.2]], wl.random_cube(5, 1.0, 41)])
    m, inc = nc._handles(ctx, cfg)
    om = cfg["omegas"]
    E, B = ctx.eval(m, inc, om, torch.tensor(pts, device="cuda"))
    torch.cuda.synchronize()
    mo, bo = wl.oracle_args(cfg)
    amp = oracle.spectrum(cfg["spectrum"], om, bo)
    sel = [0, 33, 66, 99]
    E0, B0 = oracle.field(mo, bo, om[sel], pts, amp=amp[sel])
    E, B = E.cpu().numpy(), B.cpu().numpy()
    assert max(rel_err(E[sel], E0), rel_err(B[sel], B0)) <= 1e-5
    # on the axis a radial beam focuses to E_z alone; B vanishes there
    peak = np.abs(E[:, 0, 2]).max()
    assert np.abs(E[:, 0, :2]).max() < 1e-6 * peak
    assert np.abs(B[:, 0, :]).max() < 1e-6 * peak
    # off the axis along x: E_rho = E_x and B_theta = B_y
    assert np.abs(E[:, 1, 0]).max() > 0.2 * peak and np.abs(B[:, 1, 1]).max() > 0.2 * peak


def test_convergence_with_mesh(ctx):
    cfg = nc.config(n_nodes=256)
    pts, _ = nc.cube(4.0, 1.0)
    rows = nc.convergence(ctx, cfg, [16, 32, 48, 64, 96, 256], pts)
    worst = [max(r["e_rel"].values()) for r in rows[:-1]]
    assert set(rows[0]["e_rel"]) == {"E_x", "E_y", "E_z", "B_x", "B_y"}  # B_z = 0 by symmetry
    assert worst[0] > 1e-2  # 16 x 16 nodes do not resolve a +-4 lambda region
    assert all(b <= max(a * 1.5, 1e-10) for a, b in zip(worst, worst[1:]))  # down to the FP64 floor
    # converged at mesh cells of thousands of wavelengths
    i64 = [r["n"] for r in rows].index(64)
    assert worst[i64] < 1e-9 and rows[i64]["cell_lambda"] > 1000.0


def test_maxwell_frequency_residual(ctx):
    cfg = nc.config(n_nodes=256)
    coarse = nc.maxwell_freq(ctx, cfg, dx=1e-2, omega_indices=[0, 99], precision="fp64")
    fine = nc.maxwell_freq(ctx, cfg, dx=1e-3, omega_indices=[0, 99], precision="fp64")
    floor = nc.maxwell_freq(ctx, cfg, dx=1e-4, omega_indices=[0, 99], precision="fp64")
    eps = 1.0 / (math.pi * cfg["beam"]["w0"])
    for c, f, z in zip(coarse, fine, floor):
        k = 2 * math.pi * c["omega"]
        # finite-difference limited: about (k dx)^2 / 6 per curl
        assert c["max_e_f"] < 4 * (k * 1e-2) ** 2 / 6 * 2
        assert f["max_e_f"] < c["max_e_f"] / 30
        # then the collimated beam's own O(eps) error
        assert z["max_e_f"] < 3 * eps


def test_first_order_beam_removes_the_eps_floor(ctx):
    """With the O(eps) longitudinal terms the incident beam obeys Maxwell to
    O(eps^2) (about 3e-11 here), so e_f keeps falling with dx below the
    collimated beam's eps = 5e-6 floor, down to the finite-difference error."""
    cfg = nc.config(n_nodes=256, order=1)
    eps = 1.0 / (math.pi * cfg["beam"]["w0"])
    fine = nc.maxwell_freq(ctx, cfg, dx=1e-4, omega_indices=[0, 99], precision="fp64")
    for r in fine:
        k = 2 * math.pi * r["omega"]
        assert r["max_e_f"] < 0.1 * eps
        assert r["max_e_f"] < 10 * (k * 1e-4) ** 2


def test_focal_volume_energy(ctx):
    cfg = nc.config(n_nodes=512)
    r = nc.energy(ctx, cfg, half=12.5, h=0.4, times=(-2.0, 0.0, 2.0))
    # 0.24% of the pulse energy lies more than 12.5 lambda / c from its centre
    assert 0.997 < r["ratio"][1] <= 1.0005, r
    assert abs(r["ratio"][0] - r["ratio"][1]) < 1e-3 and abs(r["ratio"][2] - r["ratio"][1]) < 1e-3

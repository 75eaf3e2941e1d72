"""Host-side planning of node tables (sc_table_count, no GPU): how many field
passes a (mirror, beam) pair costs and whether the compensated FP32 path
applies.  Covers the Chebyshev fit of k-dependent envelopes (its truncation,
the phase factoring that makes a pulse-front tilt one table, the rejection of
an envelope too rough to fit), the first-order beam and the ellipsoid's
dipole without running a kernel."""
import ctypes

import numpy as np

import paper_1609_08146_gb300 as sc


def _mirror(lib, f=20.0, r_max=40.0, n=48, ellipsoid=None):
    q = sc.sc_quadrature(0, n, n, 1)
    h = ctypes.c_void_p()
    if ellipsoid is None:
        assert lib.sc_mirror(None, f, 0.0, r_max, ctypes.byref(q), ctypes.byref(h)) == sc.SC_OK
    else:
        c, e = ellipsoid
        assert lib.sc_mirror_ellipsoid(None, c, e, 0.0, r_max, ctypes.byref(q), ctypes.byref(h)) == sc.SC_OK
    return h


def _incident(lib, kind=0, w0=6.0, pol=0, order=0, lg=(0, 0, -30.0), band=(0.8, 1.2), tol=0.0,
              envelope=None, dipole=(0.0, 0.0, 0.0), keep=None):
    prof = sc.sc_profile(kind, w0, 4, 0, None, order, lg[0], lg[1], lg[2],
                         ctypes.cast(envelope, ctypes.c_void_p) if envelope is not None else None, None,
                         band[0], band[1], tol, (ctypes.c_double * 3)(*dipole))
    spec = sc.sc_spectrum(0, 1.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    h = ctypes.c_void_p()
    st = lib.sc_incident(None, ctypes.byref(prof), ctypes.byref(sc.sc_polarization(pol, 0.3)),
                         ctypes.byref(spec), ctypes.byref(h))
    assert st == sc.SC_OK
    if keep is not None:
        keep.append(envelope)
    return h


def _count(lib, m, inc):
    n, ok = ctypes.c_int(-1), ctypes.c_int(-1)
    st = lib.sc_table_count(None, m, inc, ctypes.byref(n), ctypes.byref(ok))
    return st, n.value, ok.value


def _envelope(fn):
    def cb(user, n, xyz, k, out):
        pts = np.ctypeslib.as_array(xyz, shape=(n, 3)).copy()
        e = np.asarray(fn(pts, k), dtype=np.complex128).reshape(n, 2)
        np.ctypeslib.as_array(out, shape=(n, 4))[:] = e.view(np.float64)
    return sc.ENVELOPE_FN(cb)


def test_collimated_and_first_order_beams():
    lib = sc.load()
    m = _mirror(lib)
    assert _count(lib, m, _incident(lib)) == (sc.SC_OK, 1, 1)
    assert _count(lib, m, _incident(lib, order=1)) == (sc.SC_OK, 2, 1)


def test_laguerre_gauss_tables_shrink_with_the_tolerance():
    lib = sc.load()
    m = _mirror(lib, n=96)
    for pol, p, l in ((0, 0, 0), (0, 1, 2), (1, 0, 1), (2, 1, 1)):
        n = [_count(lib, m, _incident(lib, kind=3, pol=pol, lg=(p, l, -35.0), tol=tol))[1]
             for tol in (1e-6, 1e-8, 1e-10)]
        assert 6 <= n[0] < n[1] < n[2] <= 40, (pol, p, l, n)
        assert n[1] % 2 == 0  # complex envelopes: real and imaginary part per term


def test_tilt_is_one_table_and_a_rough_envelope_is_rejected():
    lib = sc.load()
    m = _mirror(lib, n=48)
    keep = []
    tilt = _envelope(lambda q, k: np.column_stack(
        [np.exp(-(q[:, 0] ** 2 + q[:, 1] ** 2) / 49.0) * np.exp(3j * k * q[:, 0]), 0 * q[:, 0]]))
    st, n, ok = _count(lib, m, _incident(lib, kind=4, envelope=tilt, keep=keep))
    assert (st, n, ok) == (sc.SC_OK, 1, 1)
    rough = _envelope(lambda q, k: np.column_stack([np.exp(3j * k * k * q[:, 0]), 0 * q[:, 0]]))
    st, _, _ = _count(lib, m, _incident(lib, kind=4, envelope=rough, keep=keep))
    assert st == sc.SC_ERR_INVALID


def test_ellipsoid_dipole_and_collimated_beam():
    lib = sc.load()
    ell = _mirror(lib, r_max=12.0, ellipsoid=(14.0, 6.0))
    assert _count(lib, ell, _incident(lib, kind=5, dipole=(1.0, 0.0, 0.0))) == (sc.SC_OK, 3, 1)
    assert _count(lib, ell, _incident(lib)) == (sc.SC_OK, 1, 0)  # needs FP64
    par = _mirror(lib)
    st, _, _ = _count(lib, par, _incident(lib, kind=5, dipole=(1.0, 0.0, 0.0)))
    assert st == sc.SC_ERR_INVALID

"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads,
exports every entry point include/sc.h declares, and its host-only logic
(argument validation, the spectrum generator of Eqs. 16-18 and 27) agrees
with the oracle.  No kernel is launched here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_1609_08146_gb300 as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sc_status|void|const char\s*\*)\s*(sc_\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = sc.load()
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sc.SIGNATURES), set(names) ^ set(sc.SIGNATURES)


def _header_constants():
    """Every NAME = value enumerator of include/sc.h (comments removed)."""
    txt = open(os.path.join(ROOT, "include", "sc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(SC_[A-Z0-9_]+)\s*=\s*(-?\d+)\b", txt)}


def test_binding_constants_match_the_header():
    # the binding marshals statuses and option numbers as plain integers, so
    # each of its SC_* names must carry the header's value
    hdr = _header_constants()
    assert len(hdr) >= 20
    mine = {k: v for k, v in vars(sc).items() if k.startswith("SC_") and isinstance(v, int)}
    common = set(hdr) & set(mine)
    assert {"SC_OK", "SC_ERR_BUSY", "SC_OPT_SERVE_PRIORITY", "SC_OPT_TILE_LAYOUT"} <= common
    for k in sorted(common):
        assert mine[k] == hdr[k], (k, mine[k], hdr[k])
    # every option the header declares is reachable from the binding
    assert {k for k in hdr if k.startswith("SC_OPT_")} <= set(mine)


def test_host_validation_without_gpu():
    lib = sc.load()
    h = ctypes.c_void_p()
    q = sc.sc_quadrature(0, 8, 8, 1)
    assert lib.sc_mirror(None, -1.0, 0.0, 1.0, ctypes.byref(q), ctypes.byref(h)) == sc.SC_ERR_INVALID
    assert lib.sc_mirror(None, 1.0, 2.0, 1.0, ctypes.byref(q), ctypes.byref(h)) == sc.SC_ERR_INVALID
    bad = sc.sc_quadrature(0, 0, 8, 1)
    assert lib.sc_mirror(None, 1.0, 0.0, 1.0, ctypes.byref(bad), ctypes.byref(h)) == sc.SC_ERR_INVALID
    assert lib.sc_mirror(None, 1.0, 0.0, 2.0, ctypes.byref(q), ctypes.byref(h)) == sc.SC_OK
    lib.sc_mirror_free(h)
    # composite Simpson (Sec. III.C.1) needs an odd node count >= 3
    for n_r, want in ((3, sc.SC_OK), (9, sc.SC_OK), (1, sc.SC_ERR_INVALID), (8, sc.SC_ERR_INVALID)):
        qs = sc.sc_quadrature(sc.RADIAL_RULES["simpson"], n_r, 8, 1)
        assert lib.sc_mirror(None, 1.0, 0.0, 2.0, ctypes.byref(qs), ctypes.byref(h)) == want, n_r
        assert lib.sc_mirror_ellipsoid(None, 14.0, 6.0, 0.0, 2.0, ctypes.byref(qs), ctypes.byref(h)) == want
        if want == sc.SC_OK:
            lib.sc_mirror_free(h)
    unknown = sc.sc_quadrature(2, 9, 8, 1)
    assert lib.sc_mirror(None, 1.0, 0.0, 2.0, ctypes.byref(unknown), ctypes.byref(h)) == sc.SC_ERR_INVALID
    prof = sc.sc_profile(0, -1.0, 4, 0, None)
    pol = sc.sc_polarization(0, 0.0)
    spec = sc.sc_spectrum(0, 1.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    assert lib.sc_incident(None, ctypes.byref(prof), ctypes.byref(pol), ctypes.byref(spec),
                           ctypes.byref(h)) == sc.SC_ERR_INVALID
    assert lib.sc_eval(None, None, None, None, 0, None, 0, 0, None, None, None) == sc.SC_ERR_INVALID
    assert lib.sc_create(0, None, 0, None) == sc.SC_ERR_INVALID


def test_first_order_beam_validation():
    """Beam order 1 (the O(eps) longitudinal terms) needs a smooth profile."""
    lib = sc.load()
    pol = sc.sc_polarization(0, 0.0)
    spec = sc.sc_spectrum(0, 1.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    cases = [(0, 0, sc.SC_OK), (0, 1, sc.SC_OK), (1, 1, sc.SC_OK), (2, 0, sc.SC_OK),
             (2, 1, sc.SC_ERR_INVALID), (0, 2, sc.SC_ERR_INVALID), (0, -1, sc.SC_ERR_INVALID)]
    for kind, order, want in cases:
        h = ctypes.c_void_p()
        prof = sc.sc_profile(kind, 2.0, 4, 0, None, order)
        st = lib.sc_incident(None, ctypes.byref(prof), ctypes.byref(pol), ctypes.byref(spec), ctypes.byref(h))
        assert st == want, (kind, order)
        if st == sc.SC_OK:
            lib.sc_incident_free(h)


def test_envelope_beam_validation():
    """Kinds 3 (Laguerre-Gauss) and 4 (caller's envelope) need a band, valid
    mode indices, a function and a spectrum that needs no beam power."""
    lib = sc.load()
    mono = sc.sc_spectrum(0, 1.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    gtime = sc.sc_spectrum(1, 3.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    fn = sc.ENVELOPE_FN(lambda user, n, xyz, k, e: None)
    fptr = ctypes.cast(fn, ctypes.c_void_p)

    def prof(kind, p=0, l=0, lo=0.8, hi=1.2, f=None, order=0):
        return sc.sc_profile(kind, 5.0, 4, 0, None, order, p, l, -10.0, f, None, lo, hi, 0.0)

    cases = [
        (prof(3), 0, mono, sc.SC_OK),
        (prof(3, 2, 3), 0, gtime, sc.SC_OK),
        (prof(3, lo=0.0), 0, mono, sc.SC_ERR_INVALID),
        (prof(3, lo=1.2, hi=1.1), 0, mono, sc.SC_ERR_INVALID),
        (prof(3, -1), 0, mono, sc.SC_ERR_INVALID),
        (prof(3, 0, 2), 1, mono, sc.SC_ERR_INVALID),   # radial needs |l| = 1
        (prof(3, 0, -1), 2, mono, sc.SC_OK),
        (prof(3, order=1), 0, mono, sc.SC_ERR_INVALID),
        (prof(4), 0, mono, sc.SC_ERR_INVALID),         # no function
        (prof(4, f=fptr), 0, mono, sc.SC_OK),
        (prof(4, f=fptr), 0, gtime, sc.SC_ERR_INVALID),  # no beam power for Eq. 16
    ]
    for pr, polk, spec, want in cases:
        h = ctypes.c_void_p()
        pol = sc.sc_polarization(polk, 0.0)
        st = lib.sc_incident(None, ctypes.byref(pr), ctypes.byref(pol), ctypes.byref(spec), ctypes.byref(h))
        assert st == want, (pr.kind, pr.lg_p, pr.lg_l, polk, want)
        if st == sc.SC_OK:
            lib.sc_incident_free(h)


def test_ellipsoid_and_dipole_validation():
    lib = sc.load()
    q = sc.sc_quadrature(0, 8, 8, 1)
    h = ctypes.c_void_p()
    for c, e, rmax, want in [(14.0, 6.0, 12.0, sc.SC_OK), (14.0, 6.0, 12.9, sc.SC_ERR_INVALID),
                             (6.0, 6.0, 1.0, sc.SC_ERR_INVALID), (14.0, 0.0, 1.0, sc.SC_ERR_INVALID)]:
        st = lib.sc_mirror_ellipsoid(None, c, e, 0.0, rmax, ctypes.byref(q), ctypes.byref(h))
        assert st == want, (c, e, rmax)
        if st == sc.SC_OK:
            lib.sc_mirror_free(h)
    pol = sc.sc_polarization(0, 0.0)
    mono = sc.sc_spectrum(0, 1.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    gtime = sc.sc_spectrum(1, 3.0, 1.0, 0.1, 3, 1.0, 0, None, None, 0, None)
    for dip, spec, order, want in [((1.0, 0.0, 0.0), mono, 0, sc.SC_OK), ((0.0, 0.0, 0.0), mono, 0, sc.SC_ERR_INVALID),
                                   ((1.0, 0.0, 0.0), gtime, 0, sc.SC_ERR_INVALID),
                                   ((0.0, 1.0, 0.0), mono, 1, sc.SC_ERR_INVALID)]:
        prof = sc.sc_profile(5, 1.0, 4, 0, None, order, 0, 0, 0.0, None, None, 0.0, 0.0, 0.0,
                             (ctypes.c_double * 3)(*dip))
        st = lib.sc_incident(None, ctypes.byref(prof), ctypes.byref(pol), ctypes.byref(spec), ctypes.byref(h))
        assert st == want, (dip, order)
        if st == sc.SC_OK:
            lib.sc_incident_free(h)


def _incident(lib, beam, spec):
    keep = []
    prof = sc.sc_profile(sc.PROFILES[beam["profile"]], beam["w0"], beam.get("sg_order", 4), 0, None)
    pol = sc.sc_polarization(sc.POLS[beam.get("pol", "linear")], 0.0)
    phi = np.ascontiguousarray(spec.get("phi", []), dtype=np.float64)
    keep.append(phi)
    s = sc.sc_spectrum(sc.SPECTRA[spec["kind"]], spec.get("fwhm_t", 1.0), spec.get("lambda_c", 1.0),
                       spec.get("dlambda", 0.1), spec.get("sg_n", 3), spec.get("energy", 1.0), 0, None,
                       None, phi.size, phi.ctypes.data_as(sc._DP) if phi.size else None)
    h = ctypes.c_void_p()
    assert lib.sc_incident(None, ctypes.byref(prof), ctypes.byref(pol), ctypes.byref(s),
                           ctypes.byref(h)) == sc.SC_OK
    return h, keep


@pytest.mark.parametrize(
    "beam,spec",
    [
        (dict(profile="gauss", w0=37500.0), dict(kind="gauss_time", fwhm_t=3.7474, energy=2.0)),
        (dict(profile="supergauss", sg_order=4, w0=3.0, pol="radial"),
         dict(kind="supergauss_lambda", lambda_c=1.025, dlambda=0.0854, sg_n=3, energy=150.0,
              phi=[0.1, 0.5, 3.0, -2.0])),
        (dict(profile="tophat", w0=5.0, pol="azimuthal"), dict(kind="mono", phi=[0.3])),
    ],
)
def test_spectrum_generator_matches_oracle(beam, spec):
    """a_n = E0^n e^{i phi} (Eqs. 16, 18): the library's closed-form
    normalisations against the oracle's numerical quadratures."""
    lib = sc.load()
    h, keep = _incident(lib, beam, spec)
    om = np.linspace(0.5, 1.5, 101)
    out = np.zeros(om.size, dtype=np.complex128)
    assert lib.sc_spectrum_eval(None, h, om.ctypes.data_as(sc._DP), om.size,
                                out.view(np.float64).ctypes.data_as(sc._DP)) == sc.SC_OK
    lib.sc_incident_free(h)
    ref = oracle.spectrum(spec, om, beam)
    assert np.max(np.abs(out - ref)) <= 1e-9 * np.max(np.abs(ref))

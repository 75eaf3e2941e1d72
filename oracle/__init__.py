"""FP64 CPU oracle for the physical-optics Stratton-Chu focal field.

TEST INFRASTRUCTURE ONLY: the product path (the ``paper_1609_08146_gb300``
package and its CUDA library) never imports, links or runs anything here.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.

The arithmetic lives in ``sc_oracle.c`` (plain C, OpenMP over output
points), written from the paper's Sec. II Eq. 11 (reflected field in the
physical-optics approximation after Stokes' theorem), Eq. 10 with the
Appendix-A dyadic (independent double-gradient form), Sec. III.B Eqs. 13-18
(spectrum, amplitude normalisation, semi-discrete inverse transform) and
Sec. IV.B Eq. 27 (super-Gaussian spectrum).  This module only marshals
arguments.  Parity is pinned by ``tests/test_oracle_pins.py``.

Layouts: ``field`` returns complex arrays E, B of shape [n_omega, n_pts, 3].
Units: lambda0 = c = 1; omega in units of omega0; k = 2 pi omega.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_sc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, IEEE semantics, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Mirror(ctypes.Structure):
    _fields_ = [
        ("surface", ctypes.c_int),
        ("n_r", ctypes.c_int),
        ("n_theta", ctypes.c_int),
        ("rim", ctypes.c_int),
        ("f", ctypes.c_double),
        ("z0", ctypes.c_double),
        ("r_min", ctypes.c_double),
        ("r_max", ctypes.c_double),
        ("c_ell", ctypes.c_double),
        ("e_ell", ctypes.c_double),
        ("radial", ctypes.c_int),
    ]


class _Beam(ctypes.Structure):
    _fields_ = [
        ("profile", ctypes.c_int),
        ("sg_order", ctypes.c_int),
        ("pol", ctypes.c_int),
        ("n_zern", ctypes.c_int),
        ("w0", ctypes.c_double),
        ("pol_angle", ctypes.c_double),
        ("r_norm", ctypes.c_double),
        ("zern", ctypes.POINTER(ctypes.c_double)),
        ("order", ctypes.c_int),
        ("lg_p", ctypes.c_int),
        ("lg_l", ctypes.c_int),
        ("z_waist", ctypes.c_double),
        ("env_fn", ctypes.c_void_p),
        ("env_user", ctypes.c_void_p),
        ("dip", ctypes.c_double * 3),
        ("src", ctypes.c_double * 3),
        ("phase_ref", ctypes.c_double),
    ]


# fn(user, n, xyz[n][3], k, e[n][2][2]): the caller's envelope (profile "envelope")
ENVELOPE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.c_double, ctypes.POINTER(ctypes.c_double))


def envelope_callback(fn):
    """Wrap fn(xyz [n, 3], k) -> e [n, 2] complex (the transverse envelope
    e_perp at mirror points) as a C callback.  Keep the returned object alive
    while it is in use."""
    def _cb(user, n, xyz, k, out):
        pts = np.ctypeslib.as_array(xyz, shape=(n, 3))
        e = np.asarray(fn(pts.copy(), k), dtype=np.complex128).reshape(n, 2)
        np.ctypeslib.as_array(out, shape=(n, 4))[:] = e.view(np.float64)
    return ENVELOPE_FN(_cb)


PROFILES = {"gauss": 0, "supergauss": 1, "tophat": 2, "laguerre_gauss": 3, "envelope": 4, "dipole": 5}
POLS = {"linear": 0, "radial": 1, "azimuthal": 2}
SPECTRA = {"mono": 0, "gauss_time": 1, "supergauss_lambda": 2, "sampled": 3}
_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.or_gauss_legendre.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP, _DP]
        lib.or_simpson.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP, _DP]
        lib.or_zernike.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.or_zernike.restype = ctypes.c_double
        lib.or_beam_power.argtypes = [ctypes.POINTER(_Beam)]
        lib.or_beam_power.restype = ctypes.c_double
        lib.or_field.argtypes = [
            ctypes.POINTER(_Mirror), ctypes.POINTER(_Beam), ctypes.c_int, ctypes.c_int, _DP, _DP,
            ctypes.c_int, _DP, _DP, _DP, ctypes.c_int,
        ]
        lib.or_envelope.argtypes = [ctypes.POINTER(_Beam), ctypes.c_double, ctypes.c_int, _DP, _DP]
        lib.or_mfie_current.argtypes = [ctypes.POINTER(_Mirror), ctypes.POINTER(_Beam), ctypes.c_double,
                                        ctypes.c_int, _DP, ctypes.c_int, ctypes.c_int, _DP]
        lib.or_field_mfie.argtypes = [ctypes.POINTER(_Mirror), ctypes.POINTER(_Beam), ctypes.c_int, _DP, _DP,
                                      ctypes.c_int, _DP, ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.c_int]
        lib.or_mfie_sphere_te1.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _DP, ctypes.c_int,
                                           ctypes.c_int, _DP]
        lib.or_incident.argtypes = [
            ctypes.POINTER(_Beam), ctypes.c_double, ctypes.c_int, _DP, ctypes.c_int, _DP, _DP, _DP,
        ]
        lib.or_spectrum.argtypes = [
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
            ctypes.c_double, ctypes.c_double, ctypes.c_int, _DP, ctypes.c_int, _DP, _DP, _DP,
        ]
        lib.or_time_domain.argtypes = [
            ctypes.c_int, _DP, ctypes.c_long, _DP, ctypes.c_int, _DP, _DP, ctypes.c_int,
        ]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _mirror(m: dict) -> _Mirror:
    return _Mirror(
        surface={"paraboloid": 0, "flat": 1, "ellipsoid": 2}[m.get("surface", "paraboloid")],
        n_r=int(m["n_r"]), n_theta=int(m["n_theta"]), rim=int(m.get("rim", 1)),
        f=float(m.get("f", 1.0)), z0=float(m.get("z0", 0.0)),
        r_min=float(m.get("r_min", 0.0)), r_max=float(m["r_max"]),
        c_ell=float(m.get("c", 0.0)), e_ell=float(m.get("e", 0.0)),
        radial={"gauss_legendre": 0, "simpson": 1}[m.get("radial", "gauss_legendre")],
    )


def _beam(b: dict, keep: list) -> _Beam:
    z = np.ascontiguousarray(b.get("zernike", []), dtype=np.float64)
    keep.append(z)
    return _Beam(
        profile=PROFILES[b.get("profile", "gauss")], sg_order=int(b.get("sg_order", 4)),
        pol=POLS[b.get("pol", "linear")], n_zern=int(z.size), w0=float(b.get("w0", 1.0)),
        pol_angle=float(b.get("pol_angle", 0.0)), r_norm=float(b.get("r_norm", 1.0)),
        zern=_ptr(z) if z.size else None, order=int(b.get("order", 0)),
        lg_p=int(b.get("lg_p", 0)), lg_l=int(b.get("lg_l", 0)), z_waist=float(b.get("z_waist", 0.0)),
        env_fn=ctypes.cast(b["env_fn"], ctypes.c_void_p) if b.get("env_fn") is not None else None,
        env_user=None,
        dip=(ctypes.c_double * 3)(*b.get("dipole", (0.0, 0.0, 0.0))),
        src=(ctypes.c_double * 3)(*b.get("src", (0.0, 0.0, 0.0))),
        phase_ref=float(b.get("phase_ref", 0.0)),
    )


def dipole_beam(mirror: dict, p=(1.0, 0.0, 0.0)) -> dict:
    """The dipole of reading R16 at the upper focus F1 = (0, 0, 2e) of an
    ellipsoidal mirror, phase referred to the path length 2c."""
    return dict(profile="dipole", dipole=tuple(p), src=(0.0, 0.0, 2.0 * mirror["e"]),
                phase_ref=2.0 * mirror["c"], w0=1.0)


def gauss_legendre(n: int, a: float = -1.0, b: float = 1.0):
    """Gauss-Legendre nodes and weights on [a, b] (ascending)."""
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().or_gauss_legendre(n, a, b, _ptr(x), _ptr(w)) != 0:
        raise ValueError("n must be >= 1")
    return x, w


def simpson(n: int, a: float = -1.0, b: float = 1.0):
    """Composite Simpson nodes and weights on [a, b] (n odd >= 3)."""
    x = np.zeros(n)
    w = np.zeros(n)
    if _load().or_simpson(n, a, b, _ptr(x), _ptr(w)) != 0:
        raise ValueError("n must be odd and >= 3")
    return x, w


def zernike(j: int, rho: float, theta: float) -> float:
    """Noll-ordered, Noll-normalised Zernike polynomial Z_j(rho, theta)."""
    return _load().or_zernike(j, rho, theta)


def beam_power(beam: dict) -> float:
    """SS |f_E|^2 dA of the collimated beam over the transverse plane."""
    keep: list = []
    b = _beam(beam, keep)
    return _load().or_beam_power(ctypes.byref(b))


def field(mirror: dict, beam: dict, omegas, pts, amp=None, form: str = "stokes", threads: int = 0):
    """Reflected spectral field (E, B), each complex [n_omega, n_pts, 3].

    form="stokes" evaluates Eq. 11 (surface + boundary line integral);
    form="dyadic" evaluates Eq. 10 with the Appendix-A double gradient.
    amp: complex a_n per omega, or None for a_n = 1.
    """
    om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    a = None
    if amp is not None:
        a = np.ascontiguousarray(np.asarray(amp, dtype=np.complex128).view(np.float64))
    E = np.zeros((om.size, p.shape[0], 3), dtype=np.complex128)
    B = np.zeros_like(E)
    keep: list = []
    m = _mirror(mirror)
    b = _beam(beam, keep)
    rc = _load().or_field(
        ctypes.byref(m), ctypes.byref(b), {"stokes": 0, "dyadic": 1}[form], om.size, _ptr(om),
        _ptr(a), p.shape[0], _ptr(p), _ptr(E.view(np.float64)), _ptr(B.view(np.float64)),
        int(threads),
    )
    if rc != 0:
        raise ValueError("invalid mirror or beam parameters")
    return E, B


def envelope(beam: dict, k: float, pts):
    """Transverse envelope e_perp [n, 2] complex of a built-in beam (R4
    profiles or the Laguerre-Gauss mode of R15) at points [n, 3]."""
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    e = np.zeros((p.shape[0], 2), dtype=np.complex128)
    keep: list = []
    b = _beam(beam, keep)
    if _load().or_envelope(ctypes.byref(b), float(k), p.shape[0], _ptr(p), _ptr(e.view(np.float64))):
        raise ValueError("a caller's envelope is not sampled here")
    return e


def incident(beam: dict, omegas, pts, zref: float):
    """Incident field (E_inc, B_inc) [n_omega, n_pts, 3] of readings R4 / R14
    (beam["order"] = 1 adds the first-order longitudinal terms), unit a_n,
    phase reference exp(-ik(z + zref))."""
    om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    E = np.zeros((om.size, p.shape[0], 3), dtype=np.complex128)
    B = np.zeros_like(E)
    keep: list = []
    b = _beam(beam, keep)
    _load().or_incident(ctypes.byref(b), float(zref), om.size, _ptr(om), p.shape[0], _ptr(p),
                        _ptr(E.view(np.float64)), _ptr(B.view(np.float64)))
    return E, B


def spectrum(spec: dict, omegas, beam: dict | None = None):
    """Complex amplitudes a_n at the given omegas (Eqs. 14-18, 27)."""
    om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
    kind = SPECTRA[spec.get("kind", "mono")]
    phi = np.ascontiguousarray(spec.get("phi", []), dtype=np.float64)
    amp_in = None
    if kind == 3:
        amp_in = np.ascontiguousarray(np.asarray(spec["amp"], dtype=np.complex128).view(np.float64))
    P = beam_power(beam) if (beam is not None and kind in (1, 2)) else 1.0
    out = np.zeros(om.size, dtype=np.complex128)
    rc = _load().or_spectrum(
        kind, float(spec.get("fwhm_t", 1.0)), float(spec.get("lambda_c", 1.0)),
        float(spec.get("dlambda", 0.1)), int(spec.get("sg_n", 3)), float(spec.get("energy", 1.0)),
        P, phi.size, _ptr(phi) if phi.size else None, om.size, _ptr(om), _ptr(amp_in),
        _ptr(out.view(np.float64)),
    )
    if rc != 0:
        raise ValueError("bad spectrum")
    return out


def time_domain(F, omegas, times, threads: int = 0):
    """Semi-discrete inverse transform of F[n_omega, ...] -> real [n_t, ...]."""
    F = np.ascontiguousarray(F, dtype=np.complex128)
    om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
    t = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
    nv = int(np.prod(F.shape[1:]))
    out = np.zeros((t.size,) + F.shape[1:], dtype=np.float64)
    _load().or_time_domain(om.size, _ptr(om), nv, _ptr(F.view(np.float64)), t.size, _ptr(t),
                           _ptr(out), int(threads))
    return out


def mfie_current(mirror: dict, beam: dict, omega: float, targets_xy, n_rho: int, n_phi: int):
    """First MFIE correction dJ [n, 3] complex (Sec. II's Liouville-Neumann
    series: dJ = 2 n x PV SS J0 x grad g dS, J0 = 2 J_inc) at mirror points
    above targets_xy [n, 2], polar rule n_rho x n_phi about each target."""
    xy = np.ascontiguousarray(np.asarray(targets_xy, dtype=np.float64).reshape(-1, 2))
    out = np.zeros((xy.shape[0], 3), dtype=np.complex128)
    keep: list = []
    m = _mirror(mirror)
    b = _beam(beam, keep)
    if _load().or_mfie_current(ctypes.byref(m), ctypes.byref(b), 2.0 * np.pi * float(omega), xy.shape[0],
                               _ptr(xy), int(n_rho), int(n_phi), _ptr(out.view(np.float64))):
        raise ValueError("the MFIE correction needs a disk (r_min = 0) and a collimated beam of order 0")
    return out


def field_mfie(mirror: dict, beam: dict, omegas, pts, n_rho: int, n_phi: int, amp=None, threads: int = 0):
    """Physical-optics field (Eq. 11) plus the field of the first MFIE
    correction, E, B [n_omega, n_pts, 3] complex."""
    om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.float64).reshape(-1, 3))
    a = None
    if amp is not None:
        a = np.ascontiguousarray(np.asarray(amp, dtype=np.complex128).view(np.float64))
    E = np.zeros((om.size, p.shape[0], 3), dtype=np.complex128)
    B = np.zeros_like(E)
    keep: list = []
    m = _mirror(mirror)
    b = _beam(beam, keep)
    rc = _load().or_field_mfie(ctypes.byref(m), ctypes.byref(b), om.size, _ptr(om), _ptr(a), p.shape[0], _ptr(p),
                               int(n_rho), int(n_phi), _ptr(E.view(np.float64)), _ptr(B.view(np.float64)),
                               int(threads))
    if rc != 0:
        raise ValueError("invalid mirror or beam for the MFIE correction")
    return E, B


def mfie_sphere_te1(a: float, k: float, targets, n_psi: int, n_phi: int):
    """The MFIE operator K[J] = n x PV SS J x grad g dS on a sphere of radius
    a for J = z x r^, at unit-vector targets [n, 3] (test of the operator)."""
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(-1, 3))
    out = np.zeros((t.shape[0], 3), dtype=np.complex128)
    _load().or_mfie_sphere_te1(float(a), float(k), t.shape[0], _ptr(t), int(n_psi), int(n_phi),
                               _ptr(out.view(np.float64)))
    return out

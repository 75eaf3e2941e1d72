"""GB300-native evaluator of the physical-optics Stratton-Chu focal field.

Python binding of ``libsc`` (C-ABI in ``include/sc.h``): argument
marshalling only.  Every step of the field evaluation and of the inverse
transform runs in the library's own CUDA kernels for sm_103a; there is no
CPU or PyTorch fallback, and loading fails loudly when the library is
missing.  PyTorch provides device memory and the CUDA stream.

The paper (Dumont et al., arXiv:1609.08146) evaluates Sec. II Eq. 11 over a
parabolic mirror for every frequency of a short pulse and every point near
the focus, then rebuilds the time-domain field with Sec. III.B Eq. 13.

Low-level functions carry the C names (``sc_create``, ``sc_mirror``, ...);
``Context`` wraps them for tensors and numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

__all__ = ["load", "ScError", "Context", "Mirror", "Incident"]

SC_OK, SC_ERR_INVALID, SC_ERR_OOM, SC_ERR_CUDA, SC_ERR_TIMEOUT = 0, 1, 2, 3, 4
SC_ERR_BUSY, SC_ERR_CANCELLED, SC_ERR_NOT_FOUND = 5, 6, 7
SC_FP32_COMP, SC_FP64 = 0, 1
PROFILES = {"gauss": 0, "supergauss": 1, "tophat": 2, "laguerre_gauss": 3, "envelope": 4, "dipole": 5}
POLS = {"linear": 0, "radial": 1, "azimuthal": 2}
SPECTRA = {"mono": 0, "gauss_time": 1, "supergauss_lambda": 2, "sampled": 3}
SC_OPT_TIME_FIELD, SC_OPT_NODES_PER_SPLIT, SC_OPT_WORKSPACE_CAP, SC_OPT_FLUSH_NODES = 1, 2, 3, 4
SC_OPT_GRAPHS, SC_OPT_AUTOTUNE, SC_OPT_OMEGA_CHUNKS, SC_OPT_FAIL_COPY = 5, 6, 7, 8
SC_OPT_MFIE_ORDER, SC_OPT_MFIE_RHO, SC_OPT_MFIE_PHI, SC_OPT_CLASS_STREAMS = 9, 10, 11, 12
SC_OPT_TILE_LAYOUT, SC_OPT_SERVE_PRIORITY = 13, 14

_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


class sc_quadrature(ctypes.Structure):
    _fields_ = [("radial_kind", ctypes.c_int), ("n_r", ctypes.c_int), ("n_theta", ctypes.c_int),
                ("rim_term", ctypes.c_int)]


class sc_profile(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("w0", ctypes.c_double), ("sg_order", ctypes.c_int),
                ("n_zernike", ctypes.c_int), ("zernike_noll_waves", _DP), ("order", ctypes.c_int),
                ("lg_p", ctypes.c_int), ("lg_l", ctypes.c_int), ("z_waist", ctypes.c_double),
                ("envelope", ctypes.c_void_p), ("envelope_user", ctypes.c_void_p),
                ("omega_lo", ctypes.c_double), ("omega_hi", ctypes.c_double), ("fit_tol", ctypes.c_double),
                ("dipole", ctypes.c_double * 3)]


# sc_envelope_fn: (user, n, xyz[n][3], k, e[n][2][2])
ENVELOPE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.c_double, ctypes.POINTER(ctypes.c_double))


class sc_polarization(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("angle_rad", ctypes.c_double)]


class sc_spectrum(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("fwhm_t", ctypes.c_double), ("lambda_c", ctypes.c_double),
                ("dlambda", ctypes.c_double), ("sg_n", ctypes.c_int), ("energy", ctypes.c_double),
                ("n", ctypes.c_int), ("omega", _DP), ("amp_re_im", _DP), ("n_phi", ctypes.c_int),
                ("phi_taylor", _DP)]


class sc_eval_stats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_double), ("field_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("launches", ctypes.c_int), ("tables", ctypes.c_int),
                ("kernel_class", ctypes.c_int), ("threads_per_point", ctypes.c_int),
                ("omegas_per_thread", ctypes.c_int), ("splits", ctypes.c_int)]


def _stats_dict(st):
    return dict(evals=st.evals, field_ms=st.field_ms, total_ms=st.total_ms,
                launches=st.launches, tables=st.tables, kernel_class=st.kernel_class,
                threads_per_point=st.threads_per_point, omegas_per_thread=st.omegas_per_thread,
                splits=st.splits)


class sc_counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("field_launches", ctypes.c_uint64),
                ("field_ms", ctypes.c_double), ("evals", ctypes.c_double),
                ("graph_captures", ctypes.c_uint64), ("graph_replays", ctypes.c_uint64)]


class sc_request(ctypes.Structure):
    _fields_ = [("mirror", _VP), ("incident", _VP), ("omegas", _DP), ("n_omega", ctypes.c_int),
                ("points_xyz", _VP), ("n_points", ctypes.c_int), ("E_out", _VP), ("B_out", _VP)]


# C-ABI symbol table: name -> (restype, argtypes)
SIGNATURES = {
    "sc_create": (ctypes.c_int, [ctypes.c_int, _VP, ctypes.c_size_t, ctypes.POINTER(_VP)]),
    "sc_destroy": (ctypes.c_int, [_VP]),
    "sc_last_error": (ctypes.c_char_p, [_VP]),
    "sc_mirror": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(sc_quadrature), ctypes.POINTER(_VP)]),
    "sc_mirror_ellipsoid": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(sc_quadrature), ctypes.POINTER(_VP)]),
    "sc_eval_time_domain": (ctypes.c_int, [_VP, _VP, _VP, _DP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int,
                                           _DP, ctypes.c_int, ctypes.c_int, _VP, _VP,
                                           ctypes.POINTER(sc_eval_stats)]),
    "sc_table_count": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sc_mirror_free": (None, [_VP]),
    "sc_incident": (ctypes.c_int, [_VP, ctypes.POINTER(sc_profile), ctypes.POINTER(sc_polarization),
                                   ctypes.POINTER(sc_spectrum), ctypes.POINTER(_VP)]),
    "sc_incident_free": (None, [_VP]),
    "sc_spectrum_eval": (ctypes.c_int, [_VP, _VP, _DP, ctypes.c_int, _DP]),
    "sc_eval": (ctypes.c_int, [_VP, _VP, _VP, _DP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int,
                               _VP, _VP, ctypes.POINTER(sc_eval_stats)]),
    "sc_time_domain": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _DP, ctypes.c_int, ctypes.c_int,
                                      _DP, ctypes.c_int, _VP, _VP]),
    "sc_eval_fp32_static": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, _DP, _VP, ctypes.c_int, _VP, _VP]),
    "sc_eval_batch": (ctypes.c_int, [_VP, ctypes.POINTER(sc_request), ctypes.c_int,
                                     ctypes.POINTER(sc_eval_stats)]),
    "sc_submit": (ctypes.c_int, [_VP, ctypes.POINTER(sc_request), ctypes.POINTER(ctypes.c_uint64)]),
    "sc_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "sc_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_double]),
    "sc_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "sc_fetch": (ctypes.c_int, [_VP, ctypes.c_uint64, _VP, _VP]),
    "sc_release": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "sc_ticket_times": (ctypes.c_int, [_VP, ctypes.c_uint64, _DP, _DP, _DP]),
    "sc_selftest_wait": (ctypes.c_int, [_VP]),
    "sc_get_counters": (ctypes.c_int, [_VP, ctypes.POINTER(sc_counters)]),
    "sc_measure_alu_peaks": (ctypes.c_int, [_VP, _DP, _DP, _DP]),
    "sc_plan_omega_chunks": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sc_reset_counters": (ctypes.c_int, [_VP]),
    "sc_set_option": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_longlong]),
}

_lib = None


def load(path: str | None = None):
    """Load libsc (building it first when the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        from . import build as _build

        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libsc is not built (%s); run paper_1609_08146_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    globals().update({name: getattr(lib, name) for name in SIGNATURES})
    return lib


def plan_omega_chunks(n_omega: int, pairs_per_omega: int, ctx=None):
    """Omega chunk sizes the FP32 path uses for a request (no GPU needed)."""
    lib = load()
    sizes = (ctypes.c_int * (n_omega + 1))()
    n = ctypes.c_int()
    st = lib.sc_plan_omega_chunks(ctx._h if ctx is not None else None, int(n_omega), int(pairs_per_omega),
                                  sizes, n_omega + 1, ctypes.byref(n))
    if st != SC_OK:
        raise ScError(st, "sc_plan_omega_chunks failed")
    return list(sizes[: n.value])


class ScError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("sc status %d: %s" % (status, msg))
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _addr(x):
    """Device or host address of a torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


RADIAL_RULES = {"gauss_legendre": 0, "simpson": 1}


class Mirror:
    def __init__(self, ctx, f, r_min, r_max, n_r, n_theta, rim=True, ellipsoid=None, radial="gauss_legendre"):
        """Paraboloid of focal length f, or with ellipsoid=(c, e) the ellipsoidal
        cap of semi-axis c and focal half-distance e (f is then c - e).
        radial: "gauss_legendre" (n_r >= 1) or "simpson" (odd n_r >= 3)."""
        self._lib = ctx._lib
        q = sc_quadrature(RADIAL_RULES[radial], int(n_r), int(n_theta), 1 if rim else 0)
        h = _VP()
        if ellipsoid is None:
            ctx._check(self._lib.sc_mirror(ctx._h, float(f), float(r_min), float(r_max), ctypes.byref(q),
                                           ctypes.byref(h)))
        else:
            c, e = ellipsoid
            ctx._check(self._lib.sc_mirror_ellipsoid(ctx._h, float(c), float(e), float(r_min), float(r_max),
                                                     ctypes.byref(q), ctypes.byref(h)))
        self._h = h
        self.f, self.r_min, self.r_max, self.n_r, self.n_theta, self.rim = f, r_min, r_max, n_r, n_theta, rim
        self.radial = radial

    @property
    def n_nodes(self):
        return self.n_r * self.n_theta

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.sc_mirror_free(self._h)
            self._h = None


class Incident:
    def __init__(self, ctx, profile="gauss", w0=1.0, sg_order=4, zernike=(), pol="linear",
                 pol_angle=0.0, spectrum=None, order=0, lg_p=0, lg_l=0, z_waist=0.0,
                 omega_band=(0.0, 0.0), fit_tol=0.0, envelope=None, dipole=(0.0, 0.0, 0.0)):
        """profile "laguerre_gauss" (lg_p, lg_l, z_waist) or "envelope" (envelope:
        a function (xyz [n, 3], k) -> e_perp [n, 2] complex) need omega_band =
        (lo, hi) covering every omega evaluated later."""
        self._lib = ctx._lib
        spectrum = dict(spectrum or {"kind": "mono"})
        self._keep = []
        z = np.ascontiguousarray(zernike, dtype=np.float64)
        self._keep.append(z)
        self._cb = None
        if envelope is not None:
            def _cb(user, n, xyz, k, out, fn=envelope):
                pts = np.ctypeslib.as_array(xyz, shape=(n, 3)).copy()
                e = np.asarray(fn(pts, k), dtype=np.complex128).reshape(n, 2)
                np.ctypeslib.as_array(out, shape=(n, 4))[:] = e.view(np.float64)
            self._cb = ENVELOPE_FN(_cb)
        prof = sc_profile(PROFILES[profile], float(w0), int(sg_order), int(z.size),
                          _dptr(z) if z.size else None, int(order), int(lg_p), int(lg_l), float(z_waist),
                          ctypes.cast(self._cb, ctypes.c_void_p) if self._cb else None, None,
                          float(omega_band[0]), float(omega_band[1]), float(fit_tol),
                          (ctypes.c_double * 3)(*[float(v) for v in dipole]))
        pl = sc_polarization(POLS[pol], float(pol_angle))
        kind = SPECTRA[spectrum.get("kind", "mono")]
        om = amp = None
        n = 0
        if kind == 3:
            om = np.ascontiguousarray(spectrum["omega"], dtype=np.float64)
            amp = np.ascontiguousarray(np.asarray(spectrum["amp"], dtype=np.complex128).view(np.float64))
            n = om.size
            self._keep += [om, amp]
        phi = np.ascontiguousarray(spectrum.get("phi", []), dtype=np.float64)
        self._keep.append(phi)
        sp = sc_spectrum(kind, float(spectrum.get("fwhm_t", 1.0)), float(spectrum.get("lambda_c", 1.0)),
                         float(spectrum.get("dlambda", 0.1)), int(spectrum.get("sg_n", 3)),
                         float(spectrum.get("energy", 1.0)), n, _dptr(om) if om is not None else None,
                         _dptr(amp) if amp is not None else None, int(phi.size),
                         _dptr(phi) if phi.size else None)
        h = _VP()
        ctx._check(self._lib.sc_incident(ctx._h, ctypes.byref(prof), ctypes.byref(pl), ctypes.byref(sp),
                                         ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.sc_incident_free(self._h)
            self._h = None


class Context:
    """One libsc context bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None, budget_bytes: int = 0):
        import torch

        self._lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = device
        h = _VP()
        st = self._lib.sc_create(int(device), _VP(stream.cuda_stream), int(budget_bytes), ctypes.byref(h))
        if st != SC_OK:
            raise ScError(st, "sc_create failed")
        self._h = h

    def _check(self, st):
        if st != SC_OK:
            raise ScError(st, self._lib.sc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def mirror(self, f, r_min, r_max, n_r, n_theta, rim=True, radial="gauss_legendre") -> Mirror:
        return Mirror(self, f, r_min, r_max, n_r, n_theta, rim, radial=radial)

    def ellipsoid(self, c, e, r_min, r_max, n_r, n_theta, rim=True, radial="gauss_legendre") -> Mirror:
        return Mirror(self, c - e, r_min, r_max, n_r, n_theta, rim, ellipsoid=(c, e), radial=radial)

    def incident(self, **kw) -> Incident:
        return Incident(self, **kw)

    def set_option(self, option: int, value: int):
        self._check(self._lib.sc_set_option(self._h, int(option), int(value)))

    def spectrum(self, inc: Incident, omegas) -> np.ndarray:
        om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
        out = np.zeros(om.size, dtype=np.complex128)
        self._check(self._lib.sc_spectrum_eval(self._h, inc._h, _dptr(om), om.size,
                                               _dptr(out.view(np.float64))))
        return out

    def eval(self, mirror: Mirror, inc: Incident, omegas, points, precision: str = "fp32",
             out=None, stats: bool = False):
        """Spectral field E, B [n_omega, n_pts, 3] (complex64 for "fp32",
        complex128 for "fp64").  ``points``: torch tensor (cuda -> device
        outputs) or numpy array (host outputs), [n_pts, 3] float64."""
        import torch

        om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
        prec = SC_FP32_COMP if precision == "fp32" else SC_FP64
        if isinstance(points, np.ndarray):
            pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
            npts = pts.shape[0]
            if out is None:
                dt = np.complex64 if prec == SC_FP32_COMP else np.complex128
                E = np.empty((om.size, npts, 3), dtype=dt)
                B = np.empty_like(E)
            else:
                E, B = out
        else:  # torch tensor on the device or in (pinned) host memory
            pts = points.contiguous()
            if pts.dtype != torch.float64:
                pts = pts.to(torch.float64)
            npts = pts.shape[0]
            if out is None:
                dt = torch.complex64 if prec == SC_FP32_COMP else torch.complex128
                E = torch.empty((om.size, npts, 3), dtype=dt, device=pts.device,
                                pin_memory=not pts.is_cuda and pts.is_pinned())
                B = torch.empty_like(E)
            else:
                E, B = out
        st = sc_eval_stats()
        self._check(self._lib.sc_eval(self._h, mirror._h, inc._h, _dptr(om), om.size, _addr(pts),
                                      npts, prec, _addr(E), _addr(B) if B is not None else None,
                                      ctypes.byref(st) if stats else None))
        if stats:
            return E, B, _stats_dict(st)
        return E, B

    def eval_time_domain(self, mirror: Mirror, inc: Incident, omegas, points, times, precision: str = "fp32",
                         omega_chunk: int = 0, with_B: bool = True, stats: bool = False):
        """E(t), B(t) float32 [n_t, n_pts, 3] straight from the mirror integrals,
        holding one chunk of spectra at a time (sc_eval_time_domain).  ``points``:
        torch tensor (cuda -> device outputs) or numpy array (host outputs)."""
        import torch

        om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
        tt = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
        prec = SC_FP32_COMP if precision == "fp32" else SC_FP64
        if isinstance(points, np.ndarray):
            pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
            Et = np.empty((tt.size, pts.shape[0], 3), dtype=np.float32)
            Bt = np.empty_like(Et) if with_B else None
        else:
            pts = points.contiguous().to(torch.float64)
            Et = torch.empty((tt.size, pts.shape[0], 3), dtype=torch.float32, device=pts.device)
            Bt = torch.empty_like(Et) if with_B else None
        st = sc_eval_stats()
        self._check(self._lib.sc_eval_time_domain(self._h, mirror._h, inc._h, _dptr(om), om.size, _addr(pts),
                                                  pts.shape[0], prec, _dptr(tt), tt.size, int(omega_chunk),
                                                  _addr(Et), _addr(Bt) if Bt is not None else None,
                                                  ctypes.byref(st) if stats else None))
        if stats:
            return Et, Bt, _stats_dict(st)
        return Et, Bt

    def time_domain(self, E, B, omegas, times, precision: str = "fp32", out=None):
        """Inverse transform of spectra [n_omega, n_pts, 3] -> float32
        [n_t, n_pts, 3] on the spectra's side (device or host)."""
        import torch

        om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
        t = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
        prec = SC_FP32_COMP if precision == "fp32" else SC_FP64
        npts = E.shape[1]
        if out is None:
            if isinstance(E, np.ndarray):
                Et = np.empty((t.size, npts, 3), dtype=np.float32)
                Bt = np.empty_like(Et) if B is not None else None
            else:
                Et = torch.empty((t.size, npts, 3), dtype=torch.float32, device=E.device)
                Bt = torch.empty_like(Et) if B is not None else None
        else:
            Et, Bt = out
        self._check(self._lib.sc_time_domain(self._h, prec, _addr(E), _addr(B) if B is not None else None,
                                             _dptr(om), om.size, npts, _dptr(t), t.size, _addr(Et),
                                             _addr(Bt) if Bt is not None else None))
        return Et, Bt

    def eval_batch(self, requests, stats: bool = False):
        """Evaluate many requests in one scheduled pass (FP32 path).

        requests: list of (mirror, incident, omegas, points) with points a
        cuda float64 tensor [n, 3]; returns a list of (E, B) complex64
        device tensors [n_omega, n, 3]."""
        import torch

        arr = (sc_request * len(requests))()
        keep, outs = [], []
        for i, (m, inc, om, pts) in enumerate(requests):
            om = np.ascontiguousarray(np.atleast_1d(om), dtype=np.float64)
            pts = pts.contiguous()
            E = torch.empty((om.size, pts.shape[0], 3), dtype=torch.complex64, device=pts.device)
            B = torch.empty_like(E)
            keep += [om, pts]
            outs.append((E, B))
            arr[i] = sc_request(m._h, inc._h, _dptr(om), om.size, _VP(pts.data_ptr()), pts.shape[0],
                                _VP(E.data_ptr()), _VP(B.data_ptr()))
        st = sc_eval_stats()
        self._check(self._lib.sc_eval_batch(self._h, arr, len(requests),
                                            ctypes.byref(st) if stats else None))
        if stats:
            return outs, _stats_dict(st)
        return outs

    # ---- serving
    def submit(self, mirror, inc, omegas, points, out=None):
        """Queue one request; returns its ticket.  points: numpy (host,
        copied) or cuda tensor (kept by reference); out: optional (E, B)
        caller-owned complex64 cuda tensors, else server-owned outputs."""
        om = np.ascontiguousarray(np.atleast_1d(omegas), dtype=np.float64)
        if isinstance(points, np.ndarray):
            pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
            paddr, n = pts.ctypes.data, pts.shape[0]
        else:
            pts = points.contiguous()
            paddr, n = pts.data_ptr(), pts.shape[0]
        E = B = None
        if out is not None:
            E, B = out
        req = sc_request(mirror._h, inc._h, _dptr(om), om.size, _VP(paddr), n,
                         _VP(E.data_ptr()) if E is not None else None,
                         _VP(B.data_ptr()) if B is not None else None)
        t = ctypes.c_uint64()
        self._check(self._lib.sc_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._serving_keep = getattr(self, "_serving_keep", {})
        self._serving_keep[t.value] = (om, pts, E, B, n)
        return t.value

    def poll(self, ticket) -> bool:
        d = ctypes.c_int()
        self._check(self._lib.sc_poll(self._h, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket, timeout_s: float = 60.0):
        self._check(self._lib.sc_wait(self._h, ticket, float(timeout_s)))

    def cancel(self, ticket):
        self._check(self._lib.sc_cancel(self._h, ticket))

    def fetch(self, ticket, device="cuda"):
        """Results of a finished request as complex64 tensors [n_omega, n, 3]."""
        import torch

        om, _, _, _, n = self._serving_keep[ticket]
        E = torch.empty((om.size, n, 3), dtype=torch.complex64, device=device)
        B = torch.empty_like(E)
        self._check(self._lib.sc_fetch(self._h, ticket, _VP(E.data_ptr()), _VP(B.data_ptr())))
        return E, B

    def release(self, ticket):
        self._check(self._lib.sc_release(self._h, ticket))
        getattr(self, "_serving_keep", {}).pop(ticket, None)

    def ticket_times(self, ticket):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.sc_ticket_times(self._h, ticket, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c)))
        return a.value, b.value, c.value

    def counters(self):
        c = sc_counters()
        self._check(self._lib.sc_get_counters(self._h, ctypes.byref(c)))
        return dict(launches=c.launches, field_launches=c.field_launches, field_ms=c.field_ms,
                    evals=c.evals, graph_captures=c.graph_captures, graph_replays=c.graph_replays)

    def measure_alu_peaks(self):
        """Measured FP32 FMA, packed FFMA2 and MUFU throughput of this device
        (operations per second; lane-ops for the FMA forms)."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.sc_measure_alu_peaks(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(fp32_lane_ops_per_s=a.value, fp32x2_lane_ops_per_s=b.value, mufu_ops_per_s=c.value)

    def plan_omega_chunks(self, n_omega: int, pairs_per_omega: int):
        """Omega chunk sizes of a request (host planning, see sc_plan_omega_chunks)."""
        return plan_omega_chunks(n_omega, pairs_per_omega, self)

    def reset_counters(self):
        self._check(self._lib.sc_reset_counters(self._h))

"""ctypes front end of the FP64 CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py are the only callers.
This module imports nothing from the CUDA package; configurations reach it as
any object with the attribute names below (duck typing), so the two sides share
no code.

Arrays are numpy ``complex128``; field arrays have shape ``(F, N)`` with row
0 = pump, 1 = signal, 2 = idler (Sec. 2.1 of arXiv 2410.02532).
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


class Crystal(ctypes.Structure):
    """Mirror of ``orc_crystal`` in opo_oracle.h."""
    _fields_ = [
        ("length", ctypes.c_double),
        ("nz", ctypes.c_int32),
        ("dk", ctypes.c_double),
        ("deff", ctypes.c_double),
        ("nidx", ctypes.c_double * 3),
        ("alpha", ctypes.c_double * 3),
        ("dbeta1", ctypes.c_double * 3),
        ("beta2", ctypes.c_double * 3),
        ("beta3", ctypes.c_double * 3),
        ("beta4", ctypes.c_double * 3),
        ("tod_div", ctypes.c_double),
        ("n2", ctypes.c_double),
    ]


MAX_EXTRA = 7


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in opo_oracle.h."""
    _fields_ = [
        ("n", ctypes.c_int32),
        ("nfields", ctypes.c_int32),
        ("t_window", ctypes.c_double),
        ("length", ctypes.c_double),
        ("nz", ctypes.c_int32),
        ("dk", ctypes.c_double),
        ("deff", ctypes.c_double),
        ("lambda_", ctypes.c_double * 3),
        ("nidx", ctypes.c_double * 3),
        ("alpha", ctypes.c_double * 3),
        ("dbeta1", ctypes.c_double * 3),
        ("beta2", ctypes.c_double * 3),
        ("beta3", ctypes.c_double * 3),
        ("tod_div", ctypes.c_double),
        ("w0", ctypes.c_double),
        ("resonant_mask", ctypes.c_uint32),
        ("R", ctypes.c_double * 3),
        ("delta", ctypes.c_double * 3),
        ("gdd", ctypes.c_double * 3),
        ("delay", ctypes.c_double),
        ("eom_beta", ctypes.c_double),
        ("eom_f", ctypes.c_double),
        ("t_rt", ctypes.c_double),
        ("ns_a0", ctypes.c_double),
        ("ns_fwhm", ctypes.c_double),
        ("ns_t0", ctypes.c_double),
        ("beta4", ctypes.c_double * 3),
        ("n2", ctypes.c_double),
        ("nextra", ctypes.c_int32),
        ("extra", Crystal * MAX_EXTRA),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.POINTER(Params)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_fft.argtypes = [_D, ctypes.c_int32, ctypes.c_int32]
        L.orc_fft.restype = ctypes.c_int
        L.orc_kappa.argtypes = [_P, _D]
        L.orc_omega.argtypes = [_P, ctypes.c_int32]
        L.orc_omega.restype = ctypes.c_double
        L.orc_linear_step.argtypes = [_P, _D, ctypes.c_double]
        L.orc_rk4_step.argtypes = [_P, _D, ctypes.c_double, ctypes.c_double]
        L.orc_crystal_pass.argtypes = [_P, _D]
        L.orc_crystal_k.argtypes = [_P, ctypes.c_int32, _P]
        L.orc_pump_profile.argtypes = [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _D]
        L.orc_power.argtypes = [_P, ctypes.c_int32, _D]
        L.orc_power.restype = ctypes.c_double
        L.orc_centroid.argtypes = [_P, _D]
        L.orc_centroid.restype = ctypes.c_double
        L.orc_cavity.argtypes = [_P, _D, ctypes.c_int64]
        L.orc_pump_slice.argtypes = [_P, _D, ctypes.c_int64, _D]
        L.orc_run.argtypes = [_P, _D, _D, ctypes.c_int64, ctypes.c_int64, _D, _D]
        L.orc_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _trip(v):
    v = list(v) + [0.0] * (3 - len(v))
    return (ctypes.c_double * 3)(*[float(t) for t in v[:3]])


def params(cfg, tod_div=6.0):
    """Build ``orc_params`` from a configuration object (attribute access)."""
    g = lambda name, default=0.0: getattr(cfg, name, default)  # noqa: E731
    p = Params()
    p.n = int(cfg.n)
    p.nfields = int(cfg.nfields)
    p.t_window = float(cfg.t_window)
    p.length = float(cfg.length)
    p.nz = int(cfg.nz)
    p.dk = float(g("dk"))
    p.deff = float(cfg.deff)
    p.lambda_ = _trip(cfg.lam)
    p.nidx = _trip(cfg.nidx)
    p.alpha = _trip(g("alpha", (0, 0, 0)))
    p.dbeta1 = _trip(g("dbeta1", (0, 0, 0)))
    p.beta2 = _trip(g("beta2", (0, 0, 0)))
    p.beta3 = _trip(g("beta3", (0, 0, 0)))
    p.beta4 = _trip(g("beta4", (0, 0, 0)))
    p.n2 = float(g("n2"))
    p.tod_div = float(tod_div)
    p.w0 = float(g("w0", 55e-6))
    p.resonant_mask = int(cfg.resonant_mask)
    p.R = _trip(g("R", (0, 0, 0)))
    p.delta = _trip(g("delta", (0, 0, 0)))
    p.gdd = _trip(g("gdd", (0, 0, 0)))
    p.delay = float(g("delay"))
    p.eom_beta = float(g("eom_beta"))
    p.eom_f = float(g("eom_f"))
    p.t_rt = float(g("t_rt", cfg.t_window))
    if int(g("pump_kind", 0)) == 3:  # ns-pulsed pump
        inten = float(cfg.pump_power) / (3.141592653589793 * p.w0 * p.w0)
        p.ns_a0 = (2.0 * inten / (p.nidx[0] * 8.8541878128e-12 * 299792458.0)) ** 0.5
        p.ns_fwhm = float(cfg.pump_fwhm)
        p.ns_t0 = float(g("pump_t0"))
    # further crystals: objects with the crystal attribute names above
    extra = list(g("extra_crystals", ()))
    if len(extra) > MAX_EXTRA:
        raise ValueError("at most %d extra crystals" % MAX_EXTRA)
    p.nextra = len(extra)
    for i, c in enumerate(extra):
        e = p.extra[i]
        e.length = float(c.length)
        e.nz = int(c.nz)
        e.dk = float(getattr(c, "dk", 0.0))
        e.deff = float(c.deff)
        e.nidx = _trip(c.nidx)
        e.alpha = _trip(getattr(c, "alpha", (0, 0, 0)))
        e.dbeta1 = _trip(getattr(c, "dbeta1", (0, 0, 0)))
        e.beta2 = _trip(getattr(c, "beta2", (0, 0, 0)))
        e.beta3 = _trip(getattr(c, "beta3", (0, 0, 0)))
        e.beta4 = _trip(getattr(c, "beta4", (0, 0, 0)))
        e.tod_div = float(tod_div)
        e.n2 = float(getattr(c, "n2", 0.0))
    return p


def _ptr(a):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def fft(x, direction=-1):
    """DFT with the oracle's own radix-2 code; ``direction=+1`` is the
    inverse including 1/N."""
    a = _c(x).copy()
    if lib().orc_fft(_ptr(a), a.size, int(direction)) != 0:
        raise ValueError("length must be a power of two")
    return a


def kappa(p):
    out = (ctypes.c_double * 3)()
    lib().orc_kappa(ctypes.byref(p), out)
    return np.array(out[:])


def omega(p):
    return np.array([lib().orc_omega(ctypes.byref(p), k) for k in range(p.n)])


def linear_step(p, fields, dz):
    a = _c(fields).copy()
    lib().orc_linear_step(ctypes.byref(p), _ptr(a), float(dz))
    return a


def rk4_step(p, fields, z0, h):
    a = _c(fields).copy()
    lib().orc_rk4_step(ctypes.byref(p), _ptr(a), float(z0), float(h))
    return a


def crystal_pass(p, fields):
    a = _c(fields).copy()
    lib().orc_crystal_pass(ctypes.byref(p), _ptr(a))
    return a


def crystal_k(p, k):
    """Params with the crystal fields of crystal k (0: the first)."""
    q = Params()
    lib().orc_crystal_k(ctypes.byref(p), int(k), ctypes.byref(q))
    return q


def pump_profile(p, kind, power, fwhm=0.0):
    out = np.zeros(p.n, dtype=np.complex128)
    lib().orc_pump_profile(ctypes.byref(p), int(kind), float(power), float(fwhm), _ptr(out))
    return out


def power(p, field, a):
    a = _c(a)
    return lib().orc_power(ctypes.byref(p), int(field), _ptr(a))


def centroid(p, a):
    a = _c(a)
    return lib().orc_centroid(ctypes.byref(p), _ptr(a))


def cavity(p, fields, m=0):
    a = _c(fields).copy()
    lib().orc_cavity(ctypes.byref(p), _ptr(a), int(m))
    return a


def pump_slice(p, pump_in, m):
    out = np.zeros(p.n, dtype=np.complex128)
    pin = _c(pump_in) if pump_in is not None else np.zeros(p.n, dtype=np.complex128)
    lib().orc_pump_slice(ctypes.byref(p), _ptr(pin), int(m), _ptr(out))
    return out


def run(p, fields, pump_in, m0=0, M=1):
    """Round trips ``m0 .. m0+M-1``.  Returns ``(fields, trace, out_fields,
    status)``; trace rows are ``(P_p, P_s, P_i, nu_c)``.  ``pump_in`` may be
    None for an ns-pulsed pump."""
    a = _c(fields).copy()
    pin = _c(pump_in) if pump_in is not None else np.zeros(p.n, dtype=np.complex128)
    trace = np.zeros((max(int(M), 1), 4), dtype=np.float64)
    out = np.zeros_like(a)
    st = lib().orc_run(ctypes.byref(p), _ptr(a), _ptr(pin), int(m0), int(M),
                       trace.ctypes.data_as(_D), _ptr(out))
    return a, trace[: int(M)], out, int(st)


__all__ = ["Params", "Crystal", "params", "fft", "kappa", "omega", "linear_step", "rk4_step",
           "crystal_pass", "crystal_k", "pump_profile", "pump_slice", "power", "centroid",
           "cavity", "run", "lib"]


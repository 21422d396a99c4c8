"""ctypes binding of ``libopo.so`` (C ABI in include/opo.h).

Argument marshalling only: every step of the split-step path runs in the
library's CUDA kernels.  The functions keep the C names (``opo_create``,
``opo_set_crystal``, ...) and raise :class:`OPOError` on a non-OK status.
There is no CPU fallback: :func:`lib` raises if the library is missing.

:class:`Context` wraps one instance built from a
:class:`paper_2410_02532_gb300.workloads.OPOConfig`.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libopo.so")

OPO_OK, OPO_E_INVALID, OPO_E_NOMEM, OPO_E_CUDA = 0, 1, 2, 3
OPO_E_NONFINITE, OPO_E_TIMEOUT, OPO_E_STATE, OPO_E_UNSUPPORTED = 4, 5, 6, 7
OPO_FP64, OPO_FP32_PH64 = 0, 1
OPO_PUMP_CW, OPO_PUMP_SECH2, OPO_PUMP_USER, OPO_PUMP_NS = 0, 1, 2, 3
OPO_INTRACAVITY, OPO_OUTPUT = 0, 1
OPO_PATH_AUTO, OPO_PATH_PLAIN, OPO_PATH_FUSED = 0, 1, 2

_D3 = ctypes.c_double * 3


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("t_window_s", ctypes.c_double),
                ("nfields", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("device", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class Crystal(ctypes.Structure):
    _fields_ = [("length_m", ctypes.c_double), ("nz", ctypes.c_int32),
                ("dk_per_m", ctypes.c_double), ("deff_mpv", ctypes.c_double),
                ("lambda_m", _D3), ("n", _D3), ("alpha_per_m", _D3),
                ("dbeta1_s_per_m", _D3), ("beta2_s2_per_m", _D3), ("beta3_s3_per_m", _D3),
                ("w0_m", ctypes.c_double), ("tod_div", ctypes.c_double),
                ("beta4_s4_per_m", _D3), ("n2_m2_per_W", ctypes.c_double)]


class Cavity(ctypes.Structure):
    _fields_ = [("resonant_mask", ctypes.c_uint32), ("R", _D3), ("delta_rad", _D3),
                ("gdd_s2", _D3), ("delay_s", ctypes.c_double), ("eom_beta_rad", ctypes.c_double),
                ("eom_f_hz", ctypes.c_double), ("t_rt_s", ctypes.c_double),
                ("pump_kind", ctypes.c_int32), ("pump_power_W", ctypes.c_double),
                ("pump_fwhm_s", ctypes.c_double), ("pump_user", ctypes.POINTER(ctypes.c_double)),
                ("pump_t0_s", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("rt_done", ctypes.c_int64), ("p_out_W", _D3), ("centroid_hz", ctypes.c_double),
                ("p_out_mean_W", _D3), ("centroid_mean_hz", ctypes.c_double),
                ("path", ctypes.c_int32), ("cluster", ctypes.c_int32)]


class OPOError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, status_string(status), status))


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "opo_validate": ([ctypes.POINTER(Grid), ctypes.POINTER(Crystal), ctypes.c_int32,
                      ctypes.POINTER(Cavity)], ctypes.c_int),
    "opo_create": ([ctypes.POINTER(_P), ctypes.POINTER(Grid)], ctypes.c_int),
    "opo_set_crystal": ([_P, ctypes.POINTER(Crystal)], ctypes.c_int),
    "opo_set_crystals": ([_P, ctypes.POINTER(Crystal), ctypes.c_int32], ctypes.c_int),
    "opo_set_cavity": ([_P, ctypes.POINTER(Cavity)], ctypes.c_int),
    "opo_set_fields": ([_P, ctypes.c_int32, _DP, ctypes.c_size_t, ctypes.c_int64], ctypes.c_int),
    "opo_run_roundtrips": ([_P, ctypes.c_int64, ctypes.POINTER(Stats)], ctypes.c_int),
    "opo_get_fields": ([_P, ctypes.c_int32, ctypes.c_int32, _DP, ctypes.c_size_t], ctypes.c_int),
    "opo_get_trace": ([_P, _DP, ctypes.c_int64], ctypes.c_int),
    "opo_set_output_history": ([_P, ctypes.c_int64], ctypes.c_int),
    "opo_get_output_history": ([_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _DP],
                               ctypes.c_int),
    "opo_set_fields_device": ([_P, ctypes.c_int32, _P, ctypes.c_size_t, ctypes.c_int64],
                              ctypes.c_int),
    "opo_get_fields_device": ([_P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t],
                              ctypes.c_int),
    "opo_set_path": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
                     ctypes.c_int),
    "opo_sync": ([_P], ctypes.c_int),
    "opo_fused_capacity": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "opo_destroy": ([_P], ctypes.c_int),
    "opo_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "opo_batch_create": ([ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_int32], ctypes.c_int),
    "opo_batch_run": ([_P, ctypes.c_int64], ctypes.c_int),
    "opo_batch_set_one_launch": ([_P, ctypes.c_int32], ctypes.c_int),
    "opo_batch_destroy": ([_P], ctypes.c_int),
    "opo_batch_set_fields": ([_P, _DP, ctypes.c_size_t], ctypes.c_int),
    "opo_batch_get_fields": ([_P, ctypes.c_int32, ctypes.c_int32, _DP, ctypes.c_size_t],
                             ctypes.c_int),
    "opo_batch_get_trace": ([_P, _DP, ctypes.c_int64], ctypes.c_int),
    "opo_batch_step_io": ([_P, _DP, _DP, ctypes.c_int32, ctypes.c_int64], ctypes.c_int),
    "opo_batch_io_wait": ([_P], ctypes.c_int),
}


def lib():
    """Load libopo.so; raises if it has not been built (no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libopo.so is not built (run __graft_entry__.build()); "
                               "the OPO path has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().opo_status_string(int(status)).decode()
    except Exception:  # library not loadable: still report the number
        return "status"


def _check(st, where):
    if st != OPO_OK:
        raise OPOError(st, where)


def _cplx_in(a, n):
    a = np.ascontiguousarray(a, dtype=np.complex128).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d complex values, got %d" % (n, a.size))
    return a


# ---- thin wrappers with the C names ----------------------------------------

def opo_validate(grid: Grid, crystals=(), cavity=None) -> int:
    """Status of the configuration's checks (no GPU involved): OPO_OK or
    OPO_E_INVALID."""
    arr = (Crystal * len(crystals))(*crystals) if crystals else None
    return lib().opo_validate(ctypes.byref(grid), arr, len(crystals),
                              ctypes.byref(cavity) if cavity is not None else None)


def opo_create(grid: Grid):
    h = _P()
    _check(lib().opo_create(ctypes.byref(h), ctypes.byref(grid)), "opo_create")
    return h


def opo_set_crystal(ctx, crystal: Crystal):
    _check(lib().opo_set_crystal(ctx, ctypes.byref(crystal)), "opo_set_crystal")


def opo_set_crystals(ctx, crystals):
    arr = (Crystal * len(crystals))(*crystals)
    _check(lib().opo_set_crystals(ctx, arr, len(crystals)), "opo_set_crystals")


def opo_set_cavity(ctx, cavity: Cavity):
    _check(lib().opo_set_cavity(ctx, ctypes.byref(cavity)), "opo_set_cavity")


def opo_set_fields(ctx, field: int, values, rt_index: int = -1):
    a = _cplx_in(values, np.asarray(values).size)
    _check(lib().opo_set_fields(ctx, int(field), a.ctypes.data_as(_DP), a.size, int(rt_index)),
           "opo_set_fields")


def opo_run_roundtrips(ctx, m: int, want_stats: bool = False):
    if want_stats:
        s = Stats()
        _check(lib().opo_run_roundtrips(ctx, int(m), ctypes.byref(s)), "opo_run_roundtrips")
        return s
    _check(lib().opo_run_roundtrips(ctx, int(m), None), "opo_run_roundtrips")
    return None


def opo_get_fields(ctx, field: int, which: int, n: int):
    out = np.empty(int(n), dtype=np.complex128)
    _check(lib().opo_get_fields(ctx, int(field), int(which), out.ctypes.data_as(_DP), out.size),
           "opo_get_fields")
    return out


def opo_get_trace(ctx, rows: int):
    out = np.empty((int(rows), 4), dtype=np.float64)
    _check(lib().opo_get_trace(ctx, out.ctypes.data_as(_DP), int(rows)), "opo_get_trace")
    return out


def opo_set_output_history(ctx, max_rt):
    _check(lib().opo_set_output_history(ctx, int(max_rt)), "opo_set_output_history")


def opo_get_output_history(ctx, field, row0, rows, n):
    out = np.zeros((int(rows), int(n)), dtype=np.complex128)
    _check(lib().opo_get_output_history(ctx, int(field), int(row0), int(rows),
                                        out.ctypes.data_as(_DP)), "opo_get_output_history")
    return out


def opo_set_fields_device(ctx, field: int, dev_ptr: int, n: int, rt_index: int = -1):
    _check(lib().opo_set_fields_device(ctx, int(field), ctypes.c_void_p(dev_ptr), int(n),
                                       int(rt_index)), "opo_set_fields_device")


def opo_get_fields_device(ctx, field: int, which: int, dev_ptr: int, n: int):
    _check(lib().opo_get_fields_device(ctx, int(field), int(which), ctypes.c_void_p(dev_ptr),
                                       int(n)), "opo_get_fields_device")


def opo_set_path(ctx, path: int, cluster: int = 0, rt_per_launch: int = 0, threads: int = 0):
    _check(lib().opo_set_path(ctx, int(path), int(cluster), int(rt_per_launch), int(threads)),
           "opo_set_path")


def opo_fused_capacity(ctx, cluster: int = 0, threads: int = 0):
    """(max co-resident clusters, cluster size) of the fused path."""
    a, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().opo_fused_capacity(ctx, int(cluster), int(threads), ctypes.byref(a),
                                    ctypes.byref(c)), "opo_fused_capacity")
    return a.value, c.value


def opo_sync(ctx):
    _check(lib().opo_sync(ctx), "opo_sync")


def opo_destroy(ctx):
    lib().opo_destroy(ctx)


def opo_batch_create(ctxs, cluster: int = 0, threads: int = 0):
    arr = (_P * len(ctxs))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    h = _P()
    _check(lib().opo_batch_create(ctypes.byref(h), arr, len(ctxs), int(cluster), int(threads)),
           "opo_batch_create")
    return h


def opo_batch_run(batch, m: int):
    _check(lib().opo_batch_run(batch, int(m)), "opo_batch_run")


def opo_batch_set_one_launch(batch, on=True):
    _check(lib().opo_batch_set_one_launch(batch, 1 if on else 0), "opo_batch_set_one_launch")


def opo_batch_destroy(batch):
    lib().opo_batch_destroy(batch)


def opo_batch_set_fields(batch, host):
    """host: complex128 array holding every member's F x N fields in batch
    order (a flat array of sum F N values, or anything that flattens to it;
    a pinned contiguous buffer avoids a staging copy in the CUDA runtime)."""
    a = np.ascontiguousarray(host, dtype=np.complex128).reshape(-1)
    _check(lib().opo_batch_set_fields(batch, a.ctypes.data_as(_DP), a.size),
           "opo_batch_set_fields")


def opo_batch_get_fields(batch, field, which, total_n):
    out = np.empty(int(total_n), dtype=np.complex128)
    _check(lib().opo_batch_get_fields(batch, int(field), int(which), out.ctypes.data_as(_DP),
                                      out.size), "opo_batch_get_fields")
    return out


def opo_batch_get_trace(batch, count, rows):
    out = np.empty((int(count), int(rows), 4), dtype=np.float64)
    _check(lib().opo_batch_get_trace(batch, out.ctypes.data_as(_DP), int(rows)),
           "opo_batch_get_trace")
    return out


def opo_batch_step_io(batch, host_in, host_out, field, m=1):
    """One batch step with overlapped host transfers (returns at once).
    host_in / host_out: raw addresses (int) of page-locked double buffers, or
    None; they must stay untouched until opo_batch_io_wait returns."""
    _check(lib().opo_batch_step_io(batch, ctypes.cast(host_in, _DP) if host_in else None,
                                   ctypes.cast(host_out, _DP) if host_out else None,
                                   int(field), int(m)), "opo_batch_step_io")


def opo_batch_io_wait(batch):
    _check(lib().opo_batch_io_wait(batch), "opo_batch_io_wait")


# ---- structs from a workload configuration ---------------------------------

def grid_from(cfg, precision=OPO_FP32_PH64, device=0, stream=None) -> Grid:
    return Grid(int(cfg.n), float(cfg.t_window), int(cfg.nfields), int(precision), int(device),
                stream)


def crystals_from(cfg, tod_div=0.0) -> list:
    """The configuration's crystal followed by its ``extra_crystals`` (objects
    with length, nz, dk, deff, nidx, alpha, dbeta1, beta2, beta3, beta4, n2;
    wavelengths and waist are the configuration's)."""
    out = [crystal_from(cfg, tod_div)]
    for x in getattr(cfg, "extra_crystals", ()):
        c = crystal_from(cfg, tod_div)
        c.length_m = x.length
        c.nz = x.nz
        c.dk_per_m = x.dk
        c.deff_mpv = x.deff
        c.n = _D3(*x.nidx)
        c.alpha_per_m = _D3(*x.alpha)
        c.dbeta1_s_per_m = _D3(*x.dbeta1)
        c.beta2_s2_per_m = _D3(*x.beta2)
        c.beta3_s3_per_m = _D3(*x.beta3)
        c.beta4_s4_per_m = _D3(*x.beta4)
        c.n2_m2_per_W = x.n2
        out.append(c)
    return out


def crystal_from(cfg, tod_div=0.0) -> Crystal:
    c = Crystal()
    c.length_m = cfg.length
    c.nz = cfg.nz
    c.dk_per_m = cfg.dk
    c.deff_mpv = cfg.deff
    c.lambda_m = _D3(*cfg.lam)
    c.n = _D3(*cfg.nidx)
    c.alpha_per_m = _D3(*cfg.alpha)
    c.dbeta1_s_per_m = _D3(*cfg.dbeta1)
    c.beta2_s2_per_m = _D3(*cfg.beta2)
    c.beta3_s3_per_m = _D3(*cfg.beta3)
    c.w0_m = cfg.w0
    c.tod_div = tod_div
    c.beta4_s4_per_m = _D3(*getattr(cfg, "beta4", (0.0, 0.0, 0.0)))
    c.n2_m2_per_W = getattr(cfg, "n2", 0.0)
    return c


def cavity_from(cfg, pump_user=None):
    """Returns (Cavity, keepalive); keep the second value alive across the call."""
    v = Cavity()
    v.resonant_mask = cfg.resonant_mask
    v.R = _D3(*cfg.R)
    v.delta_rad = _D3(*cfg.delta)
    v.gdd_s2 = _D3(*cfg.gdd)
    v.delay_s = cfg.delay
    v.eom_beta_rad = cfg.eom_beta
    v.eom_f_hz = cfg.eom_f
    v.t_rt_s = cfg.t_rt
    v.pump_kind = cfg.pump_kind
    v.pump_power_W = cfg.pump_power
    v.pump_fwhm_s = cfg.pump_fwhm
    v.pump_t0_s = getattr(cfg, "pump_t0", 0.0)
    keep = None
    if pump_user is not None:
        keep = _cplx_in(pump_user, cfg.n)
        v.pump_user = keep.ctypes.data_as(_DP)
    return v, keep


class Context:
    """One OPO instance on the GPU, configured from an ``OPOConfig``."""

    def __init__(self, cfg, precision=OPO_FP32_PH64, device=0, stream=None, fields=None,
                 pump_user=None, tod_div=0.0):
        self.cfg = cfg
        self.n = int(cfg.n)
        self.nfields = int(cfg.nfields)
        self.precision = precision
        self.h = opo_create(grid_from(cfg, precision, device, stream))
        try:
            opo_set_crystals(self.h, crystals_from(cfg, tod_div))
            cav, keep = cavity_from(cfg, pump_user)
            opo_set_cavity(self.h, cav)
            del keep
            start = cfg.initial_fields() if fields is None else fields
            self.set_fields(start, rt_index=0)
        except Exception:
            opo_destroy(self.h)
            self.h = None
            raise

    def reset(self, cfg, fields=None, pump_user=None, tod_div=0.0):
        """Reuse this context (same N, field count, precision) for another
        configuration: crystal, cavity and start fields are replaced and the
        round-trip counter restarts at 0."""
        if int(cfg.n) != self.n or int(cfg.nfields) != self.nfields:
            raise ValueError("reset needs the same N and field count")
        self.cfg = cfg
        opo_set_crystals(self.h, crystals_from(cfg, tod_div))
        cav, keep = cavity_from(cfg, pump_user)
        opo_set_cavity(self.h, cav)
        del keep
        self.set_fields(cfg.initial_fields() if fields is None else fields, rt_index=0)

    def set_fields(self, fields, rt_index=-1):
        fields = np.asarray(fields, dtype=np.complex128).reshape(self.nfields, self.n)
        for x in range(self.nfields):
            opo_set_fields(self.h, x, fields[x], rt_index if x == 0 else -1)

    def get_fields(self, which=OPO_INTRACAVITY):
        return np.stack([opo_get_fields(self.h, x, which, self.n) for x in range(self.nfields)])

    def set_path(self, path, cluster=0, rt_per_launch=0, threads=0):
        opo_set_path(self.h, path, cluster, rt_per_launch, threads)

    def run(self, m, stats=True):
        return opo_run_roundtrips(self.h, m, stats)

    def trace(self, rows):
        return opo_get_trace(self.h, rows)

    def set_history(self, max_rt):
        """Record the output-coupled fields of every round trip of the next
        calls (up to max_rt per call); 0 turns it off."""
        opo_set_output_history(self.h, max_rt)

    def history(self, rows, row0=0):
        """(rows, F, N) complex output fields of round trips row0.. of the
        last call."""
        return np.stack([opo_get_output_history(self.h, x, row0, rows, self.n)
                         for x in range(self.nfields)], axis=1)

    def sync(self):
        opo_sync(self.h)

    def close(self):
        if self.h is not None:
            opo_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

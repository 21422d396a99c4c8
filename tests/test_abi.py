"""CPU checks of the C ABI: the library builds, loads, exports every symbol
that include/opo.h declares, validates arguments before touching the GPU, and
fails loudly (no CPU fallback) where no GPU is present."""
import ctypes
import os
import re

import pytest

from paper_2410_02532_gb300 import build as lib_build
from paper_2410_02532_gb300 import opo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            names |= set(re.findall(r"OPO_API\s+[\w\s\*]*?\b(opo_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return opo.lib()


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(L, name), name
    assert set(names) >= set(opo._SIGS)


def test_status_strings(L):
    for s in range(8):
        assert opo.status_string(s) not in ("", "unknown status")
    assert opo.status_string(99) == "unknown status"


def _grid(**kw):
    g = dict(n=1024, t_window_s=1e-10, nfields=3, precision=opo.OPO_FP32_PH64, device=0,
             stream=None)
    g.update(kw)
    return opo.Grid(g["n"], g["t_window_s"], g["nfields"], g["precision"], g["device"],
                    g["stream"])


@pytest.mark.parametrize("kw", [dict(n=1000), dict(n=8), dict(n=1 << 18), dict(nfields=4),
                                dict(nfields=1), dict(precision=7), dict(t_window_s=0.0),
                                dict(t_window_s=float("nan"))])
def test_create_rejects_invalid_grid(L, kw):
    h = ctypes.c_void_p()
    assert L.opo_create(ctypes.byref(h), ctypes.byref(_grid(**kw))) == opo.OPO_E_INVALID
    assert not h.value


def test_null_arguments(L):
    assert L.opo_create(None, None) == opo.OPO_E_INVALID
    h = ctypes.c_void_p()
    assert L.opo_create(ctypes.byref(h), None) == opo.OPO_E_INVALID
    assert L.opo_set_crystal(None, None) == opo.OPO_E_INVALID
    assert L.opo_set_crystals(None, None, 1) == opo.OPO_E_INVALID
    assert L.opo_run_roundtrips(None, 1, None) == opo.OPO_E_INVALID
    assert L.opo_destroy(None) == opo.OPO_OK
    assert L.opo_batch_create(None, None, 0, 0, 0) == opo.OPO_E_INVALID
    assert L.opo_batch_set_fields(None, None, 0) == opo.OPO_E_INVALID
    assert L.opo_batch_get_fields(None, 0, 0, None, 0) == opo.OPO_E_INVALID
    assert L.opo_batch_get_trace(None, None, 0) == opo.OPO_E_INVALID
    assert L.opo_batch_step_io(None, None, None, 0, 1) == opo.OPO_E_INVALID
    assert L.opo_batch_io_wait(None) == opo.OPO_E_INVALID
    assert L.opo_set_output_history(None, 1) == opo.OPO_E_INVALID
    assert L.opo_get_output_history(None, 0, 0, 1, None) == opo.OPO_E_INVALID


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_have_gpu(), reason="checks the no-GPU failure mode")
def test_no_gpu_fails_loudly(L):
    h = ctypes.c_void_p()
    assert L.opo_create(ctypes.byref(h), ctypes.byref(_grid())) == opo.OPO_E_CUDA
    with pytest.raises(opo.OPOError):
        opo.opo_create(_grid())


def test_python_binding_has_no_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(opo, "_lib", None)
    monkeypatch.setattr(opo, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        opo.lib()


# ---------------------------------------------- validation without a GPU

def _valid_config():
    from paper_2410_02532_gb300 import workloads as W
    cfg = W.cw_sro_16k().replace(n=1024)
    grid = opo.grid_from(cfg)
    crys = opo.crystals_from(cfg)
    cav, keep = opo.cavity_from(cfg)
    return cfg, grid, crys, cav, keep


def test_validate_accepts_the_presets(L):
    from paper_2410_02532_gb300 import workloads as W
    for make in W.PRESETS.values():
        cfg = make()
        cav, keep = opo.cavity_from(cfg)
        assert opo.opo_validate(opo.grid_from(cfg), opo.crystals_from(cfg), cav) == opo.OPO_OK, \
            cfg.name
    assert opo.opo_validate(opo.grid_from(W.cw_sro_1024())) == opo.OPO_OK  # grid alone


def _bad(field, value):
    def f(obj):
        setattr(obj, field, value)
    return f


def _bad_triple(field, i, value):
    def f(obj):
        getattr(obj, field)[i] = value
    return f


NAN, INF = float("nan"), float("inf")
CAVITY_BREAKS = {
    "pump_t0_nan": _bad("pump_t0_s", NAN),
    "pump_t0_inf": _bad("pump_t0_s", -INF),
    "R_above_one": _bad_triple("R", 1, 1.01),
    "R_nan": _bad_triple("R", 0, NAN),
    "mask_beyond_fields": _bad("resonant_mask", 0b1000),
    "delay_inf": _bad("delay_s", INF),
    "eom_f_nan": _bad("eom_f_hz", NAN),
    "t_rt_negative": _bad("t_rt_s", -1e-12),
    "pump_negative": _bad("pump_power_W", -1.0),
    "pump_kind_unknown": _bad("pump_kind", 9),
    "sech2_without_width": lambda v: (setattr(v, "pump_kind", opo.OPO_PUMP_SECH2),
                                      setattr(v, "pump_fwhm_s", 0.0)),
    "user_without_profile": _bad("pump_kind", opo.OPO_PUMP_USER),
    "gdd_nan": _bad_triple("gdd_s2", 1, NAN),
}


@pytest.mark.parametrize("name", sorted(CAVITY_BREAKS))
def test_validate_rejects_bad_cavity(L, name):
    cfg, grid, crys, cav, keep = _valid_config()
    assert opo.opo_validate(grid, crys, cav) == opo.OPO_OK
    CAVITY_BREAKS[name](cav)
    assert opo.opo_validate(grid, crys, cav) == opo.OPO_E_INVALID


CRYSTAL_BREAKS = {
    "length_zero": _bad("length_m", 0.0),
    "length_nan": _bad("length_m", NAN),
    "nz_zero": _bad("nz", 0),
    "dk_inf": _bad("dk_per_m", INF),
    "w0_zero": _bad("w0_m", 0.0),
    "tod_div_negative": _bad("tod_div", -6.0),
    "tod_div_inf": _bad("tod_div", INF),
    "index_zero": _bad_triple("n", 2, 0.0),
    "lambda_negative": _bad_triple("lambda_m", 1, -1e-6),
    "beta4_nan": _bad_triple("beta4_s4_per_m", 0, NAN),
    "n2_inf": _bad("n2_m2_per_W", INF),
}


@pytest.mark.parametrize("name", sorted(CRYSTAL_BREAKS))
def test_validate_rejects_bad_crystal(L, name):
    cfg, grid, crys, cav, keep = _valid_config()
    CRYSTAL_BREAKS[name](crys[0])
    assert opo.opo_validate(grid, crys, cav) == opo.OPO_E_INVALID


def test_validate_crystal_list_and_grid(L):
    cfg, grid, crys, cav, keep = _valid_config()
    two = [crys[0], opo.crystal_from(cfg)]
    assert opo.opo_validate(grid, two, cav) == opo.OPO_OK
    two[1].lambda_m[1] = 1.6e-6  # another signal wavelength: not the same fields
    assert opo.opo_validate(grid, two, cav) == opo.OPO_E_INVALID
    assert opo.opo_validate(grid, [crys[0]] * 9, cav) == opo.OPO_E_INVALID  # > 8 crystals
    for kw in (dict(n=1000), dict(n=1 << 18), dict(nfields=1), dict(precision=5),
               dict(t_window_s=-1.0)):
        assert opo.opo_validate(_grid(**kw), crys, cav) == opo.OPO_E_INVALID, kw
    # a degenerate (two-field) grid may not mark the idler resonant
    g2 = _grid(nfields=2)
    cav.resonant_mask = 0b100
    assert opo.opo_validate(g2, [], cav) == opo.OPO_E_INVALID
    assert L.opo_validate(None, None, 0, None) == opo.OPO_E_INVALID

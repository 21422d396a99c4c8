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

"""GPU test of opo_crystal_pass_noalloc, the entry point for callers that
cannot allocate device memory (code running inside another framework's memory
pool, or under a locked-down or exhausted allocator).

It runs one crystal pass on caller-owned device fields with all of its
scratch in a fixed device array inside the library.  Here it is checked,
through the C ABI and on two calls in a row, against the context API: a
plain-path round trip whose cavity is transparent (every field resonant,
R = 1, no detuning, GDD, delay or EOM, no input pump) is exactly one crystal
pass.  This file
sorts last so that a run stopping at the first failure has run everything
else first.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_02532_gb300 import opo
from paper_2410_02532_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {opo.OPO_FP64: 1e-10, opo.OPO_FP32_PH64: 1e-4}


def _lib():
    from paper_2410_02532_gb300 import build
    build.build()
    L = opo.lib()
    L.opo_crystal_pass_noalloc.argtypes = [ctypes.POINTER(opo.Grid), ctypes.POINTER(opo.Crystal),
                                           ctypes.c_void_p, ctypes.c_void_p]
    L.opo_crystal_pass_noalloc.restype = ctypes.c_int
    return L


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _transparent(cfg):
    # a resonant pump gets the input pump added at entry: no input pump
    return cfg.replace(resonant_mask=(1 << cfg.nfields) - 1, R=(1.0, 1.0, 1.0),
                       delta=(0.0, 0.0, 0.0), gdd=(0.0, 0.0, 0.0), delay=0.0, eom_beta=0.0,
                       pump_power=0.0)


def _context_passes(cfg, start, prec, count):
    out = []
    with opo.Context(_transparent(cfg), precision=prec, fields=start) as ctx:
        ctx.set_path(opo.OPO_PATH_PLAIN)
        for _ in range(count):
            ctx.run(1)
            out.append(ctx.get_fields())
    return out


def _start(cfg):
    a = cfg.initial_fields()
    for x in range(cfg.nfields):
        a[x] = a[x] + W.noise(cfg.n, 3e6, cfg.seed + 5, 0, x)
    return a


CASES = {
    "3field_dispersive_dk": W.cw_sro_16k().replace(n=1024, nz=12, dk=120.0),
    "2field_degenerate": W.degenerate_2field(n=2048, level=3.0).replace(nz=9, dk=-40.0),
}


@pytest.mark.parametrize("prec", [opo.OPO_FP64, opo.OPO_FP32_PH64], ids=["fp64", "fp32ph64"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_pass_matches_context_api(case, prec):
    torch = pytest.importorskip("torch")
    L = _lib()
    cfg = CASES[case]
    a0 = _start(cfg)
    ref = _context_passes(cfg, a0, prec, 2)
    dt = torch.complex128 if prec == opo.OPO_FP64 else torch.complex64
    dev = torch.tensor(a0, dtype=dt, device="cuda").contiguous()
    grid = opo.grid_from(cfg, prec)
    crys = opo.crystal_from(cfg)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the scratch array
        st = L.opo_crystal_pass_noalloc(ctypes.byref(grid), ctypes.byref(crys), dev.data_ptr(),
                                        stream)
        assert st == opo.OPO_OK, opo.status_string(st)
        torch.cuda.synchronize()
        got = dev.cpu().numpy().astype(np.complex128)
        for x in range(cfg.nfields):
            assert _rel_l2(got[x], ref[call][x]) <= TOL[prec], (case, call, x)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = _lib()
    cfg = W.sync_pumped_64k()  # 3 fields x 2^16 points: 7 MiB of FP64 scratch > 4 MiB
    grid = opo.grid_from(cfg, opo.OPO_FP64)
    crys = opo.crystal_from(cfg)
    buf = torch.zeros(16, dtype=torch.complex128, device="cuda")  # never touched
    st = L.opo_crystal_pass_noalloc(ctypes.byref(grid), ctypes.byref(crys), buf.data_ptr(), None)
    assert st == opo.OPO_E_INVALID
    assert L.opo_crystal_pass_noalloc(None, ctypes.byref(crys), buf.data_ptr(), None) == \
        opo.OPO_E_INVALID

"""GPU test of opo_crystal_pass_noalloc, the entry point for callers that
cannot allocate device memory (code running inside another framework's memory
pool, or under a locked-down or exhausted allocator).

It runs one crystal pass on caller-owned device fields with all of its
scratch in a fixed device array inside the library.  Here it is checked,
through the C ABI and on two calls in a row, against the context API: a
plain-path round trip whose cavity is transparent (every field resonant,
R = 1, no detuning, GDD, delay or EOM, no input pump) is exactly one crystal
pass of the same kernels with the same tables, so the two agree bit for bit.
One case sits at the largest size the fixed scratch accepts (three FP32
fields of 2^16 points); the next size up is refused.  This file sorts last so
that a run stopping at the first failure has run everything else first.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_02532_gb300 import opo
from paper_2410_02532_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2410_02532_gb300 import build
    build.build()
    L = opo.lib()
    L.opo_crystal_pass_noalloc.argtypes = [ctypes.POINTER(opo.Grid), ctypes.POINTER(opo.Crystal),
                                           ctypes.c_void_p, ctypes.c_void_p]
    L.opo_crystal_pass_noalloc.restype = ctypes.c_int
    return L


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
    "3field_dispersive_dk": (W.cw_sro_16k().replace(n=1024, nz=12, dk=120.0), None),
    "2field_degenerate": (W.degenerate_2field(n=2048, level=3.0).replace(nz=9, dk=-40.0), None),
    # the largest accepted size: 3 x 2^16 FP32 fields (3.5 MiB of the 4 MiB scratch)
    "3field_n65536_largest": (W.sync_pumped_64k(delay_fs=10.0).replace(nz=3),
                              opo.OPO_FP32_PH64),
}
PARAMS = [(c, p) for c in sorted(CASES) for p in (opo.OPO_FP64, opo.OPO_FP32_PH64)
          if CASES[c][1] in (None, p)]


@pytest.mark.parametrize("case,prec", PARAMS,
                         ids=["%s-%s" % (c, "fp64" if p == opo.OPO_FP64 else "fp32ph64")
                              for c, p in PARAMS])
def test_noalloc_pass_matches_context_api(case, prec):
    torch = pytest.importorskip("torch")
    L = _lib()
    cfg = CASES[case][0]
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
        # the same kernels, tables and arguments: bit for bit
        assert np.array_equal(got, ref[call]), (case, call)


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
    # one size above the largest accepted FP32 request: 3 x 2^17 points (7 MiB)
    big = cfg.replace(n=1 << 17)
    st = L.opo_crystal_pass_noalloc(ctypes.byref(opo.grid_from(big, opo.OPO_FP32_PH64)),
                                    ctypes.byref(opo.crystal_from(big)), buf.data_ptr(), None)
    assert st == opo.OPO_E_INVALID
    # the crystal checks of opo_set_crystal apply here too (a negative TOD
    # divisor is refused by both)
    small = W.cw_sro_1024()
    bad = opo.crystal_from(small)
    bad.tod_div = -6.0
    st = L.opo_crystal_pass_noalloc(ctypes.byref(opo.grid_from(small)), ctypes.byref(bad),
                                    buf.data_ptr(), None)
    assert st == opo.OPO_E_INVALID

"""Serving loop on the GPU: continuous batching admits requests while others
run, and every result equals the same request run alone."""
import numpy as np
import pytest

from paper_2410_02532_gb300 import opo
from paper_2410_02532_gb300 import serving
from paper_2410_02532_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2410_02532_gb300 import build
    build.build()
    opo.lib()


def _requests():
    base = W.cw_sro_16k()
    mk = lambda n, **kw: base.replace(n=n, nz=6, **kw)  # noqa: E731
    cfgs = [
        (mk(4096), 20, 0.00),
        (W.degenerate_2field(n=8192, level=3.0).replace(nz=5), 35, 0.01),
        (mk(16384, pump_kind=W.PUMP_SECH2, pump_fwhm=1e-12, eom_beta=0.5, eom_f=10e9,
            delay=10e-15), 17, 0.02),
        (mk(4096, instance=7, pump_power=2 * base.pump_power), 50, 0.05),
        # fused with the exchange through global memory in FP32; too large
        # for the fused path in FP64 (plain path)
        (mk(131072), 4, 0.06),
    ]
    return [serving.Request(i, c.replace(instance=i), m, t) for i, (c, m, t) in enumerate(cfgs)]


@pytest.mark.parametrize("prec,mode", [(opo.OPO_FP32_PH64, "auto"), (opo.OPO_FP64, "auto"),
                                       (opo.OPO_FP32_PH64, "plain")],
                         ids=["fp32-auto", "fp64-auto", "fp32-plain"])
def test_results_do_not_depend_on_the_mix(prec, mode):
    reqs = _requests()
    srv = serving.Server(precision=prec, tick_rt=8, path=mode)
    res = {r.rid: r for r in srv.run(reqs)}
    assert sorted(res) == [r.rid for r in reqs]
    assert srv.ticks >= 5
    paths = set()
    for req in reqs:
        with opo.Context(req.cfg, precision=prec) as ctx:
            try:
                if mode == "plain":
                    raise opo.OPOError(opo.OPO_E_UNSUPPORTED, "plain requested")
                ctx.set_path(opo.OPO_PATH_FUSED)
                path = opo.OPO_PATH_FUSED
            except opo.OPOError:
                ctx.set_path(opo.OPO_PATH_PLAIN)
                path = opo.OPO_PATH_PLAIN
            ctx.run(req.rounds)
            alone_out = ctx.get_fields(opo.OPO_OUTPUT)
            alone_tr = ctx.trace(req.rounds)
        got = res[req.rid]
        assert got.path == path
        paths.add(path)
        assert got.trace.shape == (req.rounds, 4)
        assert np.array_equal(got.out_fields, alone_out), req.rid
        # the trace of a lone call covers all rounds; the server's is per tick
        assert np.array_equal(got.trace, alone_tr), req.rid
    want = {"auto": {opo.OPO_PATH_FUSED} if prec == opo.OPO_FP32_PH64 else
            {opo.OPO_PATH_FUSED, opo.OPO_PATH_PLAIN}, "plain": {opo.OPO_PATH_PLAIN}}[mode]
    assert paths == want


def test_admission_respects_budgets():
    reqs = _requests()[:4]
    srv = serving.Server(tick_rt=8, gpu_share=0.1)
    res = srv.run(reqs)
    assert len(res) == 4
    st = serving.latency_stats(res)
    assert st["count"] == 4 and st["p99_s"] >= st["p50_s"] > 0
    # with a tenth of the GPU at a time, later requests wait
    assert max(r.admitted - r.arrival for r in res) > 0

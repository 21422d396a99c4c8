"""The batched plain path: many instances on the one-kernel-per-operation
chain (Sec. 2.2 and the main loop of Sec. 4.1), every launch applying one
operation to all members of a group.

Each member must advance bit for bit as the same instance does alone on the
plain path (which the parity tests compare with the oracle), whatever the
mix: sizes, field counts, cavity elements (GDD and delay or a plain signal
copy), pump regimes, Kerr terms, several crystals, output history.  One case
is also compared with the oracle directly.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2410_02532_gb300 import opo
from paper_2410_02532_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2410_02532_gb300 import build
    build.build()
    opo.lib()


def start(cfg, amp=2e6, seed_off=0):
    a = cfg.initial_fields()
    for x in range(1, cfg.nfields):
        a[x] = a[x] + W.noise(cfg.n, amp, cfg.seed + 41 + seed_off, cfg.instance, x)
    return a


def mix():
    b = W.cw_sro_16k()
    return [
        # GDD + delay on the signal: the cavity visit transforms every field
        b.replace(n=1024, nz=6, delay=12e-15, name="gdd_delay"),
        # no GDD, no delay: the visit transforms a signal copy only
        W.cw_sro_1024().replace(nz=5, name="copy_only"),
        # same size and steps, other parameters (pump level, EOM, dk, loss)
        W.cw_sro_1024().replace(nz=5, dk=90.0, alpha=(1.0, 0.5, 2.0), eom_beta=0.4,
                                eom_f=13e9, pump_power=3 * b.pump_power / 16,
                                name="eom_dk_loss"),
        # two fields, Kerr terms and fourth-order dispersion
        W.degenerate_2field(n=1024, level=3.0).replace(nz=5, dk=60.0, n2=2e-17,
                                                       beta4=(4e-55, -3e-55, 0.0),
                                                       name="deg_kerr"),
        # pump-resonant cavity with the ns-pulsed pump
        W.tro_cw(n=2048).replace(nz=4, pump_kind=W.PUMP_NS, pump_power=40.0,
                                 pump_fwhm=300e-12, pump_t0=300e-12, name="tro_ns"),
        # two crystals (5 + 3 steps), sech^2 pump
        b.replace(n=2048, nz=5, length=6e-3, pump_kind=W.PUMP_SECH2, pump_fwhm=1e-12,
                  extra_crystals=(W.Crystal(length=4e-3, nz=3, dk=-40.0),), name="two_crystals"),
    ]


@pytest.mark.parametrize("prec", [opo.OPO_FP64, opo.OPO_FP32_PH64], ids=["fp64", "fp32ph64"])
def test_plain_batch_matches_alone_bitwise(prec):
    cfgs = mix()
    starts = [start(c, seed_off=i) for i, c in enumerate(cfgs)]
    calls = (2, 3)
    ref = []
    for c, a in zip(cfgs, starts):
        with opo.Context(c, precision=prec, fields=a) as ctx:
            ctx.set_fields(a, rt_index=2)
            ctx.set_path(opo.OPO_PATH_PLAIN)
            r = []
            for m in calls:
                ctx.run(m)
                r.append((ctx.get_fields(), ctx.get_fields(opo.OPO_OUTPUT), ctx.trace(m)))
            ref.append(r)
    ctxs = [opo.Context(c, precision=prec, fields=a) for c, a in zip(cfgs, starts)]
    try:
        for c, a in zip(ctxs, starts):
            c.set_fields(a, rt_index=2)
            c.set_path(opo.OPO_PATH_PLAIN)
        b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
        for k, m in enumerate(calls):
            opo.opo_batch_run(b, m)
            for i, ctx in enumerate(ctxs):
                f, o, t = ref[i][k]
                assert np.array_equal(ctx.get_fields(), f), (cfgs[i].name, k)
                assert np.array_equal(ctx.get_fields(opo.OPO_OUTPUT), o), (cfgs[i].name, k)
                assert np.array_equal(ctx.trace(m), t), (cfgs[i].name, k)
        s = ctxs[0].run(0)
        assert s.rt_done == 2 + sum(calls)
        opo.opo_batch_destroy(b)
    finally:
        for c in ctxs:
            c.close()


def test_plain_batch_against_oracle():
    """One member of a mixed plain batch, one round trip, element by element
    against the oracle (FP32 fields with FP64 phases: <= 1e-4)."""
    cfgs = mix()
    starts = [start(c, seed_off=i) for i, c in enumerate(cfgs)]
    ctxs = [opo.Context(c, fields=a) for c, a in zip(cfgs, starts)]
    try:
        for c in ctxs:
            c.set_path(opo.OPO_PATH_PLAIN)
        b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
        opo.opo_batch_run(b, 1)
        for cfg, a, ctx in zip(cfgs, starts, ctxs):
            p = orc.params(cfg)
            kind = cfg.pump_kind if cfg.pump_kind in (W.PUMP_CW, W.PUMP_SECH2) else W.PUMP_CW
            pump = orc.pump_profile(p, kind, cfg.pump_power, cfg.pump_fwhm)
            ref, _, _, st = orc.run(p, a, pump, 0, 1)
            assert st == 0
            got = ctx.get_fields()
            for x in range(cfg.nfields):
                e = np.linalg.norm(got[x] - ref[x]) / np.linalg.norm(ref[x])
                assert e <= 1e-4, (cfg.name, x, e)
        opo.opo_batch_destroy(b)
    finally:
        for c in ctxs:
            c.close()


def test_mixed_fused_and_plain_batch():
    """One FP64 batch with fused members (2^12, 2^14) and members the
    automatic choice puts on the plain path (three FP64 fields at 2^17), or
    that ask for it: each equals its lone run bit for bit."""
    b16 = W.cw_sro_16k()
    prec = opo.OPO_FP64
    cfgs = [b16.replace(n=1 << 12, nz=3), b16.replace(nz=2),
            W.sync_pumped_64k(delay_fs=5.0).replace(n=1 << 17, nz=2),
            b16.replace(n=1 << 12, nz=3, delay=8e-15)]
    paths = [opo.OPO_PATH_AUTO, opo.OPO_PATH_AUTO, opo.OPO_PATH_AUTO, opo.OPO_PATH_PLAIN]
    starts = [start(c, seed_off=i) for i, c in enumerate(cfgs)]
    ref = []
    for c, a, pth in zip(cfgs, starts, paths):
        with opo.Context(c, precision=prec, fields=a) as ctx:
            ctx.set_path(pth)
            s = ctx.run(2)
            ref.append((ctx.get_fields(), ctx.trace(2), s.path))
    assert [r[2] for r in ref] == [opo.OPO_PATH_FUSED, opo.OPO_PATH_FUSED, opo.OPO_PATH_PLAIN,
                                   opo.OPO_PATH_PLAIN]
    ctxs = [opo.Context(c, precision=prec, fields=a) for c, a in zip(cfgs, starts)]
    try:
        for c, pth in zip(ctxs, paths):
            c.set_path(pth)
        b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
        opo.opo_batch_run(b, 2)
        for i, ctx in enumerate(ctxs):
            assert np.array_equal(ctx.get_fields(), ref[i][0]), i
            assert np.array_equal(ctx.trace(2), ref[i][1]), i
        opo.opo_batch_destroy(b)
    finally:
        for c in ctxs:
            c.close()


def test_plain_batch_history_and_stale_member():
    cfgs = mix()[:3]
    starts = [start(c, seed_off=i) for i, c in enumerate(cfgs)]
    hist_ref = []
    for c, a in zip(cfgs, starts):
        with opo.Context(c, fields=a) as ctx:
            ctx.set_path(opo.OPO_PATH_PLAIN)
            ctx.set_history(3)
            ctx.run(3)
            hist_ref.append(ctx.history(3))
    ctxs = [opo.Context(c, fields=a) for c, a in zip(cfgs, starts)]
    try:
        for c in ctxs:
            c.set_path(opo.OPO_PATH_PLAIN)
            c.set_history(3)
        b = opo.opo_batch_create([c.h for c in ctxs], 0, 0)
        opo.opo_batch_run(b, 3)
        for ctx, h in zip(ctxs, hist_ref):
            assert np.array_equal(ctx.history(3), h)
        # a member whose crystal now has another step count no longer fits
        # its group: the batch refuses to run
        opo.opo_set_crystals(ctxs[1].h, opo.crystals_from(cfgs[1].replace(nz=7)))
        with pytest.raises(opo.OPOError) as ei:
            opo.opo_batch_run(b, 1)
        assert ei.value.status == opo.OPO_E_STATE
        opo.opo_batch_destroy(b)
    finally:
        for c in ctxs:
            c.close()

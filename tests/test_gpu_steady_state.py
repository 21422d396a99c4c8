"""Steady state after many round trips: the GPU's output signal power and
spectral centroid, averaged over the last round trips, against the oracle's
from the same start (<= 1e-3 relative on P_s,out in FP32 with FP64 phases;
the centroid within 1e-3 of the output's rms spectral width, floored at half a
frequency bin).  The steady-state signal phase is free, so only these
phase-invariant scalars are compared; the configurations settle (relative
change of P_s,out over 100 round trips below 1e-7 in the oracle) within the
run.
"""
import numpy as np
import pytest

import parity_log
from oracle import oracle as orc
from paper_2410_02532_gb300 import opo
from paper_2410_02532_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M = 300
LAST = 20
TOL = {opo.OPO_FP64: 1e-6, opo.OPO_FP32_PH64: 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2410_02532_gb300 import build
    build.build()
    opo.lib()


def sro_off_carrier():
    """SRO with GVM (idler against signal), GVD, TOD and intracavity GDD, a
    phase mismatch that moves the gain peak 1.88 THz below the signal
    carrier, R_s = 0.7, 2.5x threshold; the start is a tone at that peak, so
    the steady state (and its centroid) is off the carrier."""
    b = W.cw_sro_16k()
    c = W.OPOConfig(n=1024, nz=25, length=5e-3, R=(0.0, 0.7, 0.0), dk=400.0,
                    dbeta1=(b.dbeta1[0], 0.0, -5e-11), beta2=b.beta2, beta3=b.beta3,
                    gdd=(0.0, -100e-30, 0.0), name="steady_sro")
    return c.replace(pump_power=2.5 * W.sro_threshold_power(c))


def degenerate():
    d = W.degenerate_2field(n=1024).replace(R=(0.0, 0.7, 0.0), nz=25, dbeta1=(1e-10, 0, 0),
                                            beta2=(3.8e-25, 1.1e-25, 0), name="steady_deg")
    return d.replace(pump_power=2.0 * W.sro_threshold_power(d))


def start(cfg, tone=0):
    a = cfg.initial_fields()
    j = np.arange(cfg.n)
    a[1] = 1e6 * np.exp(0.3j + 2j * np.pi * tone * j / cfg.n) + W.noise(cfg.n, 1e3, cfg.seed + 3, 0, 1)
    return a


_ref_cache = {}


def oracle_steady(name, cfg, a):
    if name not in _ref_cache:
        p = orc.params(cfg)
        pump = orc.pump_profile(p, 0, cfg.pump_power)
        out, tr, outf, st = orc.run(p, a, pump, 0, M)
        assert st == 0
        ps = tr[:, 1]
        assert abs(ps[-1] - ps[-101]) <= 1e-7 * ps[-1]  # settled
        X = np.abs(np.fft.fft(outf[1])) ** 2
        f = np.fft.fftfreq(cfg.n, cfg.t_window / cfg.n)
        mu = float(np.sum(f * X) / np.sum(X))
        width = float(np.sqrt(np.sum((f - mu) ** 2 * X) / np.sum(X)))
        _ref_cache[name] = (tr, width)
    return _ref_cache[name]


CASES = {"sro_off_carrier": (sro_off_carrier, -188), "degenerate": (degenerate, 0)}


@pytest.mark.parametrize("prec", [opo.OPO_FP64, opo.OPO_FP32_PH64], ids=["fp64", "fp32ph64"])
@pytest.mark.parametrize("path", [opo.OPO_PATH_PLAIN, opo.OPO_PATH_FUSED], ids=["plain", "fused"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_steady_state_power_and_centroid(name, path, prec):
    make, tone = CASES[name]
    cfg = make()
    a = start(cfg, tone)
    ref, width = oracle_steady(name, cfg, a)
    with opo.Context(cfg, precision=prec, fields=a) as ctx:
        ctx.set_path(path)
        ctx.run(M)
        tr = ctx.trace(M)
    tol = TOL[prec]
    ps_ref, ps = ref[-LAST:, 1].mean(), tr[-LAST:, 1].mean()
    assert abs(ps - ps_ref) <= tol * ps_ref, (ps, ps_ref)
    nu_ref, nu = ref[-LAST:, 3].mean(), tr[-LAST:, 3].mean()
    floor = 0.5 / cfg.t_window
    assert abs(nu - nu_ref) <= tol * max(width, floor), (nu, nu_ref)
    if name == "sro_off_carrier":
        # the steady state sits far off the carrier compared with the tolerance
        assert abs(nu_ref) > 100 * tol * max(width, floor)


# ----------------------------------------------- the 2^14-point workload
# The stored oracle run (tests/golden/steady_state_cw_sro_16k.json, written by
# tests/golden/make_steady_state.py from oracle/ only): the 2^14-point CW SRO
# with GVM, GVD, TOD and intracavity GDD at 4x threshold, from the seeded
# 1e-15 V/m noise through growth (~1700 round trips), saturation and 3000
# round trips in all.  By then the output powers have settled (to about 1e-3
# per 300 round trips), but the signal spectrum is still walking away from
# the carrier (its centroid moves ~0.2 THz per 100 round trips and reaches a
# fixed point near 12 THz only after ~2e4 round trips).  The walk is not
# chaotic: a start perturbed by 1e-7 stays within 1e-9 of the oracle run, and
# the FP64 path tracks it within 1e-6; FP32 rounding changes the rate of the
# walk by a few per cent.  So at 3000 round trips: FP64 -- powers and
# centroid within 1e-6; FP32 fields with FP64 phases -- output powers within
# 1e-3, the centroid within 5% of its distance from the carrier.

import json  # noqa: E402
import os  # noqa: E402

GOLDEN_16K = os.path.join(os.path.dirname(__file__), "golden", "steady_state_cw_sro_16k.json")


@pytest.mark.parametrize("prec,path", [(opo.OPO_FP32_PH64, opo.OPO_PATH_FUSED),
                                       (opo.OPO_FP32_PH64, opo.OPO_PATH_PLAIN),
                                       (opo.OPO_FP64, opo.OPO_PATH_FUSED)],
                         ids=["fp32ph64-fused", "fp32ph64-plain", "fp64-fused"])
def test_n16384_from_noise_through_saturation(prec, path):
    """Same start (the seeded noise), same number of round trips as the
    oracle run; means over the last K round trips of the output signal and
    pump powers and of the signal centroid."""
    ref = json.load(open(GOLDEN_16K))
    cfg = W.cw_sro_16k()
    assert ref["workload"] == cfg.name
    M, K = ref["rt"], ref["last"]
    with opo.Context(cfg, precision=prec) as ctx:
        ctx.set_path(path)
        ctx.run(M)
        tr = ctx.trace(M)
    fp64 = prec == opo.OPO_FP64
    tol = 1e-6 if fp64 else 1e-3
    parity_log.record("steady_state", "cw_sro_16k_%d_rt" % M, prec, path, n=cfg.n,
                      fields=cfg.nfields, nz=cfg.nz,
                      rel_power_signal=abs(tr[-K:, 1].mean() / ref["p_out_mean_W"][1] - 1),
                      pump_dev_over_input=abs(tr[-K:, 0].mean() - ref["p_out_mean_W"][0])
                      / cfg.pump_power,
                      centroid_rel=abs(tr[-K:, 3].mean() / ref["centroid_mean_hz"] - 1),
                      centroid_over_width=abs(tr[-K:, 3].mean() - ref["centroid_mean_hz"])
                      / ref["width_hz"])
    ps, ps_ref = tr[-K:, 1].mean(), ref["p_out_mean_W"][1]
    assert abs(ps - ps_ref) <= tol * ps_ref, (ps, ps_ref)
    # the pump's depletion, in units of the input pump power
    pp, pp_ref = tr[-K:, 0].mean(), ref["p_out_mean_W"][0]
    assert abs(pp - pp_ref) <= tol * cfg.pump_power, (pp, pp_ref)
    nu, nu_ref = tr[-K:, 3].mean(), ref["centroid_mean_hz"]
    bound = tol * max(ref["width_hz"], 0.5 / cfg.t_window) if fp64 else 0.05 * abs(nu_ref)
    assert abs(nu - nu_ref) <= bound, (nu, nu_ref, bound)


# The same workload after 20000 round trips: tests/golden/
# steady_state_cw_sro_16k_long.json, written by
#   python tests/golden/make_steady_state.py --rt 20000 \
#       --out tests/golden/steady_state_cw_sro_16k_long.json
# (oracle/ only; about four hours of one core).  By then the output powers
# have settled (the mean P_s,out of the last two 2000-round-trip windows
# differs by 2.5e-7), so the FP32 fields with FP64 phases (both paths) are
# held to the 1e-3 bar on both powers with the transient gone.  The signal
# centroid has not settled: it is on a slow excursion (up to 11.2 THz at
# ~11000 round trips, back to 9.7 THz at 20000, still moving ~4% per 2000
# round trips), and FP32 rounding shifts the excursion's phase (8-20% apart
# at 20000 round trips), so the centroid is recorded here, not held to a
# steady-state bar; the FP64 path tracks the oracle's centroid within 1e-10
# through the first 3000 round trips (above).
GOLDEN_16K_LONG = os.path.join(os.path.dirname(__file__), "golden",
                               "steady_state_cw_sro_16k_long.json")


@pytest.mark.parametrize("path", [opo.OPO_PATH_FUSED, opo.OPO_PATH_PLAIN], ids=["fused", "plain"])
def test_n16384_settled_after_20000_round_trips(path):
    ref = json.load(open(GOLDEN_16K_LONG))
    cfg = W.cw_sro_16k()
    assert ref["workload"] == cfg.name
    M, K = ref["rt"], ref["last"]
    # the oracle run has settled: the mean output signal power of its last
    # two K-round-trip windows agree well inside the bar
    assert ref["window_drift"] < 1e-4, ref["window_drift"]
    with opo.Context(cfg, precision=opo.OPO_FP32_PH64) as ctx:
        ctx.set_path(path)
        ctx.run(M)
        tr = ctx.trace(M)
    ps, ps_ref = tr[-K:, 1].mean(), ref["p_out_mean_W"][1]
    pp, pp_ref = tr[-K:, 0].mean(), ref["p_out_mean_W"][0]
    nu, nu_ref = tr[-K:, 3].mean(), ref["centroid_mean_hz"]
    parity_log.record("steady_state", "cw_sro_16k_%d_rt" % M, opo.OPO_FP32_PH64, path, n=cfg.n,
                      fields=cfg.nfields, nz=cfg.nz, rel_power_signal=abs(ps / ps_ref - 1),
                      pump_dev_over_input=abs(pp - pp_ref) / cfg.pump_power,
                      centroid_rel=abs(nu / nu_ref - 1),
                      centroid_over_width=abs(nu - nu_ref) / ref["width_hz"])
    assert abs(ps - ps_ref) <= 1e-3 * ps_ref, (ps, ps_ref)
    assert abs(pp - pp_ref) <= 1e-3 * cfg.pump_power, (pp, pp_ref)
    # sanity only (not a parity bar): the centroid is on the oracle's side
    # of the carrier and within one rms spectral width of the oracle's
    assert nu > 0 and abs(nu - nu_ref) <= ref["width_hz"], (nu, nu_ref)

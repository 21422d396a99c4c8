"""Seeded synthetic inputs and the workload presets of the OPO hot path.

This module holds input generation only: parameter presets (SI units), the
seeded complex noise that starts the signal and idler (Sec. 4.2 of arXiv
2410.02532: "random amplitude and phase"), and the pump level expressed as a
multiple of the plane-wave singly-resonant threshold.  It contains none of the
split-step arithmetic; both the CUDA library and the FP64 oracle consume what
it produces as plain data.

Noise recipe (counter-based, reproducible on any host):
  key   = mix64(seed + G * (1 + 4*instance + field))
  u_j   = (mix64(key + G * (1 + 2*index + j)) >> 11 + 0.5) * 2^-53,  j = 0, 1
  g     = sqrt(-2 ln u_0) * (cos 2 pi u_1, sin 2 pi u_1)      (Box-Muller)
  A     = amp * (g_re + i g_im) / sqrt(2)
with mix64 the SplitMix64 finaliser and G = 0x9E3779B97F4A7C15.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass

import numpy as np

EPS0 = 8.8541878128e-12  # vacuum permittivity [F/m]
C0 = 299792458.0         # speed of light [m/s]

PUMP_CW, PUMP_SECH2, PUMP_USER, PUMP_NS = 0, 1, 2, 3

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def noise(n: int, amp: float, seed: int, instance: int = 0, fld: int = 1) -> np.ndarray:
    """Seeded complex Gaussian noise of rms amplitude ``amp`` (complex128, n)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed) + _G * np.uint64(1 + 4 * instance + fld)],
                              dtype=np.uint64))[0]
        idx = np.arange(n, dtype=np.uint64)
        c0 = key + _G * (np.uint64(1) + np.uint64(2) * idx)
        c1 = key + _G * (np.uint64(2) + np.uint64(2) * idx)
    u0 = ((_mix64(c0) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u1 = ((_mix64(c1) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u0))
    g = r * np.cos(2.0 * np.pi * u1) + 1j * r * np.sin(2.0 * np.pi * u1)
    return (amp / math.sqrt(2.0)) * g


@dataclass(frozen=True)
class Crystal:
    """A further nonlinear crystal of the round trip (after the configuration's
    own): its length, step count, phase mismatch, d_eff, indices, loss,
    dispersion and Kerr index.  Wavelengths are the configuration's."""
    length: float = 5e-3
    nz: int = 50
    dk: float = 0.0
    deff: float = 14e-12
    nidx: tuple = (2.15, 2.14, 2.08)
    alpha: tuple = (0.0, 0.0, 0.0)
    dbeta1: tuple = (0.0, 0.0, 0.0)
    beta2: tuple = (0.0, 0.0, 0.0)
    beta3: tuple = (0.0, 0.0, 0.0)
    beta4: tuple = (0.0, 0.0, 0.0)
    n2: float = 0.0


@dataclass
class OPOConfig:
    """One OPO instance: grid, crystal and cavity, SI units.

    Field order is (pump, signal, idler); two-field configurations use
    (pump, signal) and ignore the third entry of each triple.
    """
    name: str = "custom"
    n: int = 1024
    t_window: float = 100e-12
    nfields: int = 3
    length: float = 5e-3
    nz: int = 50
    dk: float = 0.0
    deff: float = 14e-12
    lam: tuple = (1.064e-6, 1.55e-6, 1.064e-6 * 1.55e-6 / (1.55e-6 - 1.064e-6))
    nidx: tuple = (2.15, 2.14, 2.08)
    alpha: tuple = (0.0, 0.0, 0.0)
    dbeta1: tuple = (0.0, 0.0, 0.0)
    beta2: tuple = (0.0, 0.0, 0.0)
    beta3: tuple = (0.0, 0.0, 0.0)
    beta4: tuple = (0.0, 0.0, 0.0)
    n2: float = 0.0
    extra_crystals: tuple = ()   # Crystal objects passed after this one
    w0: float = 55e-6
    resonant_mask: int = 0b010
    R: tuple = (0.0, 0.98, 0.0)
    delta: tuple = (0.0, 0.0, 0.0)
    gdd: tuple = (0.0, 0.0, 0.0)
    delay: float = 0.0
    eom_beta: float = 0.0
    eom_f: float = 0.0
    t_rt: float = 100e-12
    pump_kind: int = PUMP_CW
    pump_power: float = 1.0
    pump_fwhm: float = 0.0
    pump_t0: float = 0.0
    noise_amp: float = 1e-15
    seed: int = 20241004
    instance: int = 0
    M: int = 10

    def replace(self, **kw) -> "OPOConfig":
        return dataclasses.replace(self, **kw)

    def initial_fields(self) -> np.ndarray:
        """(F, N) complex128 start state: pump 0, signal/idler seeded noise."""
        a = np.zeros((self.nfields, self.n), dtype=np.complex128)
        for x in range(1, self.nfields):
            a[x] = noise(self.n, self.noise_amp, self.seed, self.instance, x)
        return a


def sro_threshold_power(cfg: OPOConfig) -> float:
    """Plane-wave threshold pump power [W] with only the signal resonant, for
    the crystal length and signal reflectivity of ``cfg`` (no dispersion).

    Three fields (idler dumped each pass): round-trip small-signal power gain
    R cosh^2(Gamma L), Gamma = sqrt(kappa_s kappa_i) |A_p|, so threshold is
    Gamma L = acosh(R^-1/2).  Two fields (degenerate): R exp(2 kappa_s |A_p| L).
    Used only to pick pump levels for the presets.
    """
    kap = [2 * math.pi * cfg.deff / (cfg.nidx[x] * cfg.lam[x]) if cfg.lam[x] > 0 else 0.0
           for x in range(3)]
    if cfg.nfields == 2:
        # degenerate: amplitude gain e^{kappa_s |A_p| L} on the amplified quadrature
        a_th = math.log(1.0 / math.sqrt(cfg.R[1])) / (kap[1] * cfg.length)
    else:
        g = math.acosh(1.0 / math.sqrt(cfg.R[1])) / cfg.length
        a_th = g / math.sqrt(kap[1] * kap[2])
    intensity = 0.5 * cfg.nidx[0] * EPS0 * C0 * a_th * a_th
    return intensity * math.pi * cfg.w0 * cfg.w0


# ------------------------------------------------------------------ presets

def _fs2mm(v):  # fs^2/mm -> s^2/m
    return v * 1e-30 / 1e-3


def _fs3mm(v):  # fs^3/mm -> s^3/m
    return v * 1e-45 / 1e-3


def cw_sro_1024() -> OPOConfig:
    """N=1024, 3 fields, 5 mm PPLN, 50 z-steps, SRO R_s=0.98, 2x threshold,
    no dispersion, 10 round trips (the small parity workload)."""
    c = OPOConfig(name="cw_sro_n1024_3f_L5mm_nz50", n=1024, nz=50, length=5e-3, M=10,
                  seed=20241004)
    return c.replace(pump_power=2.0 * sro_threshold_power(c))


def cw_sro_16k() -> OPOConfig:
    """N=2^14 in a 100 ps window, 3 fields, 20 mm PPLN, 100 z-steps, GVM
    pump-signal 0.1 ps/mm, GVD 380/110/-750 fs^2/mm, TOD 250 fs^3/mm,
    intracavity GDD -500 fs^2 on the signal, 4x threshold, 1000 round trips."""
    c = OPOConfig(name="cw_sro_n16384_3f_L20mm_nz100_gdd", n=1 << 14, nz=100, length=20e-3,
                  dbeta1=(0.1e-12 / 1e-3, 0.0, 0.0),
                  beta2=(_fs2mm(380), _fs2mm(110), _fs2mm(-750)),
                  beta3=(_fs3mm(250), _fs3mm(250), _fs3mm(250)),
                  gdd=(0.0, -500e-30, 0.0), M=1000, seed=20241005)
    return c.replace(pump_power=4.0 * sro_threshold_power(c))


def sync_pumped_64k(delay_fs: float = 0.0) -> OPOConfig:
    """N=2^16, sech^2 pump 200 fs FWHM at 1.064 um, 1 mm PPLN, 64 z-steps,
    cavity timing mismatch ``delay_fs`` in [-20, 20] fs, EOM 0.5 rad at the
    round-trip rate (10 GHz), 2000 round trips; peak 3x CW threshold."""
    c = OPOConfig(name="sync_pumped_n65536_3f_L1mm_nz64_eom", n=1 << 16, nz=64, length=1e-3,
                  dbeta1=(0.1e-12 / 1e-3, 0.0, 0.0),
                  beta2=(_fs2mm(380), _fs2mm(110), _fs2mm(-750)),
                  beta3=(_fs3mm(250), _fs3mm(250), _fs3mm(250)),
                  delay=delay_fs * 1e-15, eom_beta=0.5, eom_f=10e9,
                  pump_kind=PUMP_SECH2, pump_fwhm=200e-15, M=2000, seed=20241006)
    return c.replace(pump_power=3.0 * sro_threshold_power(c))


def degenerate_2field(n: int = 1024, level: float = 2.0) -> OPOConfig:
    """Degenerate OPO (Sec. 4.4): 0.532 -> 1.064 um, signal resonant.
    n_p(0.532 um) = 2.23 is an assumed value; n_s = 2.15."""
    c = OPOConfig(name="degenerate_2f", n=n, nfields=2, lam=(0.532e-6, 1.064e-6, 0.0),
                  nidx=(2.23, 2.15, 1.0), R=(0.0, 0.98, 0.0), resonant_mask=0b010,
                  seed=20241007)
    return c.replace(pump_power=level * sro_threshold_power(c))


def ns_pulsed_degenerate(peak_w: float = 75.0, n: int = 1024) -> OPOConfig:
    """ns-pulsed degenerate OPO (Sec. 4.2 example): 0.532 -> 1.064 um, 5 mm
    crystal, 10 ns FWHM Gaussian pump of peak power ``peak_w`` (the paper's
    examples use 75, 100 and 250 W), signal resonant, 100 ps round trip,
    pulse centred at 30 ns, 600 round trips (60 ns).  Cavity length, waist
    and mirror reflectivity of the paper's example are not given; these are
    the defaults of the other presets."""
    return degenerate_2field(n=n).replace(
        name="ns_pulsed_n%d_2f_L5mm_nz50_%gW" % (n, peak_w), length=5e-3, nz=50,
        pump_kind=PUMP_NS, pump_power=float(peak_w), pump_fwhm=10e-9, pump_t0=30e-9, M=600,
        seed=20241009)


def tro_cw(n: int = 1024, level: float = 0.05) -> OPOConfig:
    """Triply resonant CW OPO (pump-resonant cavity, Sec. 4.2): 3 fields, 5 mm,
    R = 0.9 / 0.98 / 0.98; the input pump is added to the circulating one each
    round trip (cavity enhancement 1/(1 - sqrt R_p)^2 ~ 380 below threshold).
    ``level`` is the input pump power in units of the SRO threshold."""
    c = OPOConfig(name="tro_cw_n%d_3f_L5mm_nz50" % n, n=n, nz=50, length=5e-3,
                  resonant_mask=0b111, R=(0.9, 0.98, 0.98), M=400, seed=20241010)
    return c.replace(pump_power=level * sro_threshold_power(c.replace(resonant_mask=0b010)))


def sweep_instances(count: int = 256, seed: int = 20241007) -> list:
    """Batched sweep: N log-uniform over 2^12..2^15, pump 1-5x threshold,
    timing mismatch within +-50 fs, L in 5-30 mm, 100 z-steps; 50% SRO 3-field,
    25% DRO 3-field (R_s = R_i = 0.98), 25% degenerate 2-field."""
    rng = np.random.default_rng(seed)
    out = []
    base16k = cw_sro_16k()
    for i in range(count):
        n = 1 << int(12 + (i % 4))
        kind = ("sro", "sro", "dro", "deg")[(i // 4) % 4]
        L = float(rng.uniform(5e-3, 30e-3))
        level = float(rng.uniform(1.0, 5.0))
        delay = float(rng.uniform(-50e-15, 50e-15))
        if kind == "deg":
            c = degenerate_2field(n=n).replace(length=L, nz=100)
        else:
            c = OPOConfig(n=n, length=L, nz=100)
            if kind == "dro":
                c = c.replace(resonant_mask=0b110, R=(0.0, 0.98, 0.98))
        c = c.replace(name="sweep_%d_%s" % (i, kind), dbeta1=base16k.dbeta1,
                      beta2=base16k.beta2, beta3=base16k.beta3, delay=delay,
                      seed=seed, instance=i, M=1000)
        c = c.replace(pump_power=level * sro_threshold_power(c))
        out.append(c)
    return out


PRESETS = {
    "cw_sro_1024": cw_sro_1024,
    "cw_sro_16k": cw_sro_16k,
    "sync_pumped_64k": sync_pumped_64k,
    "degenerate_2field": degenerate_2field,
    "ns_pulsed_degenerate": ns_pulsed_degenerate,
    "tro_cw": tro_cw,
}

__all__ = ["OPOConfig", "Crystal", "noise", "sro_threshold_power", "PRESETS", "cw_sro_1024", "cw_sro_16k",
           "sync_pumped_64k", "degenerate_2field", "ns_pulsed_degenerate", "tro_cw",
           "sweep_instances", "EPS0", "C0", "PUMP_CW", "PUMP_SECH2", "PUMP_USER", "PUMP_NS"]

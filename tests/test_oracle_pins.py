"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a brute-force computation, a closed form,
a conservation law, a special case that reduces to a library routine, or a
value printed in arXiv 2410.02532 (tests/golden/paper_values.json).  The
parameters are chosen so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import special
from scipy.optimize import brentq

from paper_2410_02532_gb300 import workloads as W

EPS0 = 8.8541878128e-12  # CODATA 2018, the tests' own copy
C0 = 299792458.0
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def kappas(cfg):
    return [2 * math.pi * cfg.deff / (cfg.nidx[x] * cfg.lam[x]) if cfg.lam[x] > 0 else 0.0
            for x in range(3)]


def cw(n=4, **kw):
    """Plane-wave (CW) configuration on a tiny grid: all points identical."""
    base = dict(n=n, nz=50, length=5e-3, t_window=100e-12)
    base.update(kw)
    return W.OPOConfig(**base)


def amp_for_power(cfg, power):
    inten = power / (math.pi * cfg.w0 ** 2)
    return math.sqrt(2 * inten / (cfg.nidx[0] * EPS0 * C0))


# ----------------------------------------------------------------- 1. DFT

@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_fft_matches_bruteforce_dft(orc, n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(k, k) / n)
    assert rel_l2(orc.fft(x, -1), F @ x) <= 1e-13
    assert rel_l2(orc.fft(x, +1), (np.conj(F) @ x) / n) <= 1e-13


@pytest.mark.parametrize("n", [1024, 1 << 14])
def test_fft_matches_library_fft(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel_l2(orc.fft(x, -1), np.fft.fft(x)) <= 1e-13
    assert rel_l2(orc.fft(x, +1), np.fft.ifft(x)) <= 1e-13


def test_fft_rejects_non_power_of_two(orc):
    with pytest.raises(ValueError):
        orc.fft(np.ones(12), -1)


# ------------------------------------------------- 2-6. linear operator

def test_parseval_and_unitarity(orc):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    X = orc.fft(x, -1)
    assert abs(np.sum(abs(X) ** 2) - 256 * np.sum(abs(x) ** 2)) <= 1e-12 * np.sum(abs(X) ** 2)
    assert rel_l2(orc.fft(X, +1), x) <= 1e-14 * 8
    cfg = cw(n=256, t_window=10e-12, dbeta1=(1e-10, -2e-10, 3e-11),
             beta2=(3.8e-25, 1.1e-25, -7.5e-25), beta3=(2.5e-40, 2.5e-40, 2.5e-40))
    p = orc.params(cfg)
    A = np.stack([rng.standard_normal(256) + 1j * rng.standard_normal(256) for _ in range(3)])
    B = orc.linear_step(p, A, 1e-3)
    for x_ in range(3):
        assert abs(np.linalg.norm(B[x_]) / np.linalg.norm(A[x_]) - 1) <= 1e-14 * 10


def test_loss_only(orc):
    cfg = cw(n=64, alpha=(3.0, 7.0, 11.0))
    p = orc.params(cfg)
    rng = np.random.default_rng(2)
    A = np.stack([rng.standard_normal(64) + 1j * rng.standard_normal(64) for _ in range(3)])
    dz = 2e-3
    B = orc.linear_step(p, A, dz)
    for x_, a in enumerate(cfg.alpha):
        assert rel_l2(B[x_], A[x_] * math.exp(-a * dz / 2)) <= 1e-14


@pytest.mark.parametrize("shift", [3, -5])
def test_gvm_is_exact_shift_to_later_time(orc, shift):
    """A field slower than the signal (dbeta1 > 0) arrives later: +tau."""
    n, T = 128, 10e-12
    dt = T / n
    L = 4e-3
    db1 = shift * dt / L
    cfg = cw(n=n, t_window=T, dbeta1=(db1, 0.0, -db1))
    p = orc.params(cfg)
    rng = np.random.default_rng(3)
    A = np.stack([rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(3)])
    B = orc.linear_step(p, A, L)
    assert rel_l2(B[0], np.roll(A[0], shift)) <= 1e-13
    assert rel_l2(B[1], A[1]) <= 1e-14
    assert rel_l2(B[2], np.roll(A[2], -shift)) <= 1e-13


def _gaussian_grid(n=1024, T=20e-12):
    dt = T / n
    tau = (np.arange(n) - n // 2) * dt
    return tau


def test_gvd_gaussian_closed_form(orc):
    """A0 = exp(-tau^2/2T0^2) -> T0 (T0^2 - i b2 z)^-1/2 exp(-tau^2 / 2(T0^2 - i b2 z))."""
    n, T, T0 = 1024, 20e-12, 0.5e-12
    tau = _gaussian_grid(n, T)
    b2 = 1e-24
    z = T0 ** 2 / b2  # width grows by sqrt(2)
    cfg = cw(n=n, t_window=T, nfields=2, beta2=(b2, -b2, 0.0))
    p = orc.params(cfg)
    A0 = np.exp(-tau ** 2 / (2 * T0 ** 2)).astype(complex)
    B = orc.linear_step(p, np.stack([A0, A0]), z)
    for x_, bb in enumerate((b2, -b2)):
        q = T0 ** 2 - 1j * bb * z
        ref = T0 / np.sqrt(q) * np.exp(-tau ** 2 / (2 * q))
        assert rel_l2(B[x_], ref) <= 1e-12
    w_in = np.sqrt(np.sum(tau ** 2 * abs(A0) ** 2) / np.sum(abs(A0) ** 2))
    w_out = np.sqrt(np.sum(tau ** 2 * abs(B[0]) ** 2) / np.sum(abs(B[0]) ** 2))
    assert abs(w_out / w_in - math.sqrt(2)) <= 1e-9


@pytest.mark.parametrize("b3", [1e-38, -2e-38])
def test_tod_first_moment(orc, b3):
    """<tau> = beta3 z / (4 T0^2) for a Gaussian (Taylor factor 1/6)."""
    n, T, T0 = 2048, 20e-12, 0.5e-12
    tau = _gaussian_grid(n, T)
    z = 0.1
    cfg = cw(n=n, t_window=T, nfields=2, beta3=(b3, 0.0, 0.0))
    p = orc.params(cfg)
    A0 = np.exp(-tau ** 2 / (2 * T0 ** 2)).astype(complex)
    B = orc.linear_step(p, np.stack([A0, A0]), z)
    m1 = np.sum(tau * abs(B[0]) ** 2) / np.sum(abs(B[0]) ** 2)
    assert abs(m1 - b3 * z / (4 * T0 ** 2)) <= 1e-9 * abs(b3 * z / (4 * T0 ** 2))
    assert rel_l2(B[1], A0) <= 1e-14


def test_gdd_cancels_crystal_gvd_and_matches_gaussian(orc):
    n, T, T0 = 1024, 20e-12, 0.4e-12
    tau = _gaussian_grid(n, T)
    b2, L = 3.8e-25, 0.5
    A0 = np.exp(-tau ** 2 / (2 * T0 ** 2)).astype(complex)
    cfg = cw(n=n, t_window=T, nfields=2, length=L, nz=7, deff=0.0, beta2=(0.0, b2, 0.0),
             resonant_mask=0b010, R=(0.0, 1.0, 0.0), gdd=(0.0, -b2 * L, 0.0))
    p = orc.params(cfg)
    st = np.stack([np.zeros(n, complex), A0])
    after_pass = orc.crystal_pass(p, st)
    assert rel_l2(after_pass[1], A0) > 1e-2  # the crystal did disperse it
    back = orc.cavity(p, after_pass, 0)
    assert rel_l2(back[1], A0) <= 1e-12
    # GDD alone acts like GVD with beta2 z -> gamma
    gam = 2e-25
    p2 = orc.params(cfg.replace(gdd=(0.0, gam, 0.0)))
    out = orc.cavity(p2, st, 0)
    q = T0 ** 2 - 1j * gam
    assert rel_l2(out[1], T0 / np.sqrt(q) * np.exp(-tau ** 2 / (2 * q))) <= 1e-12


# ---------------------------------------------- 7-9. nonlinear operator

@pytest.mark.parametrize("dkL", [0.0, 3.0, -1.7])
def test_undepleted_pump_parametric_gain(orc, dkL):
    """A_s(L) = A_s0 e^{i dk L/2}[cosh gL - i dk/(2g) sinh gL],
    A_i(L) = e^{i dk L/2} i kappa_i A_p A_s0* sinh(gL)/g."""
    cfg = cw(n=4, nz=100, length=5e-3)
    k = kappas(cfg)
    L = cfg.length
    Gam = 1.2 / L
    ap = Gam / math.sqrt(k[1] * k[2]) * np.exp(0.3j)
    dk = dkL / L
    cfg = cfg.replace(dk=dk)
    p = orc.params(cfg)
    as0 = 1e-3 * (1 + 0.5j)
    A = np.stack([np.full(4, ap), np.full(4, as0), np.zeros(4, complex)])
    B = orc.crystal_pass(p, A)
    g = np.sqrt(complex(Gam ** 2 - dk ** 2 / 4))
    ph = np.exp(1j * dk * L / 2)
    s_ref = as0 * ph * (np.cosh(g * L) - 1j * dk / (2 * g) * np.sinh(g * L))
    i_ref = ph * 1j * k[2] * ap * np.conj(as0) * np.sinh(g * L) / g
    assert rel_l2(B[1], np.full(4, s_ref)) <= 1e-9
    assert rel_l2(B[2], np.full(4, i_ref)) <= 1e-9
    assert rel_l2(B[0], np.full(4, ap)) <= 1e-12


def test_shg_two_field_closed_form(orc):
    """A_p(0)=0: |A_p(z)| = sqrt(n_s/n_p)|A_s0| tanh(sqrt(n_p/n_s) kappa_p |A_s0| z/2)."""
    cfg = cw(n=4, nfields=2, lam=(0.532e-6, 1.064e-6, 0.0), nidx=(2.23, 2.15, 1.0), nz=200)
    k = kappas(cfg)
    a0 = 1e7
    L = 2.0 / (math.sqrt(cfg.nidx[0] / cfg.nidx[1]) * k[0] * a0 / 2) / 2
    cfg = cfg.replace(length=L)
    p = orc.params(cfg)
    B = orc.crystal_pass(p, np.stack([np.zeros(4, complex), np.full(4, a0 + 0j)]))
    th = math.sqrt(cfg.nidx[0] / cfg.nidx[1]) * k[0] * a0 * L / 2
    assert abs(abs(B[0][0]) - math.sqrt(cfg.nidx[1] / cfg.nidx[0]) * a0 * math.tanh(th)) <= 1e-9 * a0
    assert abs(abs(B[1][0]) - a0 / math.cosh(th)) <= 1e-9 * a0
    # SH phase: dA_p/dz = i(kappa_p/2)A_s^2 with A_s real -> A_p along +i
    assert abs(np.angle(B[0][0]) - math.pi / 2) <= 1e-12


def test_degenerate_quadrature_gain(orc):
    """Undepleted real pump: the pi/4 quadrature grows as e^{kappa_s |A_p| z}, the
    -pi/4 one decays as e^{-kappa_s |A_p| z}."""
    cfg = cw(n=4, nfields=2, lam=(0.532e-6, 1.064e-6, 0.0), nidx=(2.23, 2.15, 1.0), nz=50)
    k = kappas(cfg)
    ap = 1.0 / (k[1] * cfg.length)
    p = orc.params(cfg)
    for phi, sgn in ((math.pi / 4, 1), (-math.pi / 4, -1)):
        as0 = 1e-4 * np.exp(1j * phi)
        B = orc.crystal_pass(p, np.stack([np.full(4, ap + 0j), np.full(4, as0)]))
        assert rel_l2(B[1], np.full(4, as0 * math.exp(sgn * 1.0))) <= 1e-9


def _conserved(cfg, A):
    om = [2 * math.pi * C0 / l for l in cfg.lam]
    e = [cfg.nidx[x] * np.sum(abs(A[x]) ** 2) for x in range(3)]
    return (e[0] + e[1] + e[2], e[1] / om[1] - e[2] / om[2], e[0] / om[0] + e[1] / om[1])


def test_power_and_manley_rowe_conservation(orc):
    """alpha = 0, dk != 0, full dispersion: sum n|A|^2 and the Manley-Rowe
    combinations hold to RK4 truncation, which falls as dz^4."""
    n, T = 64, 4e-12
    tau = (np.arange(n) - n // 2) * T / n
    base = cw(n=n, t_window=T, length=4e-3, dk=800.0, dbeta1=(1e-10, 0, -2e-10),
              beta2=(3.8e-25, 1.1e-25, -7.5e-25), beta3=(2.5e-40, 2.5e-40, 2.5e-40))
    rng = np.random.default_rng(9)
    A = np.stack([
        3e7 * np.exp(-tau ** 2 / (2 * (0.5e-12) ** 2)) * np.exp(0.2j),
        1e7 * np.exp(-(tau - 0.2e-12) ** 2 / (2 * (0.4e-12) ** 2)) + 1e5 * rng.standard_normal(n),
        3e6 * np.exp(-tau ** 2 / (2 * (0.6e-12) ** 2)) * np.exp(-0.7j),
    ])
    c0 = np.array(_conserved(base, A))
    errs = []
    for nz in (10, 20):
        cfg = base.replace(nz=nz)
        B = orc.crystal_pass(orc.params(cfg), A)
        c1 = np.array(_conserved(cfg, B))
        errs.append(abs(c1 - c0) / abs(c0[0]))
        assert np.all(errs[-1] <= 1e-5)
    # some energy moved (the test exercises the coupling) ...
    Bf = orc.crystal_pass(orc.params(base.replace(nz=20)), A)
    assert abs(np.sum(abs(Bf[1]) ** 2) / np.sum(abs(A[1]) ** 2) - 1) > 0.05
    # ... and the conservation error is RK4's: ~16x smaller at half the step
    ratio = errs[0][0] / errs[1][0]
    assert 10.0 <= ratio <= 20.0


def test_symmetrized_step_local_error_is_third_order(orc):
    """Sec. 2.2 Eq. (expon): one symmetrized step has local error O(dz^3)."""
    g = GOLDEN["symmetrized_scheme_local_error_order"]["value"]
    n, T = 64, 4e-12
    tau = (np.arange(n) - n // 2) * T / n
    base = cw(n=n, t_window=T, dbeta1=(3e-10, 0, -3e-10), beta2=(3e-24, 1e-24, -2e-24))
    A = np.stack([
        4e7 * np.exp(-tau ** 2 / (2 * (0.3e-12) ** 2)) + 0j,
        2e7 * np.exp(-(tau - 0.1e-12) ** 2 / (2 * (0.3e-12) ** 2)) + 0j,
        np.zeros(n, complex),
    ])
    def one_step(h, nsub):
        cfg = base.replace(length=h, nz=nsub)
        return orc.crystal_pass(orc.params(cfg), A)
    h0 = 0.4e-3
    errs = []
    for h in (h0, h0 / 2, h0 / 4):
        ref = one_step(h, 64)
        errs.append(rel_l2(one_step(h, 1), ref))
    for a, b in zip(errs, errs[1:]):
        assert abs(math.log2(a / b) - g) <= 0.3


def test_global_error_is_second_order(orc):
    n, T = 64, 4e-12
    tau = (np.arange(n) - n // 2) * T / n
    base = cw(n=n, t_window=T, length=3e-3, dbeta1=(3e-10, 0, -3e-10), beta2=(3e-24, 1e-24, -2e-24))
    A = np.stack([
        4e7 * np.exp(-tau ** 2 / (2 * (0.3e-12) ** 2)) + 0j,
        2e7 * np.exp(-(tau - 0.1e-12) ** 2 / (2 * (0.3e-12) ** 2)) + 0j,
        np.zeros(n, complex),
    ])
    ref = orc.crystal_pass(orc.params(base.replace(nz=1280)), A)
    e = [rel_l2(orc.crystal_pass(orc.params(base.replace(nz=nz)), A), ref) for nz in (10, 20, 40)]
    for a, b in zip(e, e[1:]):
        assert abs(math.log2(a / b) - 2.0) <= 0.25


# ------------------------------------------------------------ cavity, a7

def test_mirror_boundary_condition(orc):
    cfg = cw(n=8, resonant_mask=0b010, R=(0.3, 0.5, 0.7), delta=(1.0, 0.3, -0.4))
    p = orc.params(cfg)
    rng = np.random.default_rng(5)
    A = np.stack([rng.standard_normal(8) + 1j * rng.standard_normal(8) for _ in range(3)])
    B = orc.cavity(p, A, 0)
    assert rel_l2(B[1], A[1] * math.sqrt(0.5) * np.exp(0.3j)) <= 1e-15
    assert np.array_equal(B[0], A[0]) and np.array_equal(B[2], A[2])


def test_eom_jacobi_anger_sidebands(orc):
    """CW x e^{i beta sin(2 pi tau/T)}: bin k carries N J_k(beta) (-1)^k."""
    n, T, beta = 64, 100e-12, 0.7
    cfg = cw(n=n, t_window=T, t_rt=T, resonant_mask=0b010, R=(0, 1.0, 0), eom_beta=beta,
             eom_f=1.0 / T)
    p = orc.params(cfg)
    A = np.stack([np.zeros(n, complex), np.ones(n, complex), np.zeros(n, complex)])
    X = np.fft.fft(orc.cavity(p, A, 0)[1]) / n
    kk = np.fft.fftfreq(n, 1.0 / n).astype(int)
    ref = special.jv(kk, beta) * (-1.0) ** kk
    assert np.max(abs(X - ref)) <= 1e-14


def test_eom_round_trip_index(orc):
    """f_pm t_rt = 1/2: the modulation at m = 1 is the conjugate of m = 0."""
    n, T = 64, 100e-12
    cfg = cw(n=n, t_window=T, t_rt=T, resonant_mask=0b010, R=(0, 1.0, 0), eom_beta=0.5,
             eom_f=0.5 / T)
    p = orc.params(cfg)
    A = np.stack([np.zeros(n, complex), np.ones(n, complex), np.zeros(n, complex)])
    b0 = orc.cavity(p, A, 0)[1]
    b1 = orc.cavity(p, A, 1)[1]
    b2 = orc.cavity(p, A, 2)[1]
    assert np.max(abs(b1 - np.conj(b0))) <= 1e-14
    assert np.max(abs(b2 - b0)) <= 1e-13
    assert np.max(abs(b0 - 1)) > 0.1


@pytest.mark.parametrize("s", [2, -3])
def test_delay_is_exact_shift(orc, s):
    n, T = 64, 10e-12
    cfg = cw(n=n, t_window=T, resonant_mask=0b010, R=(0, 1.0, 0), delay=s * T / n)
    p = orc.params(cfg)
    rng = np.random.default_rng(6)
    A = np.stack([rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(3)])
    B = orc.cavity(p, A, 0)
    assert rel_l2(B[1], np.roll(A[1], s)) <= 1e-13


def test_entry_refreshes_pump_and_dumps_idler(orc):
    cfg = cw(n=8, deff=0.0)
    p = orc.params(cfg)
    pump = orc.pump_profile(p, 0, 5.0)
    A = np.stack([np.full(8, 123.0 + 0j), np.full(8, 2.0 + 0j), np.full(8, 7.0 + 0j)])
    out, trace, outf, st = orc.run(p, A, pump, 0, 1)
    assert st == 0
    assert np.allclose(outf[0], pump, rtol=1e-15, atol=0)
    assert np.all(outf[2] == 0)
    assert np.allclose(outf[1], 2.0 * math.sqrt(1 - 0.98), rtol=1e-15)
    assert np.allclose(out[1], 2.0 * math.sqrt(0.98), rtol=1e-15)


# ----------------------------------------------------- pump, observables

def test_pump_profiles(orc):
    n, T = 1024, 100e-12
    dt = T / n
    cfg = cw(n=n, t_window=T)
    p = orc.params(cfg)
    P = 2.5
    a = orc.pump_profile(p, 0, P)
    assert np.allclose(a, amp_for_power(cfg, P), rtol=1e-15)
    assert abs(orc.power(p, 0, a) - P) <= 1e-13 * P
    fwhm = 40 * dt
    b = orc.pump_profile(p, 1, P, fwhm)
    i0 = n // 2
    assert abs(abs(b[i0]) - amp_for_power(cfg, P)) <= 1e-15 * abs(b[i0])
    assert abs(abs(b[i0 + 20]) ** 2 / abs(b[i0]) ** 2 - 0.5) <= 1e-14
    assert abs(abs(b[i0 - 20]) ** 2 / abs(b[i0]) ** 2 - 0.5) <= 1e-14


def test_power_and_centroid(orc):
    n, T = 256, 100e-12
    cfg = cw(n=n, t_window=T)
    p = orc.params(cfg)
    j = np.arange(n)
    tone = lambda k: np.exp(2j * np.pi * k * j / n)  # noqa: E731
    assert abs(orc.centroid(p, 3.0 * tone(5)) - 5 / T) <= 1e-9 / T
    assert abs(orc.centroid(p, tone(-7)) - (-7 / T)) <= 1e-9 / T
    mix = 2.0 * tone(4) + 1.0 * tone(-2)
    assert abs(orc.centroid(p, mix) - (4 * 4 - 2 * 1) / 5 / T) <= 1e-9 / T
    a = np.full(n, 3e5 + 4e5j)
    ref = 0.5 * cfg.nidx[2] * EPS0 * C0 * (5e5) ** 2 * math.pi * cfg.w0 ** 2
    assert abs(orc.power(p, 2, a) - ref) <= 1e-14 * ref


# --------------------------- fourth-order dispersion and Kerr (chi(3)) terms

def test_beta4_matches_time_domain_fourth_derivative(orc):
    """Fourth-order dispersion in the time domain is dA/dz = i (beta4/24)
    d^4A/dtau^4 (convention-free).  For a Gaussian the fourth derivative is
    (tau^4/T0^8 - 6 tau^2/T0^6 + 3/T0^4) A (Hermite closed form); a short step
    must change A by dz times that, so sign and 1/24 are pinned."""
    n, T = 1024, 20e-12
    t = (np.arange(n) - n / 2) * (T / n)
    T0 = 0.4e-12
    A = np.exp(-t ** 2 / (2 * T0 ** 2)).astype(complex)
    b4 = 1e-52
    cfg = cw(n=n, t_window=T, beta4=(b4, 0.0, 0.0))
    p = orc.params(cfg)
    dz = 1e-6
    out = orc.linear_step(p, np.stack([A, np.zeros(n), np.zeros(n)]), dz)[0]
    d4 = (t ** 4 / T0 ** 8 - 6 * t ** 2 / T0 ** 6 + 3 / T0 ** 4) * A
    ref = 1j * b4 / 24 * d4
    got = (out - A) / dz
    assert rel_l2(got, ref) <= 1e-4


def test_beta4_single_mode_is_a_pure_phase(orc):
    """A single Fourier mode is an eigenfunction of every dispersion order:
    only its phase changes, by the same amount for bins +k and -k (even
    order), and the power is unchanged."""
    n = 64
    cfg = cw(n=n, beta4=(0.0, 3e-52, 0.0))
    p = orc.params(cfg)
    j = np.arange(n)
    for k in (3, 7):
        a = np.stack([np.zeros(n), np.exp(2j * np.pi * k * j / n), np.zeros(n)])
        b = np.stack([np.zeros(n), np.exp(-2j * np.pi * k * j / n), np.zeros(n)])
        oa = orc.linear_step(p, a, 1e-3)[1]
        ob = orc.linear_step(p, b, 1e-3)[1]
        ra = oa / a[1]
        rb = ob / b[1]
        assert np.max(np.abs(np.abs(ra) - 1)) <= 1e-13
        assert np.max(np.abs(ra - ra[0])) <= 1e-12
        assert abs(ra[0] - rb[0]) <= 1e-12


def _kerr_cfg(n2, **kw):
    base = dict(n=4, nz=100, length=5e-3, deff=0.0, n2=n2)
    base.update(kw)
    return W.OPOConfig(**base)


def test_kerr_self_phase_modulation_cw(orc):
    """One CW field with intensity I in a Kerr medium: |A| is unchanged and the
    phase grows by (2 pi / lambda) n2 I L (the nonlinear index n2 I)."""
    n2 = 3e-17
    cfg = _kerr_cfg(n2)
    p = orc.params(cfg)
    a0 = 2.0e7
    A = np.stack([np.full(4, a0 + 0j), np.zeros(4, complex), np.zeros(4, complex)])
    out = orc.crystal_pass(p, A)
    inten = 0.5 * cfg.nidx[0] * EPS0 * C0 * a0 ** 2
    phi = 2 * math.pi / cfg.lam[0] * n2 * inten * cfg.length
    assert 0.05 < phi < 2.0
    assert np.max(np.abs(out[0] - a0 * np.exp(1j * phi))) <= 1e-10 * a0


def test_kerr_cross_phase_modulation_counts_twice(orc):
    """Two CW fields at different wavelengths: each turns by
    (2 pi / lambda_x) n2 (I_x + 2 I_y) L."""
    n2 = 1e-17
    cfg = _kerr_cfg(n2)
    p = orc.params(cfg)
    ap, as_ = 1.5e7, 2.5e7
    A = np.stack([np.full(4, ap + 0j), np.full(4, as_ * 1j), np.zeros(4, complex)])
    out = orc.crystal_pass(p, A)
    Ip = 0.5 * cfg.nidx[0] * EPS0 * C0 * ap ** 2
    Is = 0.5 * cfg.nidx[1] * EPS0 * C0 * as_ ** 2
    php = 2 * math.pi / cfg.lam[0] * n2 * (Ip + 2 * Is) * cfg.length
    phs = 2 * math.pi / cfg.lam[1] * n2 * (Is + 2 * Ip) * cfg.length
    assert np.max(np.abs(out[0] - ap * np.exp(1j * php))) <= 1e-10 * ap
    assert np.max(np.abs(out[1] - 1j * as_ * np.exp(1j * phs))) <= 1e-10 * as_
    assert np.all(out[2] == 0)


def test_kerr_keeps_chi2_exchange_and_total_power(orc):
    """chi(2) + chi(3) together, no loss: the Kerr terms only rotate phases,
    so sum_x n_x |A_x|^2 stays conserved to RK4 accuracy (error ~ dz^4)."""
    cfg = W.OPOConfig(n=64, nz=100, length=10e-3, n2=3e-18)
    p = orc.params(cfg)
    rng = np.random.default_rng(5)
    A = 4e6 * (rng.standard_normal((3, 64)) + 1j * rng.standard_normal((3, 64)))
    out = orc.crystal_pass(p, A)
    e0 = sum(cfg.nidx[x] * np.sum(np.abs(A[x]) ** 2) for x in range(3))
    e1 = sum(cfg.nidx[x] * np.sum(np.abs(out[x]) ** 2) for x in range(3))
    assert abs(e1 - e0) <= 1e-9 * e0
    # and the result differs from the chi(2)-only pass
    q = orc.params(cfg.replace(n2=0.0))
    assert rel_l2(orc.crystal_pass(q, A), out) > 1e-3


# ------------------------------------------- several crystals per round trip

def _as_crystal(cfg, **kw):
    d = dict(length=cfg.length, nz=cfg.nz, dk=cfg.dk, deff=cfg.deff, nidx=cfg.nidx,
             alpha=cfg.alpha, dbeta1=cfg.dbeta1, beta2=cfg.beta2, beta3=cfg.beta3,
             beta4=cfg.beta4, n2=cfg.n2)
    d.update(kw)
    return W.Crystal(**d)


def test_crystal_split_in_two_equals_the_whole(orc):
    """With dk = 0 the step sequence of a crystal cut into two equal halves
    (z restarting in the second) is the same as the whole crystal's: the
    round trip must agree bit for bit."""
    whole = W.cw_sro_16k().replace(n=256, nz=20, n2=1e-19, beta4=(1e-55, 0, 0),
                                   alpha=(0.5, 0.2, 0.1))
    half = whole.replace(length=whole.length / 2, nz=10)
    split = half.replace(extra_crystals=(_as_crystal(half),))
    rng = np.random.default_rng(3)
    A = 1e6 * (rng.standard_normal((3, 256)) + 1j * rng.standard_normal((3, 256)))
    pa, pb = orc.params(whole), orc.params(split)
    pump = orc.pump_profile(pa, 0, whole.pump_power)
    a, ta, oa, _ = orc.run(pa, A, pump, 0, 2)
    b, tb, ob, _ = orc.run(pb, A, pump, 0, 2)
    assert np.array_equal(a, b) and np.array_equal(ta, tb) and np.array_equal(oa, ob)


def test_two_crystals_undepleted_gain_closed_form(orc):
    """Undepleted pump, two crystals with different dk, d_eff and indices, z
    restarting in each: per crystal (u, w) = (A_s e^{-i dk z/2},
    A_i* e^{+i dk z/2}) obey d/dz (u, w) = M (u, w) with
    M = [[-i dk/2, i k_s A_p], [-i k_i A_p*, i dk/2]], so each crystal maps
    (A_s, A_i*) by a 2x2 matrix exponential; the pass is their product."""
    from scipy.linalg import expm
    c1 = W.OPOConfig(n=4, nz=400, length=8e-3, dk=300.0, deff=14e-12)
    c2 = _as_crystal(c1, length=5e-3, nz=300, dk=-150.0, deff=-20e-12,
                     nidx=(2.2, 2.18, 2.1))
    cfg = c1.replace(extra_crystals=(c2,))
    p = orc.params(cfg)
    ap = 3e6 * np.exp(0.4j)
    as0, ai0 = 1.0 + 0.5j, -0.3 + 0.2j
    A = np.stack([np.full(4, ap), np.full(4, as0), np.full(4, ai0)])
    out = orc.crystal_pass(p, A)
    out = orc.crystal_pass(orc.crystal_k(p, 1), out)
    v = np.array([as0, np.conj(ai0)])
    for (L, dk, deff, nidx) in ((c1.length, c1.dk, c1.deff, c1.nidx),
                                (c2.length, c2.dk, c2.deff, c2.nidx)):
        ks = 2 * math.pi * deff / (nidx[1] * c1.lam[1])
        ki = 2 * math.pi * deff / (nidx[2] * c1.lam[2])
        M = np.array([[-0.5j * dk, 1j * ks * ap], [-1j * ki * np.conj(ap), 0.5j * dk]])
        uw = expm(M * L) @ v
        v = np.array([uw[0] * np.exp(0.5j * dk * L), uw[1] * np.exp(-0.5j * dk * L)])
    assert abs(out[1][0] - v[0]) <= 1e-9 * abs(v[0])
    assert abs(np.conj(out[2][0]) - v[1]) <= 1e-9 * abs(v[1])
    # and the run loop passes through both crystals
    pump = np.full(4, ap)
    A2 = A.copy()
    A2[0] = ap
    r, _, _, _ = orc.run(orc.params(cfg.replace(resonant_mask=0b111, R=(1.0, 1.0, 1.0))), A2,
                         0 * pump, 0, 1)
    assert abs(r[1][0] - v[0]) <= 1e-9 * abs(v[0])


def test_dispersion_of_two_crystals_adds(orc):
    """deff = 0: a single Fourier mode turns by sum_k L_k phi_k(Omega)."""
    n, T = 64, 100e-12
    c1 = W.OPOConfig(n=n, nz=7, length=3e-3, deff=0.0, beta2=(0, 2e-25, 0))
    c2 = _as_crystal(c1, length=4e-3, nz=9, beta2=(0, 0, 0), beta3=(0, 5e-39, 0),
                     dbeta1=(0, 1e-12, 0))
    cfg = c1.replace(extra_crystals=(c2,), resonant_mask=0b111, R=(1.0, 1.0, 1.0))
    p = orc.params(cfg)
    k = 5
    om = 2 * math.pi * k / T
    a = np.stack([np.zeros(n), np.exp(2j * np.pi * k * np.arange(n) / n), np.zeros(n)])
    r, _, _, _ = orc.run(p, a, np.zeros(n), 0, 1)
    phi = c1.length * 2e-25 * om ** 2 / 2 + c2.length * (-1e-12 * om - 5e-39 * om ** 3 / 6)
    assert np.max(np.abs(r[1] - a[1] * np.exp(1j * phi))) <= 1e-11


# ------------------------- ns-pulsed pump and pump-resonant (TRO) entry

def _ns_cfg(n=64, **kw):
    base = dict(n=n, nz=4, length=5e-3, t_window=100e-12, nfields=2,
                lam=(0.532e-6, 1.064e-6, 0.0), nidx=(2.23, 2.15, 1.0), deff=0.0,
                pump_kind=W.PUMP_NS, pump_power=75.0, pump_fwhm=1e-9, pump_t0=2e-9)
    base.update(kw)
    return W.OPOConfig(**base)


def test_ns_pump_slice_is_the_gaussian_read_per_round_trip(orc):
    """Sec. 4.2: the long pump is read one round trip at a time.  Peak power
    at t0, half the peak intensity at t0 +- FWHM/2 (the definition of the
    intensity FWHM), and slice m covers t = m t_rt + tau_n."""
    n, T = 64, 100e-12
    cfg = _ns_cfg(n=n)
    p = orc.params(cfg)
    dt = T / n
    # t0 = 2 ns = 20 round trips: tau_n = 0 (n = N/2) of slice 20 is the peak
    a = orc.pump_slice(p, None, 20)
    assert abs(orc.power(p, 0, np.full(n, a[n // 2])) - 75.0) <= 1e-12 * 75.0
    # t0 + FWHM/2 = 2.5 ns = slice 25 at n = N/2 ; t0 - FWHM/2 = slice 15
    for m in (15, 25):
        b = orc.pump_slice(p, None, m)
        assert abs(abs(b[n // 2]) ** 2 / abs(a[n // 2]) ** 2 - 0.5) <= 1e-13
    # every sample: intensity 2^{-(2 (t - t0)/FWHM)^2}, field real and positive
    for m in (0, 7, 19, 33):
        b = orc.pump_slice(p, None, m)
        t = m * T + (np.arange(n) - n / 2) * dt - 2e-9
        ref = 0.5 ** ((2 * t / 1e-9) ** 2)
        assert np.all(b.imag == 0) and np.all(b.real > 0)
        assert np.max(np.abs(abs(b) ** 2 / abs(a[n // 2]) ** 2 - ref)) <= 1e-13
    # the pump table is ignored in this mode
    c = orc.pump_slice(p, np.full(n, 5.0 + 0j), 20)
    assert np.array_equal(c, a)


def test_ns_pump_output_trace_follows_the_pulse(orc):
    """deff = 0, no loss or dispersion, pump not resonant: the output pump
    power of round trip m is the pulse's mean power over that slice."""
    n, T = 64, 100e-12
    cfg = _ns_cfg(n=n)
    p = orc.params(cfg)
    A = np.zeros((2, n), complex)
    _, trace, _, st = orc.run(p, A, None, 0, 40)
    assert st == 0
    dt = T / n
    for m in range(40):
        t = m * T + (np.arange(n) - n / 2) * dt - 2e-9
        ref = 75.0 * np.mean(0.5 ** ((2 * t / 1e-9) ** 2))
        assert abs(trace[m, 0] - ref) <= 1e-12 * 75.0
    # resumed at round trip 17 the slices continue from m = 17
    _, tr2, _, _ = orc.run(p, A, None, 17, 5)
    assert np.array_equal(tr2, trace[17:22])


def test_pump_resonant_entry_sums_a_geometric_series(orc):
    """TRO entry (Sec. 4.2, pump resonant): the input pump is added to the
    circulating pump, which the mirror scales by rho = sqrt(R) e^{i delta}
    each round trip.  With deff = 0 the intracavity pump of round trip m is
    A_in (1 - rho^{m+1}) / (1 - rho) and its output power
    (1 - R) |1 - rho^{m+1}|^2 / |1 - rho|^2 P_in."""
    Rp, dl = 0.9, 0.3
    cfg = cw(n=8, deff=0.0, resonant_mask=0b111, R=(Rp, 0.98, 0.98), delta=(dl, 0.0, 0.0))
    p = orc.params(cfg)
    P = 3.0
    pump = orc.pump_profile(p, 0, P)
    A = np.zeros((3, 8), complex)
    M = 60
    out, trace, outf, st = orc.run(p, A, pump, 0, M)
    assert st == 0
    rho = math.sqrt(Rp) * complex(math.cos(dl), math.sin(dl))
    for m in range(M):
        g = abs(1 - rho ** (m + 1)) ** 2 / abs(1 - rho) ** 2
        assert abs(trace[m, 0] - (1 - Rp) * g * P) <= 1e-12 * (1 - Rp) * g * P
    # state after the last cavity: rho times the last round trip's pump
    ref = pump[0] * rho * (1 - rho ** M) / (1 - rho)
    assert np.max(np.abs(out[0] - ref)) <= 1e-12 * abs(ref)
    assert np.allclose(outf[0], math.sqrt(1 - Rp) * pump[0] * (1 - rho ** M) / (1 - rho),
                       rtol=1e-12, atol=0)


# ------------------------------------------- 10-13. cavity-level physics

@pytest.mark.parametrize("level", [0.9, 1.1, 2.0])
def test_sro_round_trip_gain(orc, level):
    """SRO, idler dumped: small-signal round-trip power gain R cosh^2(Gamma L)."""
    cfg = cw(n=4)
    R = cfg.R[1]
    pth = W.sro_threshold_power(cfg)
    p = orc.params(cfg)
    pump = orc.pump_profile(p, 0, level * pth)
    A = np.stack([np.zeros(4, complex), np.full(4, 1e-3 + 0j), np.zeros(4, complex)])
    out, _, _, st = orc.run(p, A, pump, 0, 1)
    x = math.sqrt(level) * math.acosh(1 / math.sqrt(R))
    gain = np.sum(abs(out[1]) ** 2) / np.sum(abs(A[1]) ** 2)
    assert abs(gain - R * math.cosh(x) ** 2) <= 1e-10


def _dro_map(orc, cfg, power):
    """One-round-trip linear map on (A_s, A_i*) measured with the oracle."""
    p = orc.params(cfg)
    pump = orc.pump_profile(p, 0, power)
    eps = 1e-3
    cols = []
    for s0, i0 in ((eps, 0.0), (0.0, eps)):
        A = np.stack([np.zeros(4, complex), np.full(4, s0 + 0j), np.full(4, i0 + 0j)])
        out, _, _, _ = orc.run(p, A, pump, 0, 1)
        cols.append([out[1][0] / eps, np.conj(out[2][0]) / eps])
    return np.array(cols).T


def _dro_xth(Rs, Ri):
    rs, ri = math.sqrt(Rs), math.sqrt(Ri)
    f = lambda x: (1 - rs * math.cosh(x)) * (1 - ri * math.cosh(x)) - rs * ri * math.sinh(x) ** 2  # noqa: E731
    return brentq(f, 1e-9, 3.0, xtol=1e-15)


def _power_for_gamma_l(cfg, x):
    k = kappas(cfg)
    ap = x / cfg.length / math.sqrt(k[1] * k[2])
    return 0.5 * cfg.nidx[0] * EPS0 * C0 * ap ** 2 * math.pi * cfg.w0 ** 2


def test_dro_threshold_exact_and_paper_formula(orc):
    """Exact plane-wave DRO threshold (1 - r_s cosh x)(1 - r_i cosh x) = r_s r_i sinh^2 x,
    and its small-loss limit, which is Eq. (pth) of Sec. 4.3 with I = n eps0 c |A|^2/2."""
    for Rs, Ri in ((0.98, 0.98), (0.98, 0.80)):
        cfg = cw(n=4, resonant_mask=0b110, R=(0.0, Rs, Ri))
        P = _power_for_gamma_l(cfg, _dro_xth(Rs, Ri))
        rho = max(abs(np.linalg.eigvals(_dro_map(orc, cfg, P))))
        assert abs(rho - 1.0) <= 1e-9
        assert max(abs(np.linalg.eigvals(_dro_map(orc, cfg, 0.97 * P)))) < 1.0
        assert max(abs(np.linalg.eigvals(_dro_map(orc, cfg, 1.03 * P)))) > 1.0
    # small losses: oracle threshold -> Eq. (pth)
    Rs = Ri = 0.999
    cfg = cw(n=4, resonant_mask=0b110, R=(0.0, Rs, Ri))
    lo, hi = 0.5, 2.0
    a_s, a_i = (1 - Rs) / 2, (1 - Ri) / 2
    lam, nn = cfg.lam, cfg.nidx
    p_eq = (EPS0 * C0 * nn[0] * nn[1] * nn[2] * lam[1] * lam[2] * cfg.w0 ** 2
            / (8 * math.pi * cfg.deff ** 2 * cfg.length ** 2) * a_s * a_i)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if max(abs(np.linalg.eigvals(_dro_map(orc, cfg, mid * p_eq)))) > 1.0:
            hi = mid
        else:
            lo = mid
    assert abs(lo - 1.0) <= 2e-3
    # the paper's two printed thresholds follow alpha_s alpha_i of Eq. (pth) to 2%
    g = GOLDEN["dro_threshold_powers_W"]
    (r1s, r1i), (r2s, r2i) = g["reflectivities"]
    pred = ((1 - r1s) * (1 - r1i)) / ((1 - r2s) * (1 - r2i))
    assert abs(g["value"][0] / g["value"][1] / pred - 1) <= 0.02


def _steady(orc, cfg, power, a_start, M=4000):
    p = orc.params(cfg)
    pump = orc.pump_profile(p, 0, power)
    A = np.zeros((cfg.nfields, cfg.n), complex)
    for x in range(1, cfg.nfields):
        A[x] = a_start[x - 1]
    out, tr, _, st = orc.run(p, A, pump, 0, M)
    assert st == 0
    last = tr[-200:]
    assert np.ptp(last[:, 0]) <= 1e-6 * power  # settled
    return out, tr, 1 - tr[-1, 0] / power


@pytest.mark.parametrize("level,eta_ref", [(1.5, None), (2.0, None)])
def test_sro_steady_state_depletion(orc, level, eta_ref):
    """Plane-wave SRO: eta = sin^2 x with N = x^2/sin^2 x (low-loss limit)."""
    cfg = cw(n=4, nz=40)
    P = level * W.sro_threshold_power(cfg)
    x = brentq(lambda x: x * x / math.sin(x) ** 2 - level, 1e-6, math.pi - 1e-6)
    _, _, eta = _steady(orc, cfg, P, [np.full(4, 1e5 + 0j), np.zeros(4, complex)])
    assert abs(eta - math.sin(x) ** 2) <= 3e-3


def _dro_cfg():
    return cw(n=4, nz=40, resonant_mask=0b110, R=(0.0, 0.98, 0.98))


def test_dro_depletion_peaks_at_n4(orc):
    """Sec. 4.3: DRO pump depletion is maximal at N = 4; plane-wave
    eta = 4(sqrt N - 1)/N."""
    cfg = _dro_cfg()
    pth = _power_for_gamma_l(cfg, _dro_xth(0.98, 0.98))
    etas = {}
    for N in (3.0, 4.0, 5.0):
        _, _, etas[N] = _steady(orc, cfg, N * pth, [np.full(4, 1e5 + 0j), np.full(4, 1e5 + 0j)])
        assert abs(etas[N] - 4 * (math.sqrt(N) - 1) / N) <= 3e-3
    nmax = GOLDEN["dro_max_depletion_pumping_level"]["value"]
    assert max(etas, key=etas.get) == nmax


def test_degenerate_phase_and_sqrt_scaling(orc):
    """Sec. 4.4: degenerate OPO signal phase locks to pi/4 or -3pi/4; the
    signal power grows linearly with sqrt(N); depletion is maximal at N = 4."""
    phases = GOLDEN["degenerate_signal_phases_rad"]["value"]
    cfg = cw(n=4, nz=40, nfields=2, lam=(0.532e-6, 1.064e-6, 0.0), nidx=(2.23, 2.15, 1.0),
             R=(0.0, 0.98, 0.0))
    k = kappas(cfg)
    ap_th = math.log(1 / math.sqrt(0.98)) / (k[1] * cfg.length)
    pth = 0.5 * cfg.nidx[0] * EPS0 * C0 * ap_th ** 2 * math.pi * cfg.w0 ** 2
    got = []
    for start in (0.1, math.pi + 0.1):
        out, _, _ = _steady(orc, cfg, 2 * pth, [np.full(4, 1e4 * np.exp(1j * start))])
        got.append(float(np.angle(out[1][0])))
    assert abs(got[0] - phases[0]) <= 1e-6
    assert abs(got[1] - phases[1]) <= 1e-6
    ps, etas = [], {}
    levels = (2.0, 3.0, 4.0, 5.0, 6.0)
    for N in levels:
        _, tr, eta = _steady(orc, cfg, N * pth, [np.full(4, 1e4 * np.exp(0.1j))])
        ps.append(tr[-1, 1])
        etas[N] = eta
    sq = np.sqrt(levels)
    slope, icpt = np.polyfit(sq, ps, 1)
    resid = np.array(ps) - (slope * sq + icpt)
    assert np.max(abs(resid)) <= 0.01 * max(ps)
    assert abs(-icpt / slope - 1.0) <= 0.03
    assert max(etas, key=etas.get) == GOLDEN["dro_max_depletion_pumping_level"]["value"]


def test_too_large_dz_reports_nonfinite(orc):
    """Sec. 2.4: too large a dz makes the fields blow up (NaN); the oracle
    reports it through its status."""
    cfg = cw(n=4, nz=1, length=0.5)
    p = orc.params(cfg)
    pump = orc.pump_profile(p, 0, 1e12)
    A = np.stack([np.zeros(4, complex), np.full(4, 1e8 + 0j), np.full(4, 1e8 + 0j)])
    _, _, _, st = orc.run(p, A, pump, 0, 50)
    assert st == 1

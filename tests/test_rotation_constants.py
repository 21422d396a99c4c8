"""The single-precision rotation constants e^{2 pi i a/32} of the in-register
DFTs (csrc/opo_common.cuh, c32f / s32f): each pair lies within two units in
the last place of the nearest floats of cos and sin, its phase is within
1e-7 rad, and the modulus errors |w|^2 - 1 of every pair (a, 16 - a), which
each DFT uses equally often, cancel to below 1.6e-8, so that no DFT radix
carries a systematic modulus bias (the nearest floats all fall short of 1,
by a summed -6.9e-8, -3.0e-7 and -5.9e-7 at radix 8, 16 and 32)."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2410_02532_gb300", "csrc", "opo_common.cuh")


def _table(name):
    text = open(SRC).read()
    m = re.search(r"constexpr float %s\[16\] = \{([^}]*)\};" % name, text)
    assert m, name
    vals = [float(v.strip().rstrip("f")) for v in m.group(1).split(",")]
    assert len(vals) == 16
    return np.array(vals, dtype=np.float32)


def _ulps(x, ref):
    """Distance in float32 steps between x and the nearest float of ref."""
    n = np.float32(ref)
    k = 0
    a = n
    while a != x and k < 8:
        a = np.nextafter(a, np.float32(np.inf) if x > n else np.float32(-np.inf))
        k += 1
    return k


def test_balanced_rotation_constants():
    c, s = _table("c32f"), _table("s32f")
    th = 2 * np.pi * np.arange(16) / 32
    err = c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2 - 1.0
    # a = 0 and a = 8 (1 and i) are exact and applied as an identity and a
    # swap; the other fourteen are the rounded pairs
    assert (c[0], s[0], c[8], s[8]) == (1.0, 0.0, 0.0, 1.0)
    for a in [a for a in range(16) if a not in (0, 8)]:
        assert _ulps(c[a], np.cos(th[a])) <= 2, a
        assert _ulps(s[a], np.sin(th[a])) <= 2, a
        phase = np.arctan2(float(s[a]), float(c[a])) - th[a]
        assert abs(phase) < 1e-7, (a, phase)
    assert err[0] == 0.0 and err[8] == 0.0
    for a in range(1, 8):
        assert abs(err[a] + err[16 - a]) < 1.6e-8, (a, err[a], err[16 - a])
    # per radix R the DFT uses A = 0, 32/R, ..., 16 - 32/R
    for R, limit in ((8, 1.6e-8), (16, 1.6e-8), (32, 1.7e-8)):
        total = sum(err[A] for A in range(0, 16, 32 // R))
        assert abs(total) < limit, (R, total)
    # the nearest floats, for contrast, are biased low at every radix
    near = (np.cos(th).astype(np.float32).astype(np.float64) ** 2
            + np.sin(th).astype(np.float32).astype(np.float64) ** 2 - 1.0)
    for R in (8, 16, 32):
        assert sum(near[A] for A in range(0, 16, 32 // R)) < -6e-8

"""Write the oracle's steady state of the 2^14-point CW singly resonant OPO.

Workload: the 2^14-point, 3-field, 20 mm, 100-step CW SRO with GVM, GVD, TOD
and intracavity GDD -500 fs^2 on the signal, pump at 4x the plane-wave
threshold, started from the seeded 1e-15 V/m signal/idler noise (the
workload preset ``cw_sro_16k`` of the seeded input generator).  The method is
the paper's: entry, crystal pass by the symmetrized split-step method with
RK4 (Sec. 2.2, Eq. (expon)), observables, cavity boundary condition (Sec. 2.1
Eq. (BC)) and GDD (Sec. 2.3 item 1), repeated for many round trips (Sec. 2.4).

The script calls only the FP64 oracle (``oracle/``) and the input generator.
It runs ``--rt`` round trips (0 .. rt-1) from the noise start and stores in
``steady_state_cw_sro_16k.json``:

  rt             round trips run
  last           K = max(10, ceil(rt/10)) round trips averaged
  p_out_mean_W   mean output power per field over the last K round trips
  centroid_mean_hz  mean signal spectral centroid over the last K round trips
  width_hz       rms spectral width of the last output signal (the centroid's
                 tolerance scale; floored at half a bin by the test)
  window_drift   relative change of the mean P_s,out between the last two
                 K-round-trip windows (how far from stationary the mean is)
  centroid_window_drift_hz  change of the mean centroid between those windows
                 (the signal spectrum keeps walking slowly after the power
                 has settled, so GPU and oracle are compared after the same
                 number of round trips)
  p_s_every_10   output signal power at every 10th round trip

  python tests/golden/make_steady_state.py [--rt 3000] [--trace FILE.npy]

The settled state after 20000 round trips (about four hours of one core):

  python tests/golden/make_steady_state.py --rt 20000 \
      --out tests/golden/steady_state_cw_sro_16k_long.json
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_2410_02532_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "steady_state_cw_sro_16k.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rt", type=int, default=3000)
    ap.add_argument("--chunk", type=int, default=100)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--trace", default="", help="also save the full trace (rt x 4) as .npy")
    args = ap.parse_args()

    cfg = W.cw_sro_16k()
    p = orc.params(cfg)
    pump = orc.pump_profile(p, cfg.pump_kind, cfg.pump_power, cfg.pump_fwhm)
    a = cfg.initial_fields()
    traces = []
    out_fields = None
    m = 0
    t0 = time.time()
    while m < args.rt:
        k = min(args.chunk, args.rt - m)
        a, tr, out_fields, st = orc.run(p, a, pump, m, k)
        if st != 0:
            raise SystemExit("oracle reported a non-finite field at round trip %d" % m)
        traces.append(tr)
        m += k
        print("rt %5d  P_s,out %.6e W  (%.0f s)" % (m, tr[-1, 1], time.time() - t0), flush=True)
        if args.trace:
            np.save(args.trace, np.concatenate(traces))
    full = np.concatenate(traces)
    K = max(10, math.ceil(m / 10))
    X = np.abs(np.fft.fft(out_fields[1])) ** 2
    f = np.fft.fftfreq(cfg.n, cfg.t_window / cfg.n)
    mu = float(np.sum(f * X) / np.sum(X))
    width = float(np.sqrt(np.sum((f - mu) ** 2 * X) / np.sum(X)))
    last, prev = full[-K:, 1].mean(), full[-2 * K:-K, 1].mean()
    rec = {
        "_about": "FP64 oracle steady state of the 2^14-point CW SRO workload (cw_sro_16k: "
                  "GVM, GVD, TOD, GDD -500 fs^2, 4x threshold) from the seeded 1e-15 V/m "
                  "noise start; Sec. 2.1 Eq. (BC), Sec. 2.2 Eq. (expon), Sec. 2.3 item 1, "
                  "Sec. 2.4.  Written by tests/golden/make_steady_state.py, which calls "
                  "only oracle/ and the seeded input generator.",
        "workload": cfg.name,
        "rt": m,
        "last": K,
        "p_out_mean_W": [float(full[-K:, x].mean()) for x in range(3)],
        "centroid_mean_hz": float(full[-K:, 3].mean()),
        "width_hz": width,
        "window_drift": float(abs(last - prev) / last),
        "centroid_window_drift_hz": float(full[-K:, 3].mean() - full[-2 * K:-K, 3].mean()),
        "p_s_every_10": [float(v) for v in full[9::10, 1]],
        "oracle_seconds": time.time() - t0,
    }
    with open(args.out, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps({k: v for k, v in rec.items() if k != "p_s_every_10"}, indent=1))


if __name__ == "__main__":
    main()

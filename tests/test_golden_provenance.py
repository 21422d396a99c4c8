"""The stored steady-state runs come from the oracle as it stands.

tests/golden/steady_state_cw_sro_16k.json (3000 round trips) and
tests/golden/steady_state_cw_sro_16k_long.json (20000 round trips) were
written by tests/golden/make_steady_state.py from the FP64 oracle alone.
Re-running the oracle's first 20 round trips from the same seeded noise
start must give the first two stored output signal powers (round trips 9
and 19) exactly: any change to the oracle's arithmetic since then breaks
this test, and the stored runs must then be written again.
"""
import json
import os

import numpy as np

from oracle import oracle as orc
from paper_2410_02532_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FILES = ("steady_state_cw_sro_16k.json", "steady_state_cw_sro_16k_long.json")


def test_steady_state_goldens_match_the_oracle_start():
    cfg = W.cw_sro_16k()
    p = orc.params(cfg)
    pump = orc.pump_profile(p, cfg.pump_kind, cfg.pump_power, cfg.pump_fwhm)
    _, tr, _, st = orc.run(p, cfg.initial_fields(), pump, 0, 20)
    assert st == 0
    for name in FILES:
        ref = json.load(open(os.path.join(GOLDEN, name)))
        assert ref["workload"] == cfg.name
        assert ref["rt"] == 10 * len(ref["p_s_every_10"])
        got = [float(tr[9, 1]), float(tr[19, 1])]
        assert got == ref["p_s_every_10"][:2], (name, got, ref["p_s_every_10"][:2])


def test_steady_state_goldens_agree_where_they_overlap():
    """The long run repeats the short one for its first 3000 round trips."""
    a = json.load(open(os.path.join(GOLDEN, FILES[0])))
    b = json.load(open(os.path.join(GOLDEN, FILES[1])))
    n = len(a["p_s_every_10"])
    assert np.array_equal(np.array(a["p_s_every_10"]), np.array(b["p_s_every_10"][:n]))

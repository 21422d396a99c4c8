"""Host-side pieces of the serving layer (no GPU)."""
from paper_2410_02532_gb300 import serving


def test_poisson_trace_is_seeded_and_in_range():
    a = serving.poisson_trace(50, 100.0)
    b = serving.poisson_trace(50, 100.0)
    assert [(r.arrival, r.cfg.n, r.rounds, r.cfg.nfields) for r in a] == \
           [(r.arrival, r.cfg.n, r.rounds, r.cfg.nfields) for r in b]
    assert all(a[i].arrival < a[i + 1].arrival for i in range(49))
    assert {r.cfg.n for r in a} <= {4096, 8192, 16384, 32768}
    assert all(100 <= r.rounds <= 5000 for r in a)
    assert {r.cfg.nfields for r in a} <= {2, 3}
    mean_gap = (a[-1].arrival - a[0].arrival) / 49
    assert 0.005 < mean_gap < 0.02


def test_instance_bytes_and_work():
    assert serving.instance_bytes(1 << 14, 3, 1) < serving.instance_bytes(1 << 14, 3, 0)
    r = serving.poisson_trace(1, 1.0)[0]
    assert serving.request_work(r) == r.cfg.n * r.cfg.nfields * r.cfg.nz * r.rounds

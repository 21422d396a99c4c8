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


def test_autotune_classes_follow_the_kernel_variant():
    """The tuner keys a class by the nonlinear-step variant as the library
    picks its kernel: Kerr terms anywhere, else a phase mismatch anywhere,
    else the dk = 0 kernel; and its cache round-trips through a JSON file."""
    import os
    import tempfile

    from paper_2410_02532_gb300 import autotune as A
    from paper_2410_02532_gb300 import workloads as W

    base = W.cw_sro_16k()
    assert base.dk == 0.0 and base.n2 == 0.0
    assert A.variant(base) == "chi2_dk0"
    assert A.variant(base.replace(dk=10.0)) == "chi2"
    assert A.variant(base.replace(n2=2e-19)) == "kerr"
    assert A.variant(base.replace(dk=10.0, n2=2e-19)) == "kerr"
    second = W.Crystal(length=1e-3, nz=2, dk=5.0)
    assert A.variant(base.replace(extra_crystals=(second,))) == "chi2"
    keys = {A._key(base.n, base.nfields, 1, v) for v in ("chi2", "chi2_dk0", "kerr")}
    assert len(keys) == 3
    shape = {"cluster": 4, "threads": 512, "rt_per_launch": 64, "field_steps_per_s": 1.0}
    with A._lock:
        A._cache[A._key(base.n, base.nfields, 1, "kerr")] = shape
    try:
        assert A.lookup(base.n, base.nfields, 1, "kerr") == shape
        assert A.lookup(base.n, base.nfields, 1, "chi2_dk0") is None
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "tune.json")
            A.save(path)
            with A._lock:
                A._cache.clear()
            A.load(path)
            assert A.lookup(base.n, base.nfields, 1, "kerr") == shape
    finally:
        with A._lock:
            A._cache.clear()


def test_autotune_pick_prefers_larger_ctas_within_one_percent():
    from paper_2410_02532_gb300 import autotune as A

    assert A.pick([]) is None
    r = [{"cluster": 8, "threads": 128, "field_steps_per_s": 100.0},
         {"cluster": 4, "threads": 512, "field_steps_per_s": 99.5},
         {"cluster": 4, "threads": 384, "field_steps_per_s": 99.8},
         {"cluster": 16, "threads": 512, "field_steps_per_s": 90.0}]
    best = A.pick(r)
    assert (best["cluster"], best["threads"], best["candidates"]) == (4, 512, 4)
    # outside the 1% band the fastest wins whatever its CTA size
    r[1]["field_steps_per_s"] = 98.0
    r[2]["field_steps_per_s"] = 98.9
    assert (A.pick(r)["cluster"], A.pick(r)["threads"]) == (8, 128)

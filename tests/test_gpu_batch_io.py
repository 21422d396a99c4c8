"""Overlapped host transfers of a batch (opo_batch_step_io) against the same
steps done with the synchronous calls: bit for bit the same output fields
and trace rows, on fused and plain members, with the two staging slots
alternating and the host buffers reused by every step."""
import numpy as np
import pytest

from paper_2410_02532_gb300 import opo
from paper_2410_02532_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _members():
    b = W.cw_sro_16k().replace(n=1 << 12, nz=4)
    return [b.replace(instance=1), b.replace(instance=2, pump_power=b.pump_power * 1.3),
            b.replace(instance=3, delay=6e-15)]


def _starts(cfgs):
    out = []
    for c in cfgs:
        a = c.initial_fields()
        for x in range(1, c.nfields):
            a[x] = a[x] + W.noise(c.n, 2e6, c.seed + 5, c.instance, x)
        out.append(a)
    return out


@pytest.mark.parametrize("path", [opo.OPO_PATH_FUSED, opo.OPO_PATH_PLAIN], ids=["fused", "plain"])
def test_step_io_matches_synchronous_steps(path):
    cfgs = _members()
    starts = _starts(cfgs)
    host = np.concatenate([np.asarray(a, dtype=np.complex128).reshape(-1) for a in starts])
    steps, field, m = 5, 1, 2
    total_n = sum(c.n for c in cfgs)

    def make():
        ctxs = [opo.Context(c) for c in cfgs]
        for x in ctxs:
            x.set_path(path)
        return ctxs, opo.opo_batch_create([x.h for x in ctxs])

    # synchronous: every step re-loads the same start, runs m round trips and
    # reads the output signal and the last trace row
    ctxs, b = make()
    ref = []
    for _ in range(steps):
        opo.opo_batch_set_fields(b, host)
        opo.opo_batch_run(b, m)
        f = opo.opo_batch_get_fields(b, field, opo.OPO_OUTPUT, total_n)
        t = opo.opo_batch_get_trace(b, len(cfgs), m)[:, -1, :]
        ref.append((f, t))
    opo.opo_batch_destroy(b)
    for x in ctxs:
        x.close()

    ctxs, b = make()
    h_in = torch.from_numpy(host.view(np.float64).copy()).pin_memory()
    h_out = torch.zeros(2 * total_n + 4 * len(cfgs), dtype=torch.float64).pin_memory()
    for k in range(steps):
        opo.opo_batch_step_io(b, h_in.data_ptr(), h_out.data_ptr(), field, m)
        if k in (0, steps - 1):
            # the buffer is written by the last enqueued step only
            opo.opo_batch_io_wait(b)
            got = h_out.numpy().copy()
            f = got[:2 * total_n].view(np.complex128)
            t = got[2 * total_n:].reshape(len(cfgs), 4)
            assert np.array_equal(f, ref[k][0]), k
            assert np.array_equal(t, ref[k][1]), k
    opo.opo_batch_destroy(b)
    for x in ctxs:
        x.close()


def test_step_io_rejects_bad_arguments():
    cfgs = _members()
    ctxs = [opo.Context(c) for c in cfgs]
    b = opo.opo_batch_create([x.h for x in ctxs])
    L = opo.lib()
    assert L.opo_batch_step_io(b, None, None, 0, 0) == opo.OPO_E_INVALID
    assert L.opo_batch_step_io(b, None, None, -1, 1) == opo.OPO_E_INVALID
    assert L.opo_batch_step_io(b, None, None, 3, 1) == opo.OPO_E_INVALID
    # neither buffer: just the round trips
    assert L.opo_batch_step_io(b, None, None, 0, 1) == opo.OPO_OK
    assert L.opo_batch_io_wait(b) == opo.OPO_OK
    opo.opo_batch_destroy(b)
    for x in ctxs:
        x.close()

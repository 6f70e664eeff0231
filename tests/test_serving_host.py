"""Host side of the serving loop: pool allocator, footprints, admission, trace.

No GPU: the server runs on a CPU pool with a stand-in executor that sleeps,
which exercises the scheduler (slots, admission by footprint, bypass limit,
retirement) exactly as on the GPU.
"""
import threading
import time

import numpy as np
import pytest

import paper_1601_04280_gb300 as rg
from paper_1601_04280_gb300 import serving
from rlu_inputs import serving as rs

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    rg.build()
    rg.load(reload=True)


def test_pool_first_fit_and_coalescing():
    pool = serving.DevicePool(10 * 256, device="cpu")
    a = pool.alloc(256)
    b = pool.alloc(300)       # two granules
    c = pool.alloc(256)
    assert (a, b, c) == (0, 256, 768)
    assert pool.alloc(7 * 256) is None
    pool.free(b, 300)
    assert pool.alloc(512) == 256          # reuses the hole
    pool.free(256, 512)
    pool.free(a, 256)
    pool.free(c, 256)
    assert pool.free_ranges == [(0, 10 * 256)] and pool.in_use == 0


def test_pool_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(0)
    pool = serving.DevicePool(1 << 20, device="cpu")
    live = {}
    for step in range(3000):
        if live and rng.random() < 0.45:
            off = list(live)[rng.integers(len(live))]
            pool.free(off, live.pop(off))
        else:
            size = int(rng.integers(1, 40000))
            off = pool.alloc(size)
            if off is not None:
                live[off] = size
        spans = sorted((o, o + serving._up(s)) for o, s in live.items())
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0
        assert pool.in_use == sum(serving._up(s) for s in live.values())
    for off, size in list(live.items()):
        pool.free(off, size)
    assert pool.free_ranges == [(0, pool.nbytes)]


def test_footprint_is_workspace_plus_outputs():
    up = serving._up
    ws = rg.rlu_workspace_bytes(3000, 2000, 40, 60, 320, "f32")
    outs = sum(up(b) for b in (4 * 3000 * 40, 4 * 40 * 2000, 8 * 3000, 8 * 2000, 4))
    r = serving.Request(0, 3000, 2000, 40, 60, 320, 7)       # no input: as if resident on the device
    assert serving.footprint(r) == up(ws) + outs
    # a host-resident input also holds its device copy
    rh = serving.Request(0, 3000, 2000, 40, 60, 320, 7, A=torch.zeros(3000, 2000))
    assert serving.footprint(rh) == up(ws) + up(4 * 3000 * 2000) + outs
    csr = (torch.zeros(3001, dtype=torch.int64), torch.zeros(12345, dtype=torch.int32), torch.zeros(12345))
    rc = serving.Request(1, 3000, 2000, 40, 60, 320, 7, csr=csr)
    cws = rg.rlu_csr_workspace_bytes(3000, 2000, 40, 12345)
    assert serving.footprint(rc) == up(ws) + up(cws) + up(8 * 3001) + up(4 * 12345) + up(4 * 12345) + outs


def test_csr_workspace_grows_with_entries_and_is_bounded():
    small = rg.rlu_csr_workspace_bytes(1000, 800, 20, 1000)
    big = rg.rlu_csr_workspace_bytes(1000, 800, 20, 200000)
    assert big > small
    # heavy rows hold >= n/4 entries each: the dense copy is bounded by the
    # entries; the sort of the light entries by column holds two slots of
    # (column key, row, value) = 4 + 4 + 8 bytes per entry
    assert big < small + 200000 * (8 + 4 * 8 + 8 + 2 * 16) + 20 * 1000 * 8 + (1 << 22)
    with pytest.raises(rg.RluError):
        rg.rlu_csr_workspace_bytes(1000, 800, 20, -1)


class FakeServer(serving.Server):
    """The scheduler with a stand-in executor: sleeps in proportion to size."""

    def __init__(self, *a, **kw):
        super().__init__(*a, device="cpu", **kw)
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.max_bytes = 0
        self.order = []

    def _execute(self, req, carve, stream, sptr, slot=0):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.max_bytes = max(self.max_bytes, self.pool.in_use)
            self.order.append(req.rid)
        time.sleep(0.002 + 1e-9 * req.m * req.n)
        with self.lock:
            self.active -= 1
        return rg.RLU_OK, None


def _reqs(specs, rate=None):
    out, t = [], 0.0
    for s in specs:
        t += s.gap / rate if rate else 0.0
        out.append(serving.Request(s.rid, s.m, s.n, s.k, s.l, s.l1, 5, t_arrive=t))
    return out


def test_scheduler_respects_slots_and_pool():
    specs = [s for s in rs.make_trace(60, seed=3, size_max=2048)]
    reqs = _reqs(specs)
    fps = [serving.footprint(r) for r in reqs]
    pool_bytes = 3 * max(fps)
    with FakeServer(pool_bytes, slots=4) as srv:
        res, span = srv.run(reqs, open_loop=False)
    assert [r.rid for r in res] == [q.rid for q in reqs]
    assert all(r.status == rg.RLU_OK for r in res)
    assert srv.max_active <= 4
    assert srv.max_bytes <= srv.pool.nbytes
    assert srv.pool.in_use == 0 and srv.pool.free_ranges == [(0, srv.pool.nbytes)]
    assert span > 0


def test_scheduler_open_loop_latency_includes_queueing():
    specs = rs.make_trace(40, seed=4, size_max=1024)
    reqs = _reqs(specs, rate=2000.0)    # arrivals faster than one slot serves
    with FakeServer(1 << 34, slots=1) as srv:
        res, span = srv.run(reqs, open_loop=True)
    for r in res:
        assert r.t_admit >= r.t_arrive - 1e-6
        assert r.t_done >= r.t_admit
    lat = [r.latency for r in res]
    assert lat[-1] > lat[0]     # a queue builds up behind one slot
    s = serving.summarize(res, span)
    assert s["requests"] == 40 and s["ok"] == 40 and s["p99_ms"] >= s["p50_ms"]


def test_scheduler_bypass_is_bounded():
    # a large head that only fits once the pool is empty, behind small ones in flight
    small = [serving.Request(i if i < 3 else i + 1, 600, 600, 16, 36, 128, 1) for i in range(12)]
    big = serving.Request(3, 4000, 4000, 200, 220, 1600, 1)
    reqs = small[:3] + [big] + small[3:]      # arrival order = rid order
    pool_bytes = serving.footprint(big) + serving.footprint(small[0])
    with FakeServer(pool_bytes, slots=3, max_bypass=2) as srv:
        res, _ = srv.run(reqs, open_loop=False)
    assert all(r.status == rg.RLU_OK for r in res)
    # the big request is admitted after at most max_bypass later requests passed it
    order = [r.rid for r in sorted(res, key=lambda r: r.t_admit)]
    assert order.index(3) <= 3 + 2


def test_trace_is_seeded_and_shaped():
    a = rs.make_trace(4096, seed=2004)
    b = rs.make_trace(4096, seed=2004)
    assert a == b
    m = np.array([s.m for s in a])
    n = np.array([s.n for s in a])
    k = np.array([s.k for s in a])
    assert m.min() >= 512 and m.max() <= 16384 and n.min() >= 512 and n.max() <= 16384
    assert k.min() >= 16 and k.max() <= 256
    assert all(s.l == s.k + 20 and s.l1 == 8 * s.k for s in a)
    dense = np.mean([s.kind == "dense" for s in a])
    assert 0.67 < dense < 0.73
    # log-uniform: the median of log m sits in the middle of [log 512, log 16384]
    assert abs(np.median(np.log(m)) - 0.5 * (np.log(512) + np.log(16384))) < 0.15
    gaps = np.array([s.gap for s in a])
    assert abs(gaps.mean() - 1.0) < 0.06


class FailingServer(FakeServer):
    """Injected failures: request 2 raises inside the executor (reported as a
    failed request); request 5 ends its worker thread (the scheduler must
    notice instead of waiting forever)."""

    def _execute(self, req, carve, stream, sptr, slot=0):
        if req.rid == 2:
            raise ValueError("injected")
        if req.rid == 5:
            raise SystemExit
        return super()._execute(req, carve, stream, sptr, slot)


def test_executor_error_is_a_failed_request():
    reqs = [serving.Request(i, 600, 600, 16, 36, 128, 1) for i in range(4)]
    with FailingServer(1 << 32, slots=2) as srv:
        res, _ = srv.run(reqs, open_loop=False)
    assert [r.status for r in res] == [rg.RLU_OK, rg.RLU_OK, -1, rg.RLU_OK]
    assert "injected" in res[2].outputs


def test_dead_worker_is_detected():
    reqs = [serving.Request(i, 600, 600, 16, 36, 128, 1) for i in range(8)]
    srv = FailingServer(1 << 32, slots=1)
    t0 = time.perf_counter()
    with pytest.raises(RuntimeError, match="worker stopped"):
        srv.run(reqs, open_loop=False)
    assert time.perf_counter() - t0 < 10

"""Host logic of the server (admission order, chunking, completion) against a
fake batch that does the bookkeeping only; no GPU."""
import types

import numpy as np

from paper_1804_06205_gb300 import serving
from paper_1804_06205_gb300.workloads import Request


class FakeBatch:
    def __init__(self, cap):
        self.cap, self.used, self.next = cap, 0, 0
        self.live = {}
        self.steps = []

    def add_workload(self, w, tile_cells=0):
        if self.used + w.n > self.cap:
            return None
        s = self.next
        self.next += 1
        self.live[s] = [w.n, 0]
        self.used += w.n
        return s

    def step(self, k):
        self.steps.append((k, sorted(self.live)))
        for v in self.live.values():
            v[1] += k

    def sync(self):
        pass

    def get_state(self, s, force=True):
        return (None, None, None, self.live[s][1])

    def remove(self, s):
        self.used -= self.live.pop(s)[0]

    def close(self):
        pass


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001
        return self.t


def fake_server(cap, chunk):
    srv = serving.Server.__new__(serving.Server)
    srv.batch = FakeBatch(cap)
    srv.chunk, srv.table, srv.keep = chunk, None, True
    srv.clock, srv.max_resident, srv.chunks, srv.busy_s = FakeClock(), 0, 0, 0.0
    return srv


def req(rid, t, steps, n):
    w = types.SimpleNamespace(n=n, L=np.array([8.0, 8.0, 8.0]))
    return Request(rid, t, steps, w)


def test_each_request_runs_exactly_its_steps():
    reqs = [req(0, 0.0, 23, 10), req(1, 0.0, 17, 10), req(2, 0.002, 31, 10), req(3, 0.004, 9, 10)]
    srv = fake_server(cap=1000, chunk=7)
    done = srv.run(reqs)
    assert sorted(d.rid for d in done) == [0, 1, 2, 3]
    for d in done:
        assert d.state[3] == reqs[d.rid].steps
    assert all(k <= 7 for k, _ in srv.batch.steps)


def test_admission_is_first_come_first_served_and_waits_for_room():
    reqs = [req(0, 0.0, 20, 60), req(1, 0.0, 20, 60), req(2, 0.0, 5, 10)]
    srv = fake_server(cap=100, chunk=50)
    done = srv.run(reqs)
    # request 1 does not fit next to 0; request 2 would fit but must not pass it
    first = srv.batch.steps[0][1]
    assert first == [0]
    order = [d.rid for d in done]
    assert order.index(0) < order.index(1)
    assert max(len(ids) for _, ids in srv.batch.steps) <= 2


def test_summary_percentiles():
    done = [serving.Completed(i, 100, 10, 0.0, 0.0, float(i + 1)) for i in range(100)]
    s = serving.summarize(done)
    assert abs(s["p50_latency_s"] - 50.5) < 1e-9
    assert abs(s["p99_latency_s"] - 99.01) < 1e-9
    assert s["particle_steps"] == 100 * 100 * 10


def test_tile_table_lookup_picks_nearest_edge():
    t = {"threads": 128, "tiles": {"8.0": 3, "16.0": 5, "24.0": 7}}
    assert serving.tile_for(t, np.array([9.0, 9.0, 9.0])) == 3
    assert serving.tile_for(t, np.array([21.0, 21.0, 21.0])) == 7
    assert serving.tile_for(None, np.array([9.0, 9.0, 9.0])) == 0

"""The continuous-batching server on the GPU: every request's final state
equals its alone run bit for bit, whatever the systems it shared the batch
with and the chunk boundaries, and requests that do not fit wait."""
import numpy as np
import pytest

from paper_1804_06205_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    from paper_1804_06205_gb300 import build
    build.build()
    from paper_1804_06205_gb300 import dpd
    return dpd


def mini_stream():
    spec = [(0, 0.00, 23, 8.0), (1, 0.00, 17, 9.3), (2, 0.00, 31, 8.6), (3, 0.01, 9, 10.1),
            (4, 0.05, 26, 8.2), (5, 0.30, 14, 9.0)]
    return [W.Request(rid, t, steps, W.serving_system(40 + rid, edge=e, a_ab=30.0 + rid))
            for rid, t, steps, e in spec]


def alone(D, w, nsteps):
    g = D.System.from_workload(w, precision=0)
    g.set_state(w.pos, w.vel, 0)
    g.step(nsteps)
    out = g.get_state()
    g.close()
    return out


@pytest.mark.parametrize("tight", [False, True])
def test_served_results_equal_alone_runs(D, tight):
    from paper_1804_06205_gb300 import serving
    reqs = mini_stream()
    if tight:   # room for the first two requests only: the third waits for a departure
        cap = reqs[0].workload.n + reqs[1].workload.n + 10
        assert all(r.workload.n <= cap for r in reqs)
        srv = serving.Server(max_beads=cap, max_cells=10 ** 5, max_bonds=10 ** 5,
                             max_systems=8, chunk=7, keep_states=True)
    else:
        srv = serving.Server(max_beads=10 ** 6, max_cells=10 ** 6, max_bonds=10 ** 5,
                             max_systems=16, chunk=7, keep_states=True)
    done = srv.run(reqs)
    srv.close()
    assert sorted(d.rid for d in done) == list(range(len(reqs)))
    first_done = min(d.done_s for d in done)
    if tight:   # some request that arrived at once had to wait for a departure
        assert srv.max_resident < len(reqs)
        assert any(d.admit_s >= first_done for d in done if d.arrival_s < first_done)
    else:   # the first three arrive together and are admitted together
        assert srv.max_resident >= 3
    for d in done:
        r = reqs[d.rid]
        ref = alone(D, r.workload, r.steps)
        assert d.state[3] == r.steps
        assert np.array_equal(d.state[0], ref[0]) and np.array_equal(d.state[1], ref[1])
        assert d.admit_s >= d.arrival_s - 1e-9 and d.done_s > d.admit_s
    s = serving.summarize(done)
    assert s["requests"] == len(reqs) and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_autotuned_tiles_are_applied_and_results_equal_alone(D):
    """The autotuner's table (threads per block, brick length per box-edge
    class) reaches every admitted system, and each served result still equals
    its alone run with the same launch shape, bit for bit."""
    from paper_1804_06205_gb300 import autotune, serving
    table = autotune.tune(edges=(8.0, 10.0), threads=(64, 128), beads=20_000, steps=3)
    assert table["threads"] in (64, 128) and set(table["tiles"]) == {"8.0", "10.0"}
    reqs = mini_stream()
    srv = serving.Server(max_beads=10 ** 6, max_cells=10 ** 6, max_bonds=10 ** 5,
                         max_systems=16, chunk=5, keep_states=True, table=table)
    seen = {}
    add = srv.batch.add_workload

    def recording_add(w, step=0, tile_cells=0):
        seen[id(w)] = tile_cells
        return add(w, step=step, tile_cells=tile_cells)
    srv.batch.add_workload = recording_add
    done = srv.run(reqs)
    srv.close()
    assert len(done) == len(reqs)
    for d in done:
        r = reqs[d.rid]
        want = serving.tile_for(table, r.workload.L)
        assert want > 0 and seen[id(r.workload)] == want
        g = D.System.from_workload(r.workload, precision=0, threads=table["threads"],
                                   tile_cells=want)
        g.set_state(r.workload.pos, r.workload.vel, 0)
        g.step(r.steps)
        ref = g.get_state()
        g.close()
        assert np.array_equal(d.state[0], ref[0]) and np.array_equal(d.state[1], ref[1])

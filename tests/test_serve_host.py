"""Host logic of the serving loop (no GPU): requests are submitted at their
arrival times, every server with work is stepped, results are fetched once,
and the summary counts requests, right-hand sides and latencies. The
device-side server is replaced by a fake that finishes a request after a
fixed number of steps."""
import numpy as np
import pytest

from paper_2004_07930_gb300 import serve


class FakeServer:
    def __init__(self, solver, slots):
        self.slots = slots
        self.q = []        # [id, ns, steps left]
        self.fetched = []
        self.steps = 0

    def submit(self, rid, src, amp=None):
        ns = len(np.asarray(src).reshape(-1, 3))
        self.q.append([rid, ns, 2 + ns % 3])

    def pending(self):
        return (len(self.q), 0)

    def step(self):
        self.steps += 1
        done = []
        for r in self.q:
            r[2] -= 1
            if r[2] == 0:
                done.append(r[0])
        self.q = [r for r in self.q if r[2] > 0]
        return done

    def fetch(self, rid, ns):
        self.fetched.append(rid)
        return np.zeros((ns, 4)), {"converged": 1, "iterations": 3}

    def close(self):
        pass


@pytest.fixture
def loop(monkeypatch):
    monkeypatch.setattr(serve.hz, "Server", FakeServer)
    return serve.ServingLoop({3.5: object(), 5.0: object()}, 4)


def test_stream_summary(loop):
    src1 = np.zeros((1, 3))
    src3 = np.zeros((3, 3))
    reqs = [(0.0, 10, 3.5, src1), (0.0, 11, 5.0, src3), (0.02, 12, 3.5, src3), (0.04, 13, 5.0, src1)]
    summ = loop.run_stream(reqs)
    assert summ["requests"] == 4 and summ["rhs"] == 8 and summ["converged"]
    assert summ["latency_p99_s"] >= summ["latency_p50_s"] >= 0.0
    assert sorted(loop.results) == [10, 11, 12, 13]
    assert sorted(loop.servers[3.5].fetched) == [10, 12] and sorted(loop.servers[5.0].fetched) == [11, 13]
    assert all(v[0] is None for v in loop.results.values())      # wavefields dropped by default
    assert not loop.busy()


def test_idle_servers_are_not_stepped(loop):
    loop.submit(1, 5.0, np.zeros((2, 3)))
    while loop.busy():
        for f in (3.5, 5.0):
            loop.step(f)
    assert loop.servers[3.5].steps == 0 and loop.servers[5.0].steps == 4
    assert 1 in loop.results and loop.results[1][0].shape == (2, 4)


class FakeSolver:
    def __init__(self, nbytes):
        self.nbytes = nbytes

    def column_bytes(self):
        return self.nbytes


def test_slots_from_device_budget(monkeypatch):
    """Admission by footprint: each frequency gets an equal share of the
    budget, divided by the bytes one column costs on its solver."""
    monkeypatch.setattr(serve.hz, "Server", FakeServer)
    solvers = {3.5: FakeSolver(1e8), 5.0: FakeSolver(3e8), 7.0: FakeSolver(5e10)}
    loop = serve.ServingLoop(solvers, device_budget=6e9)
    assert loop.slots == {3.5: 16, 5.0: 4, 7.0: 1}          # 20, 6, 1 columns fit; powers of two
    assert loop.servers[5.0].slots == 4
    big = serve.slots_for_budget({1.0: FakeSolver(1.0)}, 1e12)
    assert big == {1.0: 64}

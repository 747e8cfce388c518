"""Host-side logic of the serving loop, with a fake backend (no GPU): admission in
arrival order under the HBM budget, memory released on completion, every
request finished once, results keyed by request."""
import numpy as np
import pytest

from paper_2602_04551_b300.serve import Request, Server, poisson_arrivals, latency_summary


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-3)


class FakeBackend:
    """Each solve needs `work` rounds; footprint proportional to n * p."""

    def __init__(self, clock):
        self.clock = clock
        self.live = {}
        self.started = []

    def footprint(self, r):
        n, p = r.dims()
        return n * p

    def start(self, r):
        self.started.append(r.rid)
        h = {"rid": r.rid, "left": r.options["work"], "nodes": 0}
        self.live[r.rid] = h
        return h

    def launch(self, h, rounds):
        h["left"] -= rounds
        h["nodes"] += rounds
        self.clock.t += 0.01

    def poll(self, h):
        return {"done": h["left"] <= 0}

    def finish(self, h):
        del self.live[h["rid"]]
        return {"status": "gap", "ub": 1.0 + h["rid"], "lb": 1.0 + h["rid"], "nodes": h["nodes"],
                "beta": np.zeros(1)}


def _req(rid, n, p, arrival, work):
    return Request(rid=rid, X=np.zeros((n, p)), y=np.zeros(n), lambda0=0.1, lambda2=0.1, M=1.0,
                   arrival=arrival, options={"work": work})


def test_admission_respects_budget_and_order():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(backend=be, budget_bytes=100, rounds_per_step=2, clock=clock, sleep=clock.sleep)
    reqs = [_req(0, 5, 10, 0.0, 10), _req(1, 5, 10, 0.0, 4), _req(2, 5, 10, 0.0, 4),
            _req(3, 2, 10, 0.05, 2)]
    res = srv.run(reqs)
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert all(r.status == "gap" for r in res)
    assert srv.peak_used <= 100
    # request 2 (50 bytes) could only be admitted once 0 or 1 released memory
    adm = {rid: t for t, rid, fp, used in srv.admission_log}
    fin = {r.rid: r.finished for r in res}
    assert adm[2] >= min(fin[0], fin[1])
    # first-come order of admission
    assert be.started == [0, 1, 2, 3]
    assert not be.live


def test_oversized_request_rejected():
    clock = FakeClock()
    srv = Server(backend=FakeBackend(clock), budget_bytes=10, clock=clock, sleep=clock.sleep)
    with pytest.raises(ValueError):
        srv.run([_req(0, 5, 10, 0.0, 1)])


def test_poisson_arrivals_and_summary():
    t = poisson_arrivals(2000, 20.0, 5000)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 20.0) < 0.005
    clock = FakeClock()
    srv = Server(backend=FakeBackend(clock), budget_bytes=10 ** 6, clock=clock, sleep=clock.sleep)
    res = srv.run([_req(i, 3, 3, float(t[i]), 3) for i in range(20)])
    s = latency_summary(res)
    assert s["solves"] == 20 and s["p99_s"] >= s["p50_s"] > 0


def test_latency_summary_splits_queueing_and_service():
    from paper_2602_04551_b300.serve import Result
    res = [Result(rid=i, status="gap" if i % 2 == 0 else "time_limit", ub=1.0, lb=0.9, nodes=10,
                  beta=np.zeros(1), arrival=float(i), admitted=float(i) + 0.5 * i,
                  finished=float(i) + 0.5 * i + 2.0) for i in range(5)]
    s = latency_summary(res)
    assert s["queue_p50_s"] == pytest.approx(1.0)          # 0, .5, 1, 1.5, 2
    assert s["service_p50_s"] == pytest.approx(2.0) and s["service_p99_s"] == pytest.approx(2.0)
    assert s["p50_s"] == pytest.approx(3.0)
    assert s["certified"] == 3 and s["solves"] == 5
    assert s["makespan_s"] == pytest.approx(4 + 2.0 + 2.0)

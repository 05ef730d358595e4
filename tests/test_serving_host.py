"""Host logic of the continuous-batching server (paper_1803_03498_gb300.serving) on CPU: the library
and CUDA streams/events are replaced by fakes that record what the server asks for, so the scheduler
itself is checked -- admission first-fit in arrival order under the memory budget, rejection of
requests that can never fit, one graph launch per quantum plus a plain tail, release of memory and
streams on completion, and results handed back per request."""
import types

import numpy as np
import pytest

from paper_1803_03498_gb300 import serving
from paper_1803_03498_gb300 import workloads as wl


class FakeState:
    def __init__(self):
        self.used = 0
        self.peak = 0
        self.created = []
        self.graph_launches = {}
        self.tails = {}
        self.ticks = []
        self.grouped = {}
        self.schedules = {}


def fake_modules(state, sizes):
    heom = types.SimpleNamespace()

    class HeomError(RuntimeError):
        pass

    heom.HeomError = HeomError
    heom.load = lambda: None
    heom.Hierarchy = lambda M, D: ("hier", M, D)
    heom.run_bytes = lambda system, hier, precision, mr: sizes[system.name]

    class Run:
        def __init__(self, system, re, im, precision, w, max_records, hier, stream):
            self.name = system.name
            self.nbytes = sizes[system.name]
            state.used += self.nbytes
            state.peak = max(state.peak, state.used)
            state.created.append(self.name)
            state.tails[self.name] = 0

        def propagate(self, dt, steps, stride):
            state.tails[self.name] += steps

        def set_schedule(self, occupancy_pct, chunks_per_warp=1, part=0):
            state.schedules[self.name] = (occupancy_pct, chunks_per_warp, part)

        def observables(self):
            return np.array([[len(self.name)]])

        def sigma0(self):
            return np.eye(2)

        def close(self):
            state.used -= self.nbytes

    class Batch:
        def __init__(self, runs, dt, steps_per_launch, stride):
            self.run = runs[0]
            self.spl = steps_per_launch
            state.graph_launches[self.run.name] = 0

        def launch(self, n):
            state.graph_launches[self.run.name] += n * self.spl

        def close(self):
            pass

    heom.Run = Run
    heom.Batch = Batch
    state.autotune = [3]

    def set_autotune(reps):
        prev = state.autotune[-1]
        state.autotune.append(reps)
        return prev

    heom.set_autotune = set_autotune

    def group_propagate(runs, dt, steps, obs_stride=0, stream=None):
        state.ticks.append({r.name: q for r, q in zip(runs, steps)})
        for r, q in zip(runs, steps):
            state.grouped[r.name] = state.grouped.get(r.name, 0) + q

    heom.group_propagate = group_propagate

    class Stream:
        def __init__(self, priority=0):
            self.priority = priority

    class Event:
        def record(self, st):
            pass

        def query(self):
            return True

    class StreamCtx:
        def __init__(self, st):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *a):
            return False

    cuda = types.SimpleNamespace(Stream=Stream, Event=Event, stream=StreamCtx)
    return heom, cuda


def make_requests(spec):
    reqs = []
    for rid, (name, steps) in enumerate(spec):
        s = wl.System(name, np.diag([0.0, 100.0]), [0, 1], [35.0, 35.0], [50.0, 50.0], [300.0, 300.0], K=0, D=2)
        prop = wl.Propagation(s, np.diag([1.0, 0.0]), np.zeros((2, 2)), 0.5, steps)
        reqs.append(wl.Request(arrival_s=0.0, prop=prop, rid=rid))
    return reqs


@pytest.mark.parametrize("workers,pct", [(0, 50), (2, 50), (2, 800)])
def test_admission_budget_quanta_and_release(monkeypatch, workers, pct):
    import torch

    import paper_1803_03498_gb300 as pkg

    state = FakeState()
    sizes = {"a": 40, "b": 50, "c": 30, "huge": 500, "d": 60}
    heom, cuda = fake_modules(state, sizes)
    monkeypatch.setattr(pkg, "heom", heom, raising=False)
    monkeypatch.setitem(__import__("sys").modules, "paper_1803_03498_gb300.heom", heom)
    monkeypatch.setattr(torch, "cuda", cuda)
    reqs = make_requests([("a", 250), ("b", 100), ("huge", 100), ("c", 40), ("d", 320)])
    stats = serving.Server(budget_bytes=100, quantum=100, max_active=3, workers=workers, group_max_ados=0,
                           large_occupancy_pct=pct).serve(reqs, real_time=False)
    res = {r.rid: r for r in stats.results}
    # the request larger than the whole budget is rejected at arrival, the rest complete
    assert res[2].rejected and "budget" in res[2].reason
    assert all(not res[i].rejected and np.isfinite(res[i].done_s) for i in (0, 1, 3, 4))
    # memory: never above the budget, all released at the end
    assert state.peak <= 100 and state.used == 0
    # first fit in arrival order: a (40) and b (50) fit together; c (30) waits for memory (with set-up
    # threads the two runs may be constructed in either order)
    assert sorted(state.created[:2]) == ["a", "b"]
    # whole quanta run as graph replays, the remainder as plain steps
    assert state.graph_launches == {"a": 200, "b": 100, "d": 300}
    assert state.tails == {"a": 50, "b": 0, "c": 40, "d": 20}
    # every larger request's body launches take the given schedule (50: half the CTA slots of each SM;
    # 800: eight waves of CTAs that retire while the launch runs)
    assert set(state.schedules.values()) == {(pct, 1, 0)} and len(state.schedules) == 4
    assert not any(r.batched for r in stats.results)
    # each result carries its own run's observables
    assert all(res[i].observables[0, 0] == len(sizes_name) for i, sizes_name in ((0, "a"), (1, "b"), (4, "d")))
    s = stats.summary()
    assert s["requests"] == 5 and s["completed"] == 4 and s["rejected"] == 1


def test_server_argument_checks():
    with pytest.raises(ValueError):
        serving.Server(quantum=100, obs_stride=30)
    with pytest.raises(ValueError):
        serving.Server(quantum=100, graph_steps=30)


@pytest.mark.parametrize("workers", [0, 2])
def test_small_requests_advance_in_batched_ticks(monkeypatch, workers):
    """Small requests advance together: each tick advances every admitted small request by up to a
    quantum in one group call; a request finishes after exactly its steps; memory is released."""
    import torch

    import paper_1803_03498_gb300 as pkg

    state = FakeState()
    sizes = {"a": 10, "b": 10, "c": 10, "d": 10}
    heom, cuda = fake_modules(state, sizes)
    monkeypatch.setattr(pkg, "heom", heom, raising=False)
    monkeypatch.setitem(__import__("sys").modules, "paper_1803_03498_gb300.heom", heom)
    monkeypatch.setattr(torch, "cuda", cuda)
    reqs = make_requests([("a", 250), ("b", 100), ("c", 40), ("d", 0)])
    stats = serving.Server(budget_bytes=100, quantum=100, max_active=4, workers=workers).serve(reqs, real_time=False)
    assert all(not r.rejected and np.isfinite(r.done_s) for r in stats.results)
    assert state.grouped == {"a": 250, "b": 100, "c": 40}
    assert state.schedules == {}  # batched requests keep their own schedules
    assert all(r.batched and r.arrival_s <= r.admitted_s <= r.active_s <= r.done_s for r in stats.results)
    assert set(stats.results[0].record()) >= {"rid", "latency_s", "n_states", "batched", "active_s"}
    assert state.graph_launches == {} and all(v == 0 for v in state.tails.values())
    # no tick advances a request by more than a quantum, and the first tick covers everything admitted
    assert all(q <= 100 for t in state.ticks for q in t.values())
    assert max(len(t) for t in state.ticks) >= 2
    assert state.used == 0


def test_cost_bounded_quantum_and_autotune(monkeypatch):
    """A larger request whose quantum would hold more than quantum_cost ADOs x n_states^2 x steps takes
    shorter quanta (here 6 ADOs x 2^2 x 30 steps = 720: 30-step graphs); run creation happens with the
    autotuner off, and the library's setting is restored afterwards."""
    import torch

    import paper_1803_03498_gb300 as pkg

    state = FakeState()
    sizes = {"a": 10, "b": 10}
    heom, cuda = fake_modules(state, sizes)
    monkeypatch.setattr(pkg, "heom", heom, raising=False)
    monkeypatch.setitem(__import__("sys").modules, "paper_1803_03498_gb300.heom", heom)
    monkeypatch.setattr(torch, "cuda", cuda)
    reqs = make_requests([("a", 250), ("b", 20)])
    assert reqs[0].prop.system.n_ado == 6
    srv = serving.Server(budget_bytes=100, quantum=100, max_active=4, workers=0, group_max_ados=0, quantum_cost=720)
    stats = srv.serve(reqs, real_time=False)
    assert all(not r.rejected and np.isfinite(r.done_s) for r in stats.results)
    assert state.graph_launches == {"a": 240} and state.tails == {"a": 10, "b": 20}
    assert state.autotune == [3, 0, 3]

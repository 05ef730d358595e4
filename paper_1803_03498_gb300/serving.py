"""Continuous-batching server for HEOM propagation requests on one GPU (host-side scheduler over the
C ABI; every step of every propagation runs in libheom's kernels).

A request is one propagation (system, rho(0), dt, steps).  The server
  * admits arrived requests first-fit while their device workspace (heom_run_bytes) fits the remaining
    memory budget; a request larger than the whole budget is rejected at once (it can never run);
  * builds each admitted request's run (link records on the host, uploads, the CUDA graph) on a pool
    of `workers` host threads -- the library releases the interpreter lock, so several runs are set
    up at once while the main loop keeps launching;
  * batches the RK4 steps of the small requests (mixed precision, at most `group_max_ados` ADOs and
    at most `group_max_cost` ADOs x n_states^2, so that no costly member stretches every tick): in
    each tick every admitted small request advances by up to `quantum` steps in one
    heom_group_propagate call, where the runs of equal n_states share one work-list launch per stage
    and part -- a few launches per step for all of them instead of eight per request; requests
    admitted during a tick join the next one;
  * gives every larger admitted request its own CUDA stream and advances it by `quantum` RK4 steps at
    a time (replays of a CUDA graph of `graph_steps` steps captured at admission, by default the whole
    quantum: one launch on the host per quantum), beside the ticks;
    so the work of all admitted requests overlaps on the device, and requests that arrive while others
    are running are admitted as soon as memory frees up (no batch boundary: continuous batching);
  * on completion copies the observables back, frees the workspace and records the latency
    (completion - arrival, wall clock).
Results of a request do not depend on what else runs: each run uses its own workspace and the kernels
are deterministic.  The paper runs independent propagations side by side (rotational averages,
polarisation sequences; section "Distributed memory HEOM implementation"); this is that, served.
"""
from __future__ import annotations

import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Result:
    rid: int
    arrival_s: float
    admitted_s: float = float("nan")
    active_s: float = float("nan")  # set-up done: the request's steps start to be enqueued
    done_s: float = float("nan")
    rejected: bool = False
    reason: str = ""
    n_ado: int = 0
    n_states: int = 0
    n_steps: int = 0
    batched: bool = False  # advanced in the batched ticks
    workspace_bytes: int = 0
    setup_run_s: float = 0.0    # set-up thread: run creation (host tables, uploads, autotuning)
    setup_graph_s: float = 0.0  # set-up thread: CUDA graph capture
    observables: np.ndarray | None = None
    sigma0: np.ndarray | None = None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s

    def record(self) -> dict:
        """The scalar fields (one line of a per-request log)."""
        return {"rid": self.rid, "arrival_s": self.arrival_s, "admitted_s": self.admitted_s,
                "active_s": self.active_s, "done_s": self.done_s, "latency_s": self.latency_s,
                "rejected": self.rejected, "n_ado": self.n_ado, "n_states": self.n_states,
                "n_steps": self.n_steps, "batched": self.batched, "workspace_bytes": self.workspace_bytes,
                "setup_run_s": self.setup_run_s, "setup_graph_s": self.setup_graph_s}


@dataclass
class _Active:
    req: object
    run: object
    stream: object
    event: object
    remaining: int
    result: Result
    nbytes: int
    graph: object = None
    small: bool = False  # advanced in the batched ticks (heom_group_propagate)
    quantum: int = 0      # steps per quantum of a larger request
    graph_steps: int = 0  # steps per replay of its graph


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    # host time of the serving loop's parts: name -> [total s, longest single s, count]
    loop: dict = field(default_factory=dict)

    def completed(self):
        return [r for r in self.results if not r.rejected and not np.isnan(r.done_s)]

    def summary(self) -> dict:
        done = self.completed()
        lat = np.array([r.latency_s for r in done]) if done else np.array([np.nan])
        evals = sum(r.n_ado * 4 * r.n_steps for r in done)
        return {
            "requests": len(self.results),
            "completed": len(done),
            "rejected": sum(r.rejected for r in self.results),
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(np.mean(lat)),
            "throughput_req_per_s": len(done) / self.wall_s if self.wall_s > 0 else 0.0,
            "ado_rhs_evals_per_s": evals / self.wall_s if self.wall_s > 0 else 0.0,
            "wall_s": self.wall_s,
        }


class Server:
    def __init__(self, budget_bytes: float = 120e9, precision: str = "fp32_mixed", quantum: int = 100,
                 max_active: int = 64, obs_stride: int = 0, keep_sigma0: bool = False, graph_steps: int | None = None,
                 workers: int = 4, group_max_ados: int = 200000, group_max_cost: float = 4e6,
                 large_occupancy_pct: int = 800, quantum_cost: float = 2e10, autotune: int = 0):
        if obs_stride > 0 and quantum % obs_stride:
            raise ValueError("obs_stride must divide quantum")
        if graph_steps is None:  # one graph per quantum (measured: fewer, longer graphs serve more)
            graph_steps = quantum
        if graph_steps < 1 or quantum % graph_steps or (obs_stride > 0 and graph_steps % obs_stride):
            raise ValueError("graph_steps must divide quantum and be a multiple of obs_stride")
        self.budget = int(budget_bytes)
        self.precision = precision
        self.quantum = int(quantum)
        self.max_active = int(max_active)
        self.obs_stride = int(obs_stride)
        self.keep_sigma0 = keep_sigma0
        self.graph_steps = int(graph_steps)
        self.workers = max(0, int(workers))
        # requests up to this many ADOs (mixed precision) advance in the batched ticks; 0: none
        self.group_max_ados = int(group_max_ados) if precision == "fp32_mixed" else 0
        # and whose ADOs x n_states^2 (the work of one stage) is at most this: a tick lasts as long as its
        # slowest member's steps, so one costly member would hold up every small request of the tick
        self.group_max_cost = float(group_max_cost)
        # the schedule of a larger request's stage launches (heom_set_schedule's occupancy_pct): above 100
        # its grid is several waves of CTAs that retire while the launch runs, so the ticks' launches on
        # the high-priority stream take SM slots within microseconds instead of waiting for the whole
        # launch; below 100 a persistent grid on that share of each SM's CTA slots (measured on the full
        # mix: 50 % slowed the largest request more than it helped the rest)
        self.large_occupancy_pct = int(large_occupancy_pct)
        # a larger request's quantum holds at most this many ADOs x n_states^2 x steps (0: no bound), so
        # that no request's queued launches occupy the GPU for long: work queued on streams that share a
        # hardware queue with it, and host calls that wait for such work, wait behind a whole quantum
        # (measured on the full mix: 100 steps of the 7M-ADO request, about 9 s, stalled the loop)
        self.quantum_cost = float(quantum_cost)
        # timed launches per candidate schedule when a request's run is created (heom_set_autotune);
        # 0: no tuning, cached or default schedules (measured on the full mix: tuning new runs while the
        # GPU is busy held their set-up for seconds, p50 68 s against 16 s); -1: the library's setting
        self.autotune = int(autotune)
        self._hier_cache = {}

    def _hier(self, heom, M, D):
        key = (M, D)
        if key not in self._hier_cache:
            self._hier_cache[key] = heom.Hierarchy(M, D)
        return self._hier_cache[key]

    def _quantum(self, r) -> tuple[int, int]:
        """Steps per quantum of a larger request and steps per replay of its graph."""
        s = r.prop.system
        q = self.quantum
        if self.quantum_cost > 0:
            q = min(q, int(self.quantum_cost // max(1, s.n_ado * s.N * s.N)))
        unit = self.graph_steps if self.graph_steps < self.quantum else max(self.obs_stride, 1)
        q = max(unit, q - q % unit)
        return q, (self.graph_steps if self.graph_steps < self.quantum else q)

    def _small(self, r) -> bool:
        s = r.prop.system
        return s.n_ado <= self.group_max_ados and s.n_ado * s.N * s.N <= self.group_max_cost

    def _build(self, heom, r, hier, mr, st, dev):
        """Set up one admitted request on its stream: the run (host link records, uploads) and, for a
        larger request with at least one whole quantum, the CUDA graph of graph_steps steps."""
        import torch

        if dev is not None:
            torch.cuda.set_device(dev)
        with torch.cuda.stream(st):
            t0 = time.perf_counter()
            run = heom.Run(r.prop.system, r.prop.rho0_re, r.prop.rho0_im, precision=self.precision,
                           w=r.prop.w, max_records=mr, hier=hier, stream=st)
            if not self._small(r) and self.large_occupancy_pct != 100:
                run.set_schedule(self.large_occupancy_pct, 1, part=0)
            t1 = time.perf_counter()
            graph = None
            q, gsteps = self._quantum(r)
            if r.prop.n_steps >= q and not self._small(r):
                graph = heom.Batch([run], r.prop.dt_fs, gsteps, self.obs_stride)
        return run, graph, t1 - t0, time.perf_counter() - t1

    def serve(self, requests, real_time: bool = True) -> ServeStats:
        """Serve `requests` (workloads.Request: arrival_s, prop, rid) and return per-request results.
        With real_time the arrivals follow the wall clock; otherwise all requests arrive at t = 0."""
        import torch

        from . import heom

        heom.load()
        prev_tune = heom.set_autotune(self.autotune) if self.autotune >= 0 else None
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        arrivals = deque(reqs)
        pending: deque = deque()
        active: list[_Active] = []
        results: dict[int, Result] = {}
        used = 0
        streams = [torch.cuda.Stream() for _ in range(self.max_active)]
        free_streams = list(range(self.max_active))
        dev = torch.cuda.current_device() if hasattr(torch.cuda, "current_device") else None
        pool = ThreadPoolExecutor(self.workers) if self.workers > 0 else None
        building: list = []  # (future, request, stream index, result)
        t0 = time.perf_counter()

        def now():
            return time.perf_counter() - t0

        loop = {}

        class timed:  # host time of one part of the loop
            def __init__(self, name):
                self.name = name

            def __enter__(self):
                self.t = time.perf_counter()

            def __exit__(self, *exc):
                d = time.perf_counter() - self.t
                e = loop.setdefault(self.name, [0.0, 0.0, 0])
                e[0] += d
                e[1] = max(e[1], d)
                e[2] += 1

        def activate(r, si, res, run, graph, t_run=0.0, t_graph=0.0):
            res.setup_run_s, res.setup_graph_s = t_run, t_graph
            res.active_s = now()
            res.batched = self._small(r)
            ev = torch.cuda.Event()
            ev.record(streams[si])
            q, gsteps = self._quantum(r)
            active.append(_Active(r, run, si, ev, r.prop.n_steps, res, res.workspace_bytes, graph, self._small(r),
                                  q, gsteps))

        def complete(a):
            nonlocal used
            res = a.result
            res.observables = a.run.observables()
            if self.keep_sigma0:
                res.sigma0 = a.run.sigma0()
            res.done_s = now()
            if a.graph is not None:
                a.graph.close()
            a.run.close()
            a.run = None
            used -= a.nbytes
            free_streams.append(a.stream)
            active.remove(a)

        # the ticks' stream has the higher priority: when SM slots free up, the block scheduler dispatches
        # the small requests' launches before those of larger requests queued on the other streams
        group_stream = torch.cuda.Stream(priority=-1) if self.group_max_ados > 0 else None
        tick = None  # event of the batched tick in flight

        while arrivals or pending or active or building or tick is not None:
            t = now()
            while arrivals and (not real_time or arrivals[0].arrival_s <= t):
                r = arrivals.popleft()
                res = Result(r.rid, r.arrival_s if real_time else 0.0, n_ado=r.prop.system.n_ado,
                             n_states=r.prop.system.N, n_steps=r.prop.n_steps)
                results[r.rid] = res
                s = r.prop.system
                # a large hierarchy whose three state copies alone exceed the budget is rejected
                # without building its tables (seconds of host time and gigabytes of host memory)
                elem = 16 if self.precision == "fp64" else 8
                if s.n_ado > 2_000_000 and 3 * s.n_ado * s.N * s.N * elem > self.budget:
                    res.rejected, res.reason = True, "workspace above the device-memory budget"
                    continue
                mr = (r.prop.n_steps // self.obs_stride + 2) if self.obs_stride > 0 else 2
                try:
                    with timed("arrival: hierarchy and workspace size"):
                        hier = self._hier(heom, s.n_modes, s.D)
                        res.workspace_bytes = heom.run_bytes(s, hier, self.precision, mr)
                except heom.HeomError as e:
                    res.rejected, res.reason = True, str(e)
                    continue
                if res.workspace_bytes > self.budget:
                    res.rejected, res.reason = True, "workspace above the device-memory budget"
                    continue
                pending.append((r, hier, mr))
            # admission: first fit in arrival order; the set-up runs on the worker threads
            i = 0
            while i < len(pending) and free_streams:
                r, hier, mr = pending[i]
                res = results[r.rid]
                if used + res.workspace_bytes <= self.budget:
                    del pending[i]
                    si = free_streams.pop()
                    used += res.workspace_bytes
                    res.admitted_s = now()
                    with timed("admission: set-up (inline) or its submission"):
                        if pool is None:
                            activate(r, si, res, *self._build(heom, r, hier, mr, streams[si], None))
                        else:
                            building.append((pool.submit(self._build, heom, r, hier, mr, streams[si], dev), r, si,
                                             res))
                else:
                    i += 1
            # set-ups that finished become active
            for b in [b for b in building if b[0].done()]:
                building.remove(b)
                fut, r, si, res = b
                with timed("activation"):
                    activate(r, si, res, *fut.result())
            # batched tick of the small requests: when the previous one is done, finished requests
            # complete and every other small request advances by up to a quantum in one call
            progressed = False
            if group_stream is not None and (tick is None or tick.query()):
                tick = None
                small = [a for a in active if a.small]
                for a in [a for a in small if a.remaining == 0]:
                    with timed("completion (batched)"):
                        complete(a)
                    progressed = True
                by_dt = {}
                for a in small:
                    if a.remaining > 0:
                        by_dt.setdefault(a.req.prop.dt_fs, []).append(a)
                for dt, members in by_dt.items():
                    steps = [min(self.quantum, a.remaining) for a in members]
                    with timed("tick: heom_group_propagate"):
                        heom.group_propagate([a.run for a in members], dt, steps, self.obs_stride,
                                             stream=group_stream)
                    for a, q in zip(members, steps):
                        a.remaining -= q
                if by_dt:
                    tick = torch.cuda.Event()
                    tick.record(group_stream)
                    progressed = True
            # progress of the larger requests: finished quanta get the next quantum or complete
            for a in list(active):
                if a.small or not a.event.query():
                    continue
                progressed = True
                if a.remaining > 0:
                    st = streams[a.stream]
                    with timed("quantum launch (larger requests)"):
                        if a.graph is not None and a.remaining >= a.quantum:
                            a.graph.launch(a.quantum // a.graph_steps)
                            q = a.quantum
                        else:
                            q = a.remaining
                            a.run.propagate(a.req.prop.dt_fs, q, self.obs_stride)
                        a.remaining -= q
                        a.event = torch.cuda.Event()
                        a.event.record(st)
                else:
                    with timed("completion (larger requests)"):
                        complete(a)
            if not progressed:
                if arrivals and real_time and not active and not pending and not building:
                    time.sleep(max(0.0, min(arrivals[0].arrival_s - now(), 0.01)))
                else:
                    time.sleep(0.0002)
        stats = ServeStats(results=[results[k] for k in sorted(results)], wall_s=now(), loop=loop)
        if pool is not None:
            pool.shutdown(wait=True)
        if prev_tune is not None:
            heom.set_autotune(prev_tune)
        return stats


def main(argv=None):
    """Rate sweep of the serving loop on seeded Poisson streams (one JSON line per offered rate)."""
    import argparse
    import json
    import os

    # many request streams: more hardware work queues than the default 8 (read at CUDA start-up)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

    from . import heom
    from . import workloads as wl

    ap = argparse.ArgumentParser(prog="python -m paper_1803_03498_gb300.serving")
    ap.add_argument("--rates", type=float, nargs="+", default=[5, 10, 20, 50, 100, 200])
    ap.add_argument("--requests", type=int, default=500)
    ap.add_argument("--max-ado-steps", type=float, default=2e7,
                    help="redraw requests above this ADOs x steps (a bounded sample of the mix); 0: the full mix")
    ap.add_argument("--budget", type=float, default=120e9)
    ap.add_argument("--precision", default="fp32_mixed")
    ap.add_argument("--workers", type=int, default=4, help="host threads that set up admitted requests")
    ap.add_argument("--quantum", type=int, default=100)
    ap.add_argument("--max-active", type=int, default=256, help="requests admitted at once (streams)")
    ap.add_argument("--group-max-ados", type=int, default=200000, help="largest request batched in ticks")
    ap.add_argument("--group-max-cost", type=float, default=4e6,
                    help="largest ADOs x n_states^2 of a request batched in ticks")
    ap.add_argument("--autotune", type=int, default=0,
                    help="timed launches per schedule candidate when a run is created (0: no tuning, the "
                         "cached or default schedules; -1: the library's setting)")
    ap.add_argument("--quantum-cost", type=float, default=2e10,
                    help="bound on ADOs x n_states^2 x steps of a larger request's quantum (0: none)")
    ap.add_argument("--dump", default="", help="write every request's timeline to <dump>_<rate>.jsonl")
    ap.add_argument("--large-occupancy", type=int, default=800,
                    help="occupancy_pct of a larger request's stage launches (above 100: waves of CTAs)")
    args = ap.parse_args(argv)
    heom.load()
    cap = args.max_ado_steps if args.max_ado_steps > 0 else None
    for rate in args.rates:
        reqs = wl.serving_stream(rate, args.requests, max_ado_steps=cap)
        st = Server(budget_bytes=args.budget, precision=args.precision, quantum=args.quantum,
                    workers=args.workers, max_active=args.max_active, group_max_ados=args.group_max_ados,
                    group_max_cost=args.group_max_cost,
                    large_occupancy_pct=args.large_occupancy, quantum_cost=args.quantum_cost,
                    autotune=args.autotune).serve(reqs, real_time=True)
        s = st.summary()
        if args.dump:
            with open(f"{args.dump}_{rate:g}.jsonl", "w") as fh:
                for res in st.results:
                    fh.write(json.dumps(res.record()) + "\n")
        s.update({"offered_rate_req_per_s": rate, "max_ado_steps": cap, "precision": args.precision,
                  "workers": args.workers, "max_active": args.max_active, "quantum": args.quantum,
                  "group_max_ados": args.group_max_ados, "group_max_cost": args.group_max_cost,
                  "large_occupancy_pct": args.large_occupancy, "autotune": args.autotune,
                  "quantum_cost": args.quantum_cost,
                  "loop_host_s": {k: {"total": round(v[0], 3), "longest": round(v[1], 3), "count": v[2]}
                                  for k, v in st.loop.items()},
                  "rejected_fraction": s["rejected"] / max(s["requests"], 1)})
        print(json.dumps(s), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())

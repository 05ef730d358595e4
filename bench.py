"""Benchmark: HEOM RK4 propagation throughput in ADO-RHS evaluations per second on GB300.

One step = one classic RK4 step over the whole hierarchy (four right-hand-side evaluations of every
ADO, fused stage kernels) plus one FP64 observable record of sigma_0.  The workload is the
LHCII-like system (14 sites, energies U[14800, 15300] cm^-1, couplings N(0, 30) cm^-1, Drude-Lorentz
baths lambda = 35 cm^-1, 1/nu = 50 fs, 300 K, K = 1 Matsubara term -> 28 modes, depth 6 ->
1,344,904 ADOs of 14 x 14, dt = 1 fs), seeded and synthetic.  The headline value is the mixed
precision path (FP32 bulk ADOs, FP64 root and reductions); the FP64 path is reported beside it.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun): every rank runs an independent replica of the workload (the method does not
shard on one node without a halo exchange; no collective touches the data path); value = the sum
over ranks, time = the max over ranks.  ``--impl reference`` times the CPU FP64 oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving leg keeps up to 64 request streams (plus each mixed run's head stream) busy: more
# hardware work queues than the default 8 let their kernels run side by side (read at CUDA start-up)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "ADO-RHS evals/s (FP64 vs mixed, pop err <=1e-6)"
UNIT = "ADO-RHS evals/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# GB300 issues 2 FP64 FMAs (4 flops) per clock per SM: the nominal 1.25 TFLOP/s at the 2.07 GHz
# maximum SM clock over 152 SMs; a dependent-FMA probe on this GPU gave 1.199 TFLOP/s at ~1.97 GHz.
FP64_FLOPS_PER_CLK_SM = 4.0
FP64_PEAK_TFLOPS = 1.2  # fallback when no SM clock was sampled


def fp64_peak_tflops(sm_mhz, n_sm=152):
    """FP64 ALU peak at the SM clock the leg ran at (nvidia-smi median under load)."""
    if not sm_mhz:
        return FP64_PEAK_TFLOPS, "fallback 1.2 TFLOP/s (no clock sample)"
    return n_sm * FP64_FLOPS_PER_CLK_SM * sm_mhz * 1e6 / 1e12, f"{n_sm} SMs x 4 flop/clk x {sm_mhz:.0f} MHz"


def _traffic():
    """DRAM bytes per launch of the dominant kernels from the committed ncu summary, or None when
    the kernel sources changed since those counters were taken."""
    import hashlib

    src = os.path.join(ROOT, "paper_1803_03498_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("stage_kernel.cuh", "stage_col.cuh", "propagate.cu"):  # the kernels and the host code that launches them
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    vals = {}
    try:
        with open(os.path.join(ROOT, "profiles", "stage_kernel_lhcii_dram.md")) as fh:
            for line in fh:
                p = line.split()
                if len(p) == 2 and (p[0].startswith("traffic_") or p[0] == "source_sha256_16"):
                    vals[p[0]] = p[1]
    except OSError:
        return None, None
    if vals.get("source_sha256_16") != h.hexdigest()[:16]:
        return None, None
    return float(vals["traffic_fp32_mixed_body_bytes_per_launch"]), float(vals["traffic_fp64_bytes_per_launch"])


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x, ws):
    """The largest x over the ranks (each rank times its own replica; the job takes the slowest)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(ws, n_ado, steps, ms_max):
    """Whole-job ADO-RHS evaluations per second: every rank runs one replica of n_ado ADOs for `steps`
    RK4 steps (4 RHS evaluations each); the job's time is the slowest rank's."""
    return ws * n_ado * 4 * steps / (ms_max / 1000.0)


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def time_gpu(prop, precision, steps, warmup, ws, clocks=None, schedule=None):
    """Device-timed propagation of `steps` RK4 steps (inputs resident in HBM).  schedule: (occupancy %,
    chunks per warp) forced on the body launches instead of the tuner's choice."""
    import torch

    from paper_1803_03498_gb300 import heom

    run = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision=precision, w=prop.w,
                   max_records=warmup + steps + 4)
    if schedule is not None:
        run.set_schedule(*schedule, part=0)
    run.propagate(prop.dt_fs, warmup, 1)
    torch.cuda.synchronize()
    run.set_timing(True)
    l0 = run.launches()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0.record(st)
    run.propagate(prop.dt_fs, steps, 1)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    _barrier(ws)
    ms = e0.elapsed_time(e1)
    launches = run.launches() - l0
    kt = run.kernel_time()
    obs = run.observables()
    # the launch schedules the autotuner picked at run creation (occupancy %, chunks per warp)
    kt["schedule"] = {"body": list(run.schedule(0))}
    if precision != "fp64":
        kt["schedule"]["head"] = list(run.schedule(1))
    run.close()
    return ms, launches, kt, obs, clk


def time_states(steps, warmup, ws, states=(14, 17, 19, 20, 22, 24), max_ados=2.5e6):
    """Mixed-precision rate across n_states: population runs from the first site of seeded random
    systems (one bath per site, K = 0, the deepest hierarchy with at most max_ados ADOs: every state
    copy larger than L2).  Per size: ADO-RHS evals/s, the body launch time and its bandwidth on the
    per-unit count (4 tile transfers of N^2 FP32 complex elements + 2 M link-table entries per
    evaluation)."""
    from math import comb

    from paper_1803_03498_gb300 import workloads as wl

    rows = []
    for N in states:
        D = 1
        while comb(N + D + 1, D + 1) <= max_ados:
            D += 1
        sysm = wl._random_system(np.random.default_rng(1000 + N), N, D, 0, f"random N={N} K=0 D={D}")
        re, im = wl._pure(N, 0)
        prop = wl.Propagation(sysm, re, im, 0.5, steps, tag="states")
        ms, _, kt, _, _ = time_gpu(prop, "fp32_mixed", steps, warmup, ws)
        body_ms = kt["ms"] / max(kt["launches"], 1)
        nb = sysm.n_ado - (1 + sysm.n_modes)
        unit = nb * (4.0 * N * N * 8 + 2 * sysm.n_modes * 4)
        rows.append({"n_states": N, "depth": D, "n_ado": sysm.n_ado, "ms_per_step": ms / steps,
                     "evals_per_s": sysm.n_ado * 4 * steps / (ms / 1000.0), "body_launch_ms": body_ms,
                     "per_unit_GBs": unit / (body_ms / 1000.0) / 1e9})
    return rows


def fp64_and_gate(prop, gate_steps, warmup, ws, clocks):
    """The FP64 path over the configuration's full length, and the mixed-precision error gate.

    One FP64 run and one mixed run, both from rho(0), gate_steps RK4 steps with a population record
    after every step.  The FP64 run's steps after the first `warmup` are device-timed (its ADO-RHS
    evals/s and the per-launch time of its stage kernel); the gate is the largest population
    difference between the two runs over all gate_steps + 1 records.  The FP64 GPU path itself is
    held to the oracle by the parity tests (1e-12)."""
    import torch

    from paper_1803_03498_gb300 import heom

    n_ado = prop.system.n_ado
    run = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp64", w=prop.w, max_records=gate_steps + 2)
    run.propagate(prop.dt_fs, warmup, 1)
    torch.cuda.synchronize()
    run.set_timing(True)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0.record(st)
    run.propagate(prop.dt_fs, gate_steps - warmup, 1)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    _barrier(ws)
    ms = _max_over_ranks(e0.elapsed_time(e1), ws)
    timed = gate_steps - warmup
    kt = run.kernel_time()
    obs64 = run.observables()
    sched = list(run.schedule(0))
    run.close()
    mixed = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp32_mixed", w=prop.w,
                     max_records=gate_steps + 2)
    mixed.propagate(prop.dt_fs, gate_steps, 1)
    obs32 = mixed.observables()
    mixed.close()
    N = prop.system.N
    assert obs64.shape == obs32.shape == (gate_steps + 1, N + 5)
    pop_err = float(np.max(np.abs(obs32[:, :N] - obs64[:, :N])))
    avg = kt["ms"] / max(kt["launches"], 1)
    ach = kt["alg_flops"] / (kt["ms"] / 1000.0) / 1e12 if kt["ms"] > 0 else 0.0
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak, basis = fp64_peak_tflops(clk["sm_mhz"] if clk else None, n_sm)
    leg = {"value": _job_value(ws, n_ado, timed, ms), "unit": UNIT, "ms_per_step": ms / timed, "steps": timed,
           "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                        "peak_basis": basis,
                        "flops": "4 N^3 per ADO (Hermitian form: H s only, s H = (H s)^dagger) + 8 N^2 "
                                 "+ 8 (N-1) per up link + 8 (2N-1) per down link",
                        "kernel": "stage_col_kernel<14> (column form, FP64)", "avg_launch_ms": avg, "schedule": sched},
           "clocks": clk}
    gate = {"steps": gate_steps, "records": gate_steps + 1, "max_pop_err": pop_err, "bar": 1e-6,
            "pass": pop_err <= 1e-6,
            "what": "max |population(mixed) - population(FP64)| over every RK4 step of the full-length run "
                    "from rho(0), dt = 1 fs"}
    return leg, gate


def time_e2e(prop, precision, steps):
    """End to end through the public API with host buffers: the hierarchy build (host), run creation
    (tables and sigma_0 go host -> device), `steps` RK4 steps, observables device -> host."""
    import torch

    from paper_1803_03498_gb300 import heom

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hier = heom.Hierarchy(prop.system.n_modes, prop.system.D)
    run = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision=precision, w=prop.w,
                   max_records=steps + 2, hier=hier)
    run.propagate(prop.dt_fs, steps, 1)
    obs = run.observables()
    t1 = time.perf_counter()
    n, M = run.N, prop.system.n_modes
    u_pitch = (run.n_ado + 63) // 64 * 64
    h2d = u_pitch * (M * 9 + 8) + 2 * n * n * 8 + (prop.system.D + 1) * M * 16 + M * 24 + (n + 1) * 4 + n * 8
    d2h = obs.size * 8 + 8
    run.close()
    return (t1 - t0), h2d / steps, d2h / steps


def time_batch(steps=20, per_launch=10):
    """The ragged batch (64 systems x 3 dipole orientations = 192 runs, N+1 in 3..17, D in 3..5,
    K in 0..1, mixed precision): all runs in one CUDA graph per `per_launch` steps, against the same
    runs propagated one after another with heom_propagate.  Dipole runs take the column-0 layout.
    Returns a dict."""
    import torch

    from paper_1803_03498_gb300 import heom
    from paper_1803_03498_gb300 import workloads as wl

    props = wl.ragged_batch()
    dt = props[0].dt_fs
    n_ado = sum(p.system.n_ado for p in props)
    runs = [heom.Run(p.system, p.rho0_re, p.rho0_im, precision="fp32_mixed", w=p.w,
                     max_records=3 * steps // per_launch + 4) for p in props]
    t0 = time.perf_counter()
    b = heom.Batch(runs, dt, per_launch, per_launch)
    t_capture = time.perf_counter() - t0
    b.launch(1)  # warm-up
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batch_timed")  # lets a profiler select the timed replays
    e0.record(st)
    b.launch(steps // per_launch)
    e1.record(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    layout = ("every run in the column-0 (coherence-block) layout" if all(r.layout() == 1 for r in runs)
              else "mixed layouts")
    sched = {}
    for body, head in b.schedules():  # per group of batched launches: what the autotuner picked
        key = f"body {body[0]}% x{body[1]} chunks, head {head[0]}% x{head[1]} chunks"
        sched[key] = sched.get(key, 0) + 1
    # sequential: one run after the other, each run's steps enqueued as separate launches
    for r in runs:
        r.propagate(dt, 1, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in runs:
        r.propagate(dt, steps, per_launch)
        torch.cuda.synchronize()
    ms_seq = (time.perf_counter() - t0) * 1000
    b.close()
    for r in runs:
        r.close()
    evals = n_ado * 4 * (steps // per_launch) * per_launch
    return {"workload": "ragged batch: 64 systems x 3 dipole orientations = 192 runs, 2,597,400 ADOs, "
                        "N+1 in 3..17, D in 3..5, K in 0..1, fp32_mixed, dt=0.5 fs",
            "value": evals / (ms_batch / 1000), "unit": UNIT, "steps": steps, "ms_per_step": ms_batch / steps,
            "sequential_value": evals / (ms_seq / 1000), "speedup_vs_sequential": ms_seq / ms_batch,
            "layout": layout,
            "group_schedules": sched,
            "graph": f"one CUDA graph per {per_launch} steps of all runs: runs up to 50,000 ADOs grouped by N into "
                     f"one launch per stage, larger runs one launch each (autotune + capture + instantiate "
                     f"{t_capture:.2f} s)"}


def time_field(steps=40, warmup=3, sm_mhz=None):
    """Pump-pulse propagation of the FMO-like two-exciton space (7 sites: 29 states, K = 1, D = 4:
    3060 ADOs of 29 x 29) on the general stage kernel: classic four-copy RK4 with H(t) at each stage
    time.  Device-timed steps; per-launch kernel time of the body launches; algorithmic flops per
    ADO-RHS evaluation 16 N^3 (complex H(t)) + 8 N^2 + 8 per link record of each coupled state."""
    import torch

    from paper_1803_03498_gb300 import heom
    from paper_1803_03498_gb300 import workloads as wl

    prop, pulse = wl.fmo_two_exciton(n_sites=7, D=4)
    s = prop.system
    N, n_ado = s.N, s.n_ado
    hier = heom.Hierarchy(s.n_modes, s.D)
    _, plus, minus = hier.export()
    per_state = s.bath_mask.sum(axis=1)  # states per bath's V
    K1 = s.K + 1
    recs = sum(int(np.sum(plus[:, l] >= 0) + np.sum(minus[:, l] >= 0)) * int(per_state[l // K1]) for l in range(s.n_modes))
    flops_eval = n_ado * (16.0 * N ** 3 + 8.0 * N ** 2) + recs * 8.0 * N * 2
    out = {"workload": "fmo-like 7-site two-exciton space (29 states) K=1 D=4 (3060 ADOs), Gaussian pump "
                       "(60 cm^-1 peak coupling, sigma 15 fs), dt=0.5 fs, classic RK4 with H(t)",
           "unit": UNIT, "steps": steps}
    for precision in ("fp64", "fp32_mixed"):
        r = heom.Run(s, prop.rho0_re, prop.rho0_im, precision=precision, max_records=4, time_dependent=True)
        r.set_field(pulse)
        r.propagate(prop.dt_fs, warmup, 0)
        torch.cuda.synchronize()
        r.set_timing(True)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r.propagate(prop.dt_fs, steps, 0)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kt = r.kernel_time()
        r.close()
        leg = {"value": n_ado * 4 * steps / (ms / 1000.0), "ms_per_step": ms / steps,
               "avg_launch_ms": kt["ms"] / max(kt["launches"], 1)}
        if precision == "fp64":
            # body launches cover every ADO: one RHS evaluation each
            ach = flops_eval / (leg["avg_launch_ms"] / 1000.0) / 1e12
            n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            peak, basis = fp64_peak_tflops(sm_mhz, n_sm)
            leg["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                               "frac": ach / peak, "peak_basis": basis, "kernel": "gen_stage_kernel<double,double>"}
        out[precision] = leg
    return out


def time_serving(rates=(5.0, 20.0, 50.0), n_requests=100, max_ado_steps=2e7, budget=120e9, max_active=256):
    """The serving loop: Poisson arrivals of population-run requests (N in 2..24, D in 2..6, K in 0..1,
    200..5000 steps, mixed precision, 120 GB device-memory budget).  The full mix is heavy-tailed
    (mean ~2.5e9 ADO-RHS evaluations per request); the timed legs use a bounded sample of it (draws
    above max_ado_steps ADOs x steps are redrawn) so that an offered rate can be sustained at all."""
    from paper_1803_03498_gb300 import heom
    from paper_1803_03498_gb300 import workloads as wl
    from paper_1803_03498_gb300.serving import Server

    full = wl.serving_stream(rates[0], 500)
    hcache, rej = {}, 0
    for r in full:
        s = r.prop.system
        key = (s.n_modes, s.D)
        if key not in hcache:
            hcache[key] = heom.Hierarchy(*key)
        if heom.run_bytes(s, hcache[key], "fp32_mixed", 2) > budget:
            rej += 1
    del hcache
    legs = []
    for rate in rates:
        reqs = wl.serving_stream(rate, n_requests, max_ado_steps=max_ado_steps)
        st = Server(budget_bytes=budget, quantum=100, max_active=max_active).serve(reqs, real_time=True)
        s = st.summary()
        s["offered_rate_req_per_s"] = rate
        legs.append(s)
    return {"workload": f"Poisson arrivals, N 2..24, D 2..6, K 0..1, 200..5000 steps, fp32_mixed; timed legs: "
                        f"{n_requests} requests redrawn to <= {max_ado_steps:.0e} ADOs x steps (the narrowed mix; "
                        f"the full mix is measured by the serving module's rate sweep with --max-ado-steps 0)",
            "server": f"up to {max_active} requests admitted; small requests (<= 200,000 ADOs and <= 4e6 ADOs x "
                      f"n_states^2) advance in batched ticks of one heom_group_propagate call (work-list launches "
                      f"per size class) on a high-priority stream, larger ones on their own streams with CUDA "
                      f"graphs and grids of 8 CTA waves; quantum 100 steps (at most 2e10 ADOs x n_states^2 x "
                      f"steps for a larger request); no autotuning at set-up",
            "budget_bytes": budget, "full_mix_rejected_fraction": rej / len(full), "legs": legs}


def cpu_baseline(prop, seconds=12.0, seed=1):
    """The CPU oracle (single thread, as it stands) on a bounded sample of the same workload: the
    right-hand side of randomly chosen ADOs of the full hierarchy, on a random dense state."""
    from oracle.oracle import Bath, OracleModel

    s = prop.system
    m = OracleModel(s.H, [Bath(st, l, t, T) for st, l, t, T in zip(s.bath_state, s.lambda_cm, s.tau_fs, s.T_K)],
                    K=s.K, D=s.D)
    rng = np.random.default_rng(seed)
    re = rng.random((m.n_ado, m.N, m.N))
    im = rng.random((m.n_ado, m.N, m.N))
    done, t_used, chunk = 0, 0.0, 2000
    while t_used < seconds:
        us = np.sort(rng.integers(0, m.n_ado, chunk)).astype(np.int64)
        t0 = time.perf_counter()
        m.rhs_list(us, re, im)
        t_used += time.perf_counter() - t0
        done += chunk
    return {"value": done / t_used, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"right-hand side of {done} random ADOs of the {m.n_ado}-ADO hierarchy (random dense state), "
                      f"{t_used:.1f} s on one host core"}


def reference_arm(args, ws, rank):
    """--impl reference: the CPU FP64 oracle on the host cores, same metric and workload."""
    from paper_1803_03498_gb300 import workloads as wl

    if rank != 0:
        return 0
    from oracle.oracle import Bath, OracleModel, build_oracle

    build_oracle()
    prop = wl.lhcii_like()
    s = prop.system
    m = OracleModel(s.H, [Bath(st, l, t, T) for st, l, t, T in zip(s.bath_state, s.lambda_cm, s.tau_fs, s.T_K)],
                    K=s.K, D=s.D)
    rng = np.random.default_rng(7)
    re = rng.random((m.n_ado, m.N, m.N))
    im = rng.random((m.n_ado, m.N, m.N))
    per_step = 4000  # ADO right-hand sides per timed step (a bounded sample of one RK4 step)
    times = []
    for i in range(args.warmup + args.steps):
        us = np.sort(rng.integers(0, m.n_ado, per_step)).astype(np.int64)
        t0 = time.perf_counter()
        m.rhs_list(us, re, im)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step * len(times) / tot
    sample = (f"each step: right-hand side of {per_step} random ADOs of the {m.n_ado}-ADO LHCII-like hierarchy "
              f"(random dense state), single-threaded C oracle")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "lhcii-like N=14 K=1 D=6 (1,344,904 ADOs), dt=1 fs", "precision": "fp64",
                       "l2": "state 4.2 GB per copy > L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the ragged-batch leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-field", action="store_true", help="skip the two-exciton laser-field leg")
    ap.add_argument("--gate-steps", type=int, default=1000,
                    help="length of the FP64 run and of the mixed-vs-FP64 population gate (the configuration's "
                         "1000 steps of 1 fs); its steps after the warm-up time the FP64 path (0: skip both)")
    ap.add_argument("--depth", type=int, default=0, help="override the hierarchy depth (profiling cases)")
    ap.add_argument("--tc-steps", type=int, default=0, help="timed steps of the split-TF32 variant (0: steps/10)")
    ap.add_argument("--only", default="", choices=["", "mixed", "fp64", "split_tf32", "dipole", "field", "states",
                                                   "batch"],
                    help="one case only, no end-to-end or CPU legs, no autotuning (profiling cases): a precision "
                         "of the LHCII-like population run, its linear-absorption run (dipole: 15 states, column-0 "
                         "layout, mixed), the pumped two-exciton leg (field), or the mixed-precision rate across "
                         "n_states (states), or the ragged batch (batch: autotuned as in the full run)")
    ap.add_argument("--schedule", default="", help="profiling cases: occupancy%%,chunks_per_warp of the body launches")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)
    args.warmup = max(args.warmup, 3)

    import torch

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0 or ws == 1:
        import __graft_entry__
        __graft_entry__.build()
    _barrier(ws)
    from paper_1803_03498_gb300 import heom
    from paper_1803_03498_gb300 import workloads as wl

    heom.load()
    prop = wl.lhcii_like()
    if args.depth:
        prop.system.D = args.depth
        prop.system.name = prop.system.name.replace("D=6", f"D={args.depth}")
    n_ado = prop.system.n_ado
    if args.only == "batch":
        if rank == 0:
            print(json.dumps({"profile_case": "ragged_batch", **time_batch(steps=args.steps)}), flush=True)
        return 0
    if args.only:
        heom.set_autotune(0)  # the same launches every time: no tuning probes before the captured ones
        if args.only == "field":
            if rank == 0:
                print(json.dumps({"profile_case": "two_exciton_field", **time_field(steps=args.steps,
                                                                                   warmup=args.warmup)}), flush=True)
            return 0
        if args.only == "states":
            rows = time_states(args.steps, args.warmup, ws)
            if rank == 0:
                print(json.dumps({"profile_case": "n_states sweep", "rows": rows}), flush=True)
            return 0
        sched = tuple(int(x) for x in args.schedule.split(",")) if args.schedule else None
        prec = {"mixed": "fp32_mixed", "fp64": "fp64", "split_tf32": "split_tf32", "dipole": "fp32_mixed"}[args.only]
        case = prop
        if args.only == "dipole":  # seeded unit dipoles, e_p = x
            dip = wl.unit_dipoles(np.random.default_rng(1803013), prop.system.N)
            case = wl.dipole_runs(prop.system, dip, prop.dt_fs, args.steps, "lhcii")[0]
        ms, launches, kt, obs, _ = time_gpu(case, prec, args.steps, args.warmup, ws, None, schedule=sched)
        if rank == 0:
            print(json.dumps({"profile_case": case.system.name, "precision": prec, "n_ado": n_ado,
                              "ms_per_step": ms / args.steps, "kernel": kt, "launches": launches}), flush=True)
        return 0
    clocks = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)

    # headline: mixed precision
    ms, launches, kt, obs, clk = time_gpu(prop, "fp32_mixed", args.steps, args.warmup, ws, clocks)
    ms_max = _max_over_ranks(ms, ws)
    value = _job_value(ws, n_ado, args.steps, ms_max)
    hbm_peak, peak_src = _peaks()
    traffic32, traffic64 = _traffic()
    avg_ms = kt["ms"] / max(kt["launches"], 1)
    # algorithmic bytes of one body launch by the per-unit figure of the roofline (classic RK4: 4 tile
    # transfers of N^2 FP32 complex elements plus 2 M 4-byte link-table entries per ADO-RHS evaluation)
    # x the body ADOs of one launch; the Horner form of RK4 moves 2.75 tile transfers per evaluation,
    # reported beside it as the stricter count
    nb = n_ado - (1 + prop.system.n_modes)
    unit4 = nb * (4.0 * prop.system.N ** 2 * 8 + 2 * prop.system.n_modes * 4)
    ach = unit4 / (avg_ms / 1000.0) / 1e9 if avg_ms > 0 else 0.0
    ach_horner = kt["alg_bytes"] / (kt["ms"] / 1000.0) / 1e9 if kt["ms"] > 0 else 0.0

    # split-TF32 variant: the commutator of the FP32 body on the tensor cores (tcgen05)
    tc_steps = args.tc_steps or max(3, args.steps // 10)
    ms_tc, _, kt_tc, obs_tc, _ = time_gpu(prop, "split_tf32", tc_steps, 3, ws, None)
    ms_tc = _max_over_ranks(ms_tc, ws)
    v_tc = _job_value(ws, n_ado, tc_steps, ms_tc)
    ach_tc = kt_tc["alg_bytes"] / (kt_tc["ms"] / 1000.0) / 1e9 if kt_tc["ms"] > 0 else 0.0
    n = prop.system.N
    k = min(obs_tc.shape[0], obs.shape[0])
    pop_diff_tc = float(np.max(np.abs(obs_tc[:k, :n] - obs[:k, :n])))

    # FP64 over the configuration's full length, and the mixed-vs-FP64 population gate
    fp64, gate = None, None
    if args.gate_steps > 0:
        fp64, gate = fp64_and_gate(prop, args.gate_steps, 3, ws, clocks)
        fp64["mixed_over_fp64"] = value / fp64["value"]
        fp64["roofline"]["traffic"] = traffic64

    # end to end through the public API (host buffers)
    t_e2e, h2d, d2h = time_e2e(prop, "fp32_mixed", args.steps)
    t_e2e = _max_over_ranks(t_e2e, ws)
    e2e_value = _job_value(ws, n_ado, args.steps, 1000.0 * t_e2e)

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 root ADO and reductions)",
            "data": "synthetic",
            "config": {"workload": "lhcii-like N=14 K=1 D=6 (1,344,904 ADOs of 14x14), dt=1 fs, RK4",
                       "precision": "fp32_mixed", "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "no flush: every ADO copy (2.1 GB FP32, 4.2 GB FP64) is larger than the 129 MB L2"},
            "clocks": clk,
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                         "frac": ach / hbm_peak, "traffic": traffic32,
                         "alg_bytes_per_launch": unit4,
                         "alg_bytes": "per-unit figure: 4 N^2 x 8 B + 2 M x 4 B per ADO-RHS evaluation x the body ADOs",
                         "frac_horner": ach_horner / hbm_peak,
                         "alg_bytes_per_launch_horner": kt["alg_bytes"] / max(kt["launches"], 1),
                         "kernel": "stage_kernel<14,float,float> (levels >= 2)",
                         "peak_source": peak_src, "timed_launches": kt["launches"], "avg_launch_ms": avg_ms,
                         "schedule": kt["schedule"]},
            "split_tf32": {"value": v_tc, "unit": UNIT, "steps": tc_steps, "ms_per_step": ms_tc / tc_steps,
                           "pop_diff_vs_mixed": pop_diff_tc,
                           "roofline": {"bound": "hbm", "achieved": ach_tc, "peak": hbm_peak, "unit": "GB/s",
                                        "frac": ach_tc / hbm_peak, "traffic": None,
                                        "kernel": "stage_tc_kernel<14> (tcgen05.mma kind::tf32, levels >= 2)",
                                        "avg_launch_ms": kt_tc["ms"] / max(kt_tc["launches"], 1),
                                        "schedule": kt_tc["schedule"]}},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "what": "hierarchy build + heom_run_create from host arrays + propagate + observables to host, "
                            "wall clock"},
        }
        if not args.no_batch:
            line["batch"] = time_batch()
        if not args.no_field:
            line["two_exciton_field"] = time_field(sm_mhz=(fp64 or {}).get("clocks", {}).get("sm_mhz")
                                                   or (clk or {}).get("sm_mhz"))
        if not args.no_serving and ws == 1:
            line["serving"] = time_serving()
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(prop)
        # the FP64 half of the metric and the mixed-precision gate close the line
        if gate is not None:
            line["mixed_vs_fp64_1000_steps"] = gate
            line["fp64"] = fp64
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

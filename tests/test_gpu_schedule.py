"""Launch schedules and the autotuner (heom_tune, heom_set_autotune, heom_set_schedule,
heom_batch_schedule).  A schedule only changes how chunks of ADOs map onto the GPU -- the grid's
CTAs per SM and, for column-0 runs, how many chunks a warp holds at once (their link records and
neighbour elements load together) -- never which terms an output element sums or their order.  So:

  * every candidate schedule gives bit-identical states and records, for matrix-layout runs
    (CUDA-core FP32 and FP64, the tensor-core body) and column-0 runs, on hierarchies large enough
    that the persistent grid strides (14 sites, D = 4: 35,960 ADOs);
  * tuning leaves the state alone (its probes write only an intermediate copy) and keeps the
    fastest candidate, which a later run of the same kind takes from the cache;
  * batches created with the tuner on give the same records as batches with the default schedule.
"""
import numpy as np
import pytest

from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    from paper_1803_03498_gb300.build import build
    build()
    from paper_1803_03498_gb300 import heom as h
    h.load()
    return h


def medium_pop():
    """LHCII-like 14 sites at D = 4 (35,960 ADOs of 14 x 14)."""
    p = wl.lhcii_like()
    s = p.system
    small = wl.System("lhcii-like D=4", s.H, s.bath_state, s.lambda_cm, s.tau_fs, s.T_K, K=1, D=4)
    return wl.Propagation(small, p.rho0_re, p.rho0_im, dt_fs=1.0, n_steps=6, tag="lhcii-d4-pop")


def medium_dip():
    """Its linear-absorption run (15 states with the ground state: the column-0 layout)."""
    p = medium_pop()
    dip = wl.unit_dipoles(np.random.default_rng(1803013), 14)
    return wl.dipole_runs(p.system, dip, 1.0, 6, "lhcii-d4")[0]


def run_with(heom, prop, precision, sched, n_steps=6, stride=2):
    r = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision=precision, w=prop.w,
                 max_records=n_steps // stride + 2)
    r.set_schedule(*sched, part=0)
    if precision != "fp64":
        r.set_schedule(*sched, part=1)
    r.propagate(prop.dt_fs, n_steps, stride)
    obs = r.observables()
    re, im = r.get_ados(0, r.n_ado)
    layout = r.layout()
    r.close()
    return obs, re, im, layout


@pytest.mark.parametrize("case", ["pop-fp32_mixed", "pop-fp64", "pop-split_tf32", "dip-fp32_mixed", "dip-fp64"])
def test_every_schedule_gives_identical_results(heom, case):
    kind, precision = case.split("-")
    prop = medium_pop() if kind == "pop" else medium_dip()
    layout = 0 if kind == "pop" else 1
    cands = heom.schedule_candidates(layout)
    assert cands[0] == (100, 1)
    ref = run_with(heom, prop, precision, cands[0])
    assert ref[3] == layout
    assert np.all(np.isfinite(ref[1])) and np.max(np.abs(ref[1][1:])) > 0  # the hierarchy is populated
    for c in cands[1:] + [(400, 1)]:  # the tuner's candidates and an oversubscribed grid
        out = run_with(heom, prop, precision, c)
        for a, b in zip(ref[:3], out[:3]):
            assert np.array_equal(a, b), (case, c)


@pytest.mark.parametrize("kind", ["pop", "dip"])
def test_tune_keeps_state_and_picks_fastest(heom, kind):
    prop = medium_pop() if kind == "pop" else medium_dip()
    prev = heom.set_autotune(0)
    try:
        heom.tune_cache_clear()
        # untuned reference
        ref = run_with(heom, prop, "fp32_mixed", (100, 1))
        r = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp32_mixed", w=prop.w, max_records=8)
        assert r.schedule(0) == (100, 1)  # autotuning off, empty cache: the default
        chosen, table = r.tune(part=0, reps=2)
        assert [t for t, _ in table] == heom.schedule_candidates(r.layout())
        ms = [m for _, m in table]
        assert all(m > 0 for m in ms)
        assert chosen == table[int(np.argmin(ms))][0] and r.schedule(0) == chosen
        hchosen, htable = r.tune(part=1, reps=2)
        assert r.schedule(1) == hchosen and len(htable) == len(table)
        r.propagate(prop.dt_fs, 6, 2)  # tuning left the state as it was
        assert np.array_equal(r.observables(), ref[0])
        re, im = r.get_ados(0, r.n_ado)
        assert np.array_equal(re, ref[1]) and np.array_equal(im, ref[2])
        r.close()
        # a new run of the same kind and size takes the tuned schedules from the cache
        r2 = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp32_mixed", w=prop.w, max_records=8)
        assert r2.schedule(0) == chosen and r2.schedule(1) == hchosen
        r2.close()
    finally:
        heom.set_autotune(prev)


def test_schedule_argument_errors(heom):
    p, _ = wl.fmo_like()
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision="fp64", max_records=4)
    for bad in [(0, 1), (1601, 1), (100, 3), (100, 0)]:
        with pytest.raises(heom.HeomError) as ei:
            r.set_schedule(*bad)
        assert ei.value.code == heom.HEOM_E_ARG
    with pytest.raises(heom.HeomError) as ei:  # FP64 runs have no head part
        r.tune(part=1)
    assert ei.value.code == heom.HEOM_E_ARG
    with pytest.raises(heom.HeomError) as ei:
        r.tune(part=0, reps=0)
    assert ei.value.code == heom.HEOM_E_ARG
    r.close()


def test_batch_every_schedule_and_tuned_equal(heom):
    """The ragged-batch shape (dipole runs of several sizes, grouped column-0 launches): every group
    schedule (forced through the default) and the tuner's choices give the same records."""
    props = wl.ragged_batch(n_systems=6, n_steps=20)
    prev = heom.set_autotune(0)
    modes = [("default", c) for c in heom.schedule_candidates(2)] + [("tuned", None)]
    out = []
    try:
        for mode, c in modes:
            heom.tune_cache_clear()
            heom.set_default_schedule(2, c)
            heom.set_autotune(0 if mode == "default" else 2)
            runs = [heom.Run(p.system, p.rho0_re, p.rho0_im, precision="fp32_mixed", w=p.w, max_records=8)
                    for p in props]
            b = heom.Batch(runs, 0.5, 10, 5)
            sch = b.schedules()
            assert len(sch) >= 1
            for body, head in sch:
                assert body in heom.schedule_candidates(2) and head in heom.schedule_candidates(2)
                if mode == "default":
                    assert body == c and head == c
            b.launch(2)
            out.append([r.observables() for r in runs])
            b.close()
            for r in runs:
                r.close()
    finally:
        heom.set_default_schedule(2, None)
        heom.set_autotune(prev)
        heom.tune_cache_clear()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)

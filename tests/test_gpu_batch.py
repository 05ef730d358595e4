"""Ragged batches (heom_batch_create / heom_batch_launch): many propagations of different sizes in one
CUDA graph.  The batched result must equal, bitwise, the same runs propagated one by one with
heom_propagate (same kernels, same order of operations per run), and small FP64 batches must match
the CPU oracle to 1e-12."""
import numpy as np
import pytest

from helpers import oracle_propagate
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    from paper_1803_03498_gb300.build import build
    build()
    from paper_1803_03498_gb300 import heom as h
    h.load()
    return h


def make_runs(heom, props, precision, steps, stride):
    return [heom.Run(p.system, p.rho0_re, p.rho0_im, precision=precision, w=p.w, max_records=steps // stride + 2)
            for p in props]


def mixed_props():
    props = wl.ragged_batch(n_systems=6, n_steps=30)      # 18 dipole runs of different N, D, K
    pop, _ = wl.fmo_like()
    return props + [pop, wl.dimer()]


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp64"])
def test_batch_equals_one_by_one(heom, precision):
    props = mixed_props()
    steps, stride, per_launch = 30, 5, 10
    dt = 0.5
    alone = make_runs(heom, props, precision, steps, stride)
    for r in alone:
        r.propagate(dt, steps, stride)
    batched = make_runs(heom, props, precision, steps, stride)
    b = heom.Batch(batched, dt, per_launch, stride)
    b.launch(steps // per_launch)
    for ra, rb in zip(alone, batched):
        oa, ob = ra.observables(), rb.observables()
        assert oa.shape == ob.shape == (steps // stride + 1, ra.record_len)
        assert np.array_equal(oa, ob)
        sa, sb = ra.get_ados(0, ra.n_ado), rb.get_ados(0, rb.n_ado)
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        assert rb.info()["steps"] == steps
    b.close()


def test_small_fp64_batch_matches_oracle(heom):
    props = [p for p in wl.ragged_batch(n_systems=12, n_steps=20) if p.system.n_ado * p.system.N ** 2 < 20000][:6]
    assert len(props) >= 3
    runs = make_runs(heom, props, "fp64", 20, 1)
    b = heom.Batch(runs, props[0].dt_fs, 10, 1)
    b.launch(2)
    for p, r in zip(props, runs):
        m, ore, oim, oobs = oracle_propagate(p, 20, stride=1)
        g = r.get_ados(0, r.n_ado)
        assert np.max(np.abs((g[0] - ore) + 1j * (g[1] - oim))) <= 1e-12
        assert np.max(np.abs(r.observables()[:, :r.N + 4] - oobs[:, :r.N + 4])) <= 1e-12
    b.close()


def test_batch_argument_errors(heom):
    p = wl.dimer()
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, max_records=3)
    with pytest.raises(heom.HeomError):
        heom.Batch([r], 1.0, 10, 3)      # stride must divide steps_per_launch
    b = heom.Batch([r], 1.0, 10, 5)
    with pytest.raises(heom.HeomError) as ei:
        b.launch(2)                       # 4 more records, room for 2
    assert ei.value.code == heom.HEOM_E_NOMEM
    b.close()


def test_grouped_runs_guard_their_stage_arguments(heom):
    """Column-0 runs of a batch share batched launches whose stage arguments live in the runs'
    workspaces: a run that joins a later batch, or leaves the column-0 layout, makes the earlier batch
    refuse to launch (HEOM_E_STATE) instead of computing with stale arguments."""
    props = [p for p in wl.ragged_batch(n_systems=4, n_steps=10)][:6]
    runs = make_runs(heom, props, "fp32_mixed", 10, 5)
    assert all(r.layout() == 1 for r in runs)
    b1 = heom.Batch(runs, 0.5, 5, 5)
    b1.launch(1)
    b2 = heom.Batch(runs[:2], 0.25, 5, 5)
    with pytest.raises(heom.HeomError) as ei:
        b1.launch(1)
    assert ei.value.code == heom.HEOM_E_STATE
    b2.launch(1)
    b3 = heom.Batch(runs, 0.5, 5, 5)
    re, im = runs[3].get_ados(0, 1)
    re[0, 0, 1] = 0.5  # outside column 0
    runs[3].set_ados(0, re, im)
    assert runs[3].layout() == 0
    with pytest.raises(heom.HeomError) as ei:
        b3.launch(1)
    assert ei.value.code == heom.HEOM_E_STATE
    for b in (b1, b2, b3):
        b.close()

"""heom_group_propagate: many runs advanced together, small mixed-precision runs of equal n_states
sharing one work-list launch per RK4 stage and part.  Every result must equal heom_propagate's bit for
bit (same arithmetic per ADO in the same order), runs of other kinds (FP64, column-0 layout) take their
own launches inside the same call, a run's steps may end before the others', more runs of one size than
one launch holds are split over launches, and a group member stays within 1e-6 of the FP64 oracle."""
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


def _system(rng, N, D, K, name):
    H = np.diag(rng.uniform(12100, 12600, N)) + np.triu(rng.normal(0, 40, (N, N)), 1)
    H = H + np.triu(H, 1).T
    return wl.System(name, H, list(range(N)), list(rng.uniform(20, 100, N)), list(rng.uniform(50, 200, N)),
                     [300.0] * N, K=K, D=D)


def _cases():
    """(propagation, precision, steps): small mixed runs of several sizes (two of N = 5 and of N = 14
    share launches), Hermitian and non-Hermitian starts, plus runs the work lists leave out."""
    rng = np.random.default_rng(1803200)
    out = []
    for N, D, K, steps in [(2, 3, 0, 37), (5, 3, 1, 50), (5, 2, 1, 23), (7, 3, 1, 41), (8, 2, 0, 50), (14, 2, 1, 19),
                           (14, 3, 0, 50), (16, 2, 1, 33), (24, 1, 1, 12)]:
        s = _system(rng, N, D, K, f"N={N} D={D} K={K}")
        rho = np.zeros((N, N))
        rho[0, 0] = 1.0
        rim = np.zeros((N, N))
        if N == 5 and steps == 23:  # a non-Hermitian start: the general link path
            rho[0, 1] = 0.3
            rim[1, 0] = 0.2
        out.append((wl.Propagation(s, rho, rim, 0.5, steps), "fp32_mixed", steps))
    pop, dips = wl.fmo_like()
    out.append((pop, "fp64", 25))                  # FP64: own launches
    out.append((dips[1], "fp32_mixed", 30))        # column-0 layout: own launches
    return out


def _run(heom, p, precision, max_records):
    return heom.Run(p.system, p.rho0_re, p.rho0_im, precision=precision, w=p.w, max_records=max_records)


def test_group_equals_one_by_one(heom):
    cases = _cases()
    stride = 3
    alone = []
    for p, prec, steps in cases:
        r = _run(heom, p, prec, steps // stride + 3)
        r.propagate(p.dt_fs, steps, stride)
        alone.append((r.observables(), *r.get_ados(0, r.n_ado)))
        r.close()
    runs = [_run(heom, p, prec, steps // stride + 3) for p, prec, steps in cases]
    heom.group_propagate(runs, 0.5, [c[2] for c in cases], obs_stride=stride)
    for (p, prec, steps), r, (obs, re, im) in zip(cases, runs, alone):
        assert r.info()["steps"] == steps
        gobs = r.observables()
        gre, gim = r.get_ados(0, r.n_ado)
        assert np.array_equal(gobs, obs), p.system.name
        assert np.array_equal(gre, re) and np.array_equal(gim, im), p.system.name
    for r in runs:
        r.close()


def test_more_runs_of_one_size_than_one_launch_holds(heom):
    """300 dimers of different couplings (64 per launch at most): each equals its own propagation."""
    rng = np.random.default_rng(1803201)
    props = []
    for k in range(300):
        H = np.array([[0.0, rng.uniform(20, 80)], [0.0, rng.uniform(50, 150)]])
        H[1, 0] = H[0, 1]
        s = wl.System(f"dimer {k}", H, [0, 1], [35.0, 35.0], [50.0, 50.0], [300.0, 300.0], K=0, D=3)
        props.append(wl.Propagation(s, np.diag([1.0, 0.0]), np.zeros((2, 2)), 1.0, 20))
    runs = [_run(heom, p, "fp32_mixed", 3) for p in props]
    heom.group_propagate(runs, 1.0, 20, obs_stride=20)
    for k in (0, 255, 256, 299):
        r = _run(heom, props[k], "fp32_mixed", 3)
        r.propagate(1.0, 20, 20)
        assert np.array_equal(r.observables(), runs[k].observables())
        r.close()
    for r in runs:
        r.close()


def test_group_member_against_oracle(heom):
    p, prec, steps = _cases()[3]  # N = 7, D = 3, K = 1
    m, ore, oim, oobs = oracle_propagate(p, steps, stride=1)
    others = [_run(heom, q, pr, st + 2) for q, pr, st in _cases()[:3]]
    r = _run(heom, p, prec, steps + 2)
    heom.group_propagate([r] + others, p.dt_fs, [steps] + [c[2] for c in _cases()[:3]], obs_stride=1)
    N = p.system.N
    assert np.max(np.abs(r.observables()[:, :N] - oobs[:, :N])) <= 1e-6
    for x in [r] + others:
        x.close()


def test_group_errors(heom):
    p, prec, steps = _cases()[1]
    r = _run(heom, p, prec, 4)
    with pytest.raises(heom.HeomError) as ei:
        heom.group_propagate([r, r], 0.5, 2)
    assert ei.value.code == heom.HEOM_E_ARG
    with pytest.raises(heom.HeomError) as ei:
        heom.group_propagate([r], 50.0, 2)
    assert ei.value.code == heom.HEOM_E_ARG
    with pytest.raises(heom.HeomError) as ei:
        heom.group_propagate([r], 0.5, 10, obs_stride=1)  # 10 records, room for 3
    assert ei.value.code == heom.HEOM_E_NOMEM
    r.set_timing(True)
    with pytest.raises(heom.HeomError) as ei:
        heom.group_propagate([r], 0.5, 2)
    assert ei.value.code == heom.HEOM_E_STATE
    r.close()

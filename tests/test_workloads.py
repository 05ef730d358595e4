"""The seeded synthetic inputs (paper_1803_03498_gb300/workloads.py) have the shapes and ranges the
benchmark and tests state, and the same seed gives the same arrays (the oracle and the GPU path are
fed from these generators, so both sides see identical inputs)."""
from math import comb

import numpy as np

from paper_1803_03498_gb300 import workloads as wl


def test_fmo_and_lhcii_shapes():
    pop, dips = wl.fmo_like()
    s = pop.system
    assert s.N == 7 and s.n_modes == 14 and s.n_ado == 3060
    assert np.allclose(s.H, s.H.T) and np.all((np.diag(s.H) >= 12100) & (np.diag(s.H) <= 12600))
    assert len(dips) == 3 and all(d.system.N == 8 for d in dips)
    for p, d in enumerate(dips):  # sigma_0(0) = mu_p^+ |0><0|: column 0 holds the weights e_p . d_a
        assert np.array_equal(d.rho0_re[:, 0], d.w) and not np.any(d.rho0_re[:, 1:])
        assert d.w[0] == 0.0
    lh = wl.lhcii_like().system
    assert lh.N == 14 and lh.n_modes == 28 and lh.n_ado == 1344904
    assert np.all((np.diag(lh.H) >= 14800) & (np.diag(lh.H) <= 15300))


def test_seeded_determinism():
    a, b = wl.fmo_like(), wl.fmo_like()
    assert np.array_equal(a[0].system.H, b[0].system.H)
    assert all(np.array_equal(x.w, y.w) for x, y in zip(a[1], b[1]))
    r1, r2 = wl.random_state(10, 3, seed=4), wl.random_state(10, 3, seed=4)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])
    assert not np.array_equal(r1[0], wl.random_state(10, 3, seed=5)[0])


def test_ragged_batch_ranges():
    props = wl.ragged_batch()
    assert len(props) == 192
    assert sum(p.system.n_ado for p in props) == 2597400
    for p in props:
        s = p.system
        n_sites = s.N - 1
        assert 2 <= n_sites <= 16 and 3 <= s.D <= 5 and s.K in (0, 1)
        assert all(20 <= x <= 100 for x in s.lambda_cm) and all(50 <= x <= 200 for x in s.tau_fs)
        assert len(set(s.T_K)) == 1 and s.T_K[0] in (77.0, 300.0)
        assert p.w is not None and p.dt_fs == 0.5


def test_serving_stream_poisson_and_redraw():
    reqs = wl.serving_stream(20.0, 400, max_ado_steps=2e7)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(np.mean(gaps) - 1 / 20.0) < 0.2 / 20.0  # exponential gaps with mean 1/rate (400 draws)
    for r in reqs:
        s = r.prop.system
        assert 2 <= s.N <= 24 and 2 <= s.D <= 6 and s.K in (0, 1)
        assert 200 <= r.prop.n_steps <= 5000
        assert comb(s.n_modes + s.D, s.D) * r.prop.n_steps <= 2e7
    full = wl.serving_stream(20.0, 400)
    assert max(comb(r.prop.system.n_modes + r.prop.system.D, r.prop.system.D) * r.prop.n_steps for r in full) > 2e7


def test_two_exciton_workload():
    prop, pulse = wl.fmo_two_exciton(n_sites=7, D=4)
    s = prop.system
    assert s.N == 29 and s.n_ado == 3060 and s.bath_mask.shape == (7, 29)
    # each site's number operator: its single and the 6 pairs containing it
    assert np.all(s.bath_mask.sum(axis=1) == 7)
    assert prop.rho0_re[0, 0] == 1.0 and np.sum(np.abs(prop.rho0_re)) == 1.0
    assert pulse.mu_plus.shape == (29, 29) and np.all(np.diag(pulse.mu_plus) == 0)
    # M+ only raises the excitation number by one: ground -> singles, singles -> pairs
    nz = np.argwhere(pulse.mu_plus != 0)
    level = np.array([0] + [1] * 7 + [2] * 21)
    assert np.all(level[nz[:, 0]] == level[nz[:, 1]] + 1)

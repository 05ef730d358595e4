"""The two-exciton space and the RWA laser field on the GPU (general stage kernel): section "Optical
spectra", Eq. h-field-rwa with the Gaussian pulse of Eq. probe_pulse, and the two-exciton states of
section "Dipole operators and rotational averaging".  Every check compares the library with the
oracle on the same inputs:

  * a pumped two-exciton FMO-like system (4 sites: 11 states; 7 sites: 29 states) propagated by
    classic four-copy RK4 with H(t) at the stage times: every element of every ADO within 1e-12
    in FP64, populations within 1e-6 in mixed precision;
  * without a field (Horner RK4 on the general kernel) from a one-exciton state, and a one-exciton
    system of 26 sites (above the specialised kernels' 24 states);
  * one right-hand side at a time inside the pulse on a random state;
  * removing the field mid-run, and the errors of the field calls.
"""
import numpy as np
import pytest

from helpers import oracle_for, oracle_start
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    from paper_1803_03498_gb300.build import build
    build()
    from paper_1803_03498_gb300 import heom as h
    h.load()
    return h


def oracle_pumped(prop, pulse, n_steps, stride):
    m = oracle_for(prop.system)
    m.set_field(pulse.mu_plus, pulse.amp_cm, pulse.t_center_fs, pulse.sigma_fs, pulse.phase, pulse.detuning_cm)
    re, im = oracle_start(m, prop.rho0_re, prop.rho0_im)
    obs = m.rk4(re, im, prop.dt_fs, n_steps, obs_stride=stride)
    return m, re, im, obs


def gpu_pumped(heom, prop, pulse, precision, n_steps, stride):
    r = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision=precision, max_records=n_steps // stride + 2,
                 time_dependent=True)
    r.set_field(pulse)
    r.propagate(prop.dt_fs, n_steps, stride)
    return r, r.observables()


@pytest.mark.parametrize("n_sites,D,steps", [(4, 3, 200), (7, 2, 120)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_pumped_two_exciton_matches_oracle(heom, n_sites, D, steps, precision):
    prop, pulse = wl.fmo_two_exciton(n_sites=n_sites, D=D)
    pulse.phase, pulse.detuning_cm = 0.4, 30.0  # complex H(t): phase and a detuned carrier
    m, re, im, oobs = oracle_pumped(prop, pulse, steps, 10)
    r, gobs = gpu_pumped(heom, prop, pulse, precision, steps, 10)
    N = prop.system.N
    assert r.layout() == 0 and N == 1 + n_sites + n_sites * (n_sites - 1) // 2
    assert gobs.shape[0] == oobs.shape[0]
    pops = oobs[:, :N]
    assert pops[-1, 0] < 0.99 and np.max(pops[-1, n_sites + 1:]) > 1e-6  # pumped, some pair population
    if precision == "fp64":
        gre, gim = r.get_ados(0, m.n_ado)
        assert np.max(np.abs((gre - re) + 1j * (gim - im))) <= 1e-12
        assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= 1e-12
    else:
        assert np.max(np.abs(gobs[:, :N] - pops)) <= 1e-6
    assert np.max(np.abs(gobs[:, N] - 1.0)) <= 1e-10   # trace
    # sigma_0 stays Hermitian (each element is computed on its own; FP32 levels >= 2 feed it in the
    # mixed precision)
    assert np.max(gobs[:, N + 4]) <= (1e-12 if precision == "fp64" else 1e-7)
    r.close()


def test_two_exciton_without_field_and_26_sites(heom):
    # general kernel, Horner RK4: a one-exciton start in the two-exciton space
    prop, _ = wl.fmo_two_exciton(n_sites=4, D=3)
    r0 = np.zeros((prop.system.N, prop.system.N))
    r0[1, 1] = 1.0
    m = oracle_for(prop.system)
    re, im = oracle_start(m, r0, np.zeros_like(r0))
    oobs = m.rk4(re, im, 0.5, 200, obs_stride=20)
    r = heom.Run(prop.system, r0, None, precision="fp64", max_records=16)
    r.propagate(0.5, 200, 20)
    gre, gim = r.get_ados(0, m.n_ado)
    assert np.max(np.abs((gre - re) + 1j * (gim - im))) <= 1e-12
    assert np.max(np.abs(r.observables()[:, :m.N + 4] - oobs)) <= 1e-12
    r.close()
    # 26 sites, one bath each (no mask): above the specialised kernels' 24 states
    rng = np.random.default_rng(1803026)
    n = 26
    H = rng.normal(0.0, 30.0, (n, n))
    H = (H + H.T) / 2
    H[np.diag_indices(n)] = rng.uniform(-150.0, 150.0, n)
    big = wl.System("26 sites", H, list(range(n)), [35.0] * n, [50.0] * n, [300.0] * n, K=0, D=2)
    r0 = np.zeros((n, n))
    r0[0, 0] = 1.0
    m = oracle_for(big)
    re, im = oracle_start(m, r0, np.zeros_like(r0))
    oobs = m.rk4(re, im, 1.0, 60, obs_stride=20)
    for precision, tol in (("fp64", 1e-12), ("fp32_mixed", 1e-6)):
        r = heom.Run(big, r0, None, precision=precision, max_records=8)
        r.propagate(1.0, 60, 20)
        gobs = r.observables()
        assert np.max(np.abs(gobs[:, :n] - oobs[:, :n])) <= tol
        if precision == "fp64":
            gre, gim = r.get_ados(0, m.n_ado)
            assert np.max(np.abs((gre - re) + 1j * (gim - im))) <= 1e-12
        r.close()


def test_rhs_inside_the_pulse(heom):
    prop, pulse = wl.fmo_two_exciton(n_sites=4, D=2)
    pulse.phase, pulse.detuning_cm = 1.1, -20.0
    r = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp64", max_records=8, time_dependent=True)
    r.set_field(pulse)
    r.propagate(prop.dt_fs, 70, 0)  # t = 35 fs, inside the pulse
    m = oracle_for(prop.system)
    m.set_field(pulse.mu_plus, pulse.amp_cm, pulse.t_center_fs, pulse.sigma_fs, pulse.phase, pulse.detuning_cm)
    m.set_time(35.0)
    rng = np.random.default_rng(5)
    re = rng.standard_normal((m.n_ado, m.N, m.N))
    im = rng.standard_normal((m.n_ado, m.N, m.N))
    r.set_ados(0, re, im)
    gre, gim = r.rhs_eval(0, m.n_ado)
    ore, oim = m.rhs(re, im)
    assert np.max(np.abs((gre - ore) + 1j * (gim - oim))) <= 1e-12 * np.max(np.abs(ore + 1j * oim))
    r.close()


def test_field_removed_mid_run_and_errors(heom):
    prop, pulse = wl.fmo_two_exciton(n_sites=3, D=2)
    m = oracle_for(prop.system)
    m.set_field(pulse.mu_plus, pulse.amp_cm, pulse.t_center_fs, pulse.sigma_fs)
    re, im = oracle_start(m, prop.rho0_re, prop.rho0_im)
    m.rk4(re, im, 0.5, 100)              # 0 .. 50 fs with the pulse
    m.set_field(None, 0, 0, 1)
    m.rk4(re, im, 0.5, 60, t0=50.0)      # then without it
    r = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp64", max_records=8, time_dependent=True)
    r.set_field(pulse)
    r.propagate(0.5, 100, 0)
    r.set_field(None)
    r.propagate(0.5, 60, 0)
    gre, gim = r.get_ados(0, m.n_ado)
    assert np.max(np.abs((gre - re) + 1j * (gim - im))) <= 1e-12
    with pytest.raises(heom.HeomError) as ei:  # a field needs a run with the fourth copy
        q = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision="fp64", max_records=2)
        q.set_field(pulse)
    assert ei.value.code == heom.HEOM_E_STATE
    bad = wl.Pulse(pulse.mu_plus, 10.0, 0.0, 0.0)
    with pytest.raises(heom.HeomError) as ei:
        r.set_field(bad)
    assert ei.value.code == heom.HEOM_E_ARG
    r.set_field(pulse)
    with pytest.raises(heom.HeomError) as ei:  # a batch graph would replay fixed times
        heom.Batch([r], 0.5, 2, 1)
    assert ei.value.code == heom.HEOM_E_ARG
    r.close()

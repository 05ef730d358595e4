"""Thermal state and static fluorescence (section "Static Fluorescence Spectra") on the GPU path:

  * the dimer's thermal state from a long GPU propagation of the Boltzmann state equals the null
    vector of the dense hierarchy Liouvillian (built from the oracle's modes), trace 1, to 1e-6, and
    its residual |L sigma| / |sigma| is small;
  * an emission run (every ADO of the FMO-like thermal state times mu_p^+, on the ground + sites
    space) propagated on the GPU in FP64 gives the oracle's correlation function from the same start
    to 1e-12, with C(0) = d_p^T sigma_0(inf) d_p;
  * the fluorescence maximum lies below the absorption maximum (Stokes shift).
"""
import copy

import numpy as np
import pytest
import scipy.linalg

import liouvillian as lv
from helpers import oracle_for
from paper_1803_03498_gb300 import spectra
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_03498_gb300.build import build
    build()


def test_dimer_thermal_state_is_liouvillian_null_vector():
    p = wl.dimer()
    s = p.system
    re, im, resid = spectra.thermal_state(s, 1.0, 6000)
    m = oracle_for(s)
    L, tuples, index = lv.build_from_oracle(m)
    ns = scipy.linalg.null_space(L)
    assert ns.shape[1] == 1
    t, _, _ = m.hierarchy()
    v = lv.from_vec(ns[:, 0], t, index, s.N)
    v = v / np.trace(v[0])
    g = re + 1j * im
    assert abs(np.trace(g[0]) - 1.0) <= 1e-12
    assert np.max(np.abs(g - v)) <= 1e-6
    assert resid <= 1e-7


def test_fmo_emission_run_matches_oracle_and_is_red_shifted():
    pop, dips = wl.fmo_like()
    s = copy.deepcopy(pop.system)
    s.D = 3
    tre, tim, resid = spectra.thermal_state(s, 1.0, 4000)
    assert resid <= 1e-4
    dip = wl.unit_dipoles(np.random.default_rng(1803012), 7)
    g_sys = wl.dipole_runs(s, dip, 0.5, 300, "fl")[0].system  # ground + sites, rotating frame
    n_steps, dt = 300, 0.5
    fl_c, la_c = [], []
    for p_ in range(3):
        w = np.zeros(8)
        w[1:] = dip[:, p_]
        xre, xim = spectra.emission_start(tre, tim, dip[:, p_])
        obs, _, _, _ = spectra.propagate_state(g_sys, xre, xim, dt, n_steps, stride=1, w=w)
        m = oracle_for(g_sys)
        ore, oim = xre.copy(), xim.copy()
        oobs = m.rk4(ore, oim, dt, n_steps, obs_stride=1, w=w)
        gc, oc = spectra.correlations(obs, 8), spectra.correlations(oobs, 8)
        assert np.max(np.abs(gc - oc)) <= 1e-12
        d = dip[:, p_]
        assert abs(gc[0] - d @ (tre[0] + 1j * tim[0]) @ d) <= 1e-12
        fl_c.append(gc)
        # absorption from the ground state with the same dipole
        a = np.zeros((g_sys.n_ado, 8, 8))
        a[0, 1:, 0] = d
        aobs, _, _, _ = spectra.propagate_state(g_sys, a, np.zeros_like(a), dt, n_steps, stride=1, w=w)
        la_c.append(spectra.correlations(aobs, 8))
    _, wref = wl.with_ground_state(s.H)
    e, fl = spectra.spectrum(np.array(fl_c), dt, omega_ref_cm=wref)
    _, la = spectra.spectrum(np.array(la_c), dt, omega_ref_cm=wref)
    band = (e > wref - 1500) & (e < wref + 1500)
    assert e[band][np.argmax(fl[band])] < e[band][np.argmax(la[band])]

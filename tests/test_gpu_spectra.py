"""Spectra from GPU propagations: the three circular-dichroism runs of the FMO-like system
(3060 ADOs, ground state + 7 sites) on the GPU in FP64 give the oracle's correlation functions to
1e-12 and therefore its CD spectrum; the linear-absorption spectrum of the 4000-step GPU dipole runs
equals the one of the stored oracle trajectories."""
import os

import numpy as np
import pytest

from helpers import gpu_run, oracle_propagate
from paper_1803_03498_gb300 import spectra
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_03498_gb300.build import build
    build()


def test_cd_spectrum_gpu_equals_oracle():
    pop, _ = wl.fmo_like()
    dip = wl.unit_dipoles(np.random.default_rng(1803012), 7)
    pos = wl.site_positions(np.random.default_rng(1803022), 7)
    runs = wl.cd_runs(pop.system, dip, pos, 0.5, 300, "fmo")
    g, o = [], []
    for p in runs:
        _, gobs = gpu_run(p, "fp64", stride=1)
        _, _, _, oobs = oracle_propagate(p, p.n_steps, stride=1)
        g.append(spectra.correlations(gobs, p.system.N))
        o.append(spectra.correlations(oobs, p.system.N))
    g, o = np.array(g), np.array(o)
    assert np.max(np.abs(g - o)) <= 1e-12
    _, wref = wl.with_ground_state(pop.system.H)
    _, sg = spectra.spectrum(g, 0.5, omega_ref_cm=wref)
    _, so = spectra.spectrum(o, 0.5, omega_ref_cm=wref)
    assert np.max(np.abs(sg - so)) <= 1e-10 * np.max(np.abs(so))


def test_absorption_spectrum_gpu_equals_oracle():
    pop, dips = wl.fmo_like()
    g, o = [], []
    for p, tag in zip(dips, ("dip0", "dip1", "dip2")):
        _, gobs = gpu_run(p, "fp64", stride=10)
        g.append(spectra.correlations(gobs, p.system.N))
        o.append(spectra.correlations(np.loadtxt(os.path.join(GOLDEN, f"fmo_like_{tag}.txt")), p.system.N))
    _, wref = wl.with_ground_state(pop.system.H)
    _, sg = spectra.spectrum(np.array(g), 5.0, omega_ref_cm=wref)
    _, so = spectra.spectrum(np.array(o), 5.0, omega_ref_cm=wref)
    assert np.max(np.abs(sg - so)) <= 1e-9 * np.max(np.abs(so))

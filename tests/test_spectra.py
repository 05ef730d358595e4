"""Spectra from dipole correlation functions (paper_1803_03498_gb300/spectra.py; sections "Linear
absorption spectra" and "Circular dichroism spectra").  CPU checks against closed forms and sum rules:

  * a single damped oscillation C(t) = exp(-(g + i W) t): the trapezoid sum has the closed form
    dt [1/2 + q / (1 - q)], q = exp((i w - g - i W) dt) (a geometric series), and tends to the
    Lorentzian g / (g^2 + (w - W)^2) as dt -> 0;
  * the sum rule (1 / 2pi) sum_j S_j dw = Re C(0) / 2 of the discrete transform; for the stored
    FMO-like oracle correlations that is sum_a |d_a|^2 / 2 = 3.5 (seven unit dipoles);
  * the absorption maximum lies inside the exciton band of the site Hamiltonian;
  * circular dichroism is conservative: C_CD(0) = sum_a d_a . (R_a x d_a) = 0, so the CD spectrum
    integrates to zero (an oracle propagation of the three CD runs of a small FMO-like hierarchy).
"""
import os

import numpy as np

from helpers import oracle_propagate
from paper_1803_03498_gb300 import spectra
from paper_1803_03498_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_single_exponential_closed_form_and_lorentzian():
    g, W, dt, n_t = 0.01, 0.05, 0.25, 6000  # rad/fs, fs; exp(-g T) = 3e-7
    t = dt * np.arange(n_t)
    c = np.exp(-(g + 1j * W) * t)
    e_cm, s = spectra.spectrum(c, dt, n_fft=1 << 16)
    w = e_cm * spectra.TWO_PI_C
    q = np.exp((1j * w - g - 1j * W) * dt)
    closed = (dt * (0.5 + q / (1 - q))).real
    assert np.max(np.abs(s - closed)) <= 1e-6 * np.max(np.abs(closed))
    lor = g / (g ** 2 + (w - W) ** 2)
    near = np.abs(w - W) < 0.2
    assert np.max(np.abs(s[near] - lor[near])) <= 2e-3 * np.max(lor)
    assert abs(w[np.argmax(s)] - W) <= 2 * np.pi / (dt * (1 << 16))


def golden_corr():
    out = []
    for p in range(3):
        obs = np.loadtxt(os.path.join(GOLDEN, f"fmo_like_dip{p}.txt"))
        out.append(spectra.correlations(obs, 8))
    return np.array(out)


def test_absorption_sum_rule_and_band():
    pop, dips = wl.fmo_like()
    c = golden_corr()
    dt = dips[0].dt_fs * 10  # the stored records are every 10 steps
    _, omega_ref = wl.with_ground_state(pop.system.H)
    e_cm, s = spectra.spectrum(c, dt, omega_ref_cm=omega_ref)
    dw = (e_cm[1] - e_cm[0]) * spectra.TWO_PI_C
    total = np.sum(s) * dw / (2 * np.pi)
    assert abs(total - 0.5 * np.sum(c[:, 0].real)) <= 1e-12 * abs(total)
    assert abs(np.sum(c[:, 0].real) - 7.0) <= 1e-12  # sum_p sum_a (e_p . d_a)^2 = sum_a |d_a|^2
    eig = np.linalg.eigvalsh(pop.system.H)
    peak = e_cm[np.argmax(s)]
    assert eig[0] - 300 <= peak <= eig[-1] + 300


def test_circular_dichroism_is_conservative():
    pop, _ = wl.fmo_like()
    s = pop.system
    small = wl.System("fmo-like small", s.H, s.bath_state, s.lambda_cm, s.tau_fs, s.T_K, K=0, D=2)
    dip = wl.unit_dipoles(np.random.default_rng(1803012), 7)
    pos = wl.site_positions(np.random.default_rng(1803022), 7)
    runs = wl.cd_runs(small, dip, pos, 1.0, 600, "cd")
    corr = []
    for p in runs:
        _, _, _, obs = oracle_propagate(p, p.n_steps, stride=1)
        corr.append(obs[:, small.N + 1 + 2] + 1j * obs[:, small.N + 1 + 3])
    corr = np.array(corr)
    rot = spectra.rotational_strengths(pos, dip)
    assert abs(np.sum(corr[:, 0])) <= 1e-13 * np.sum(np.abs(rot))
    _, omega_ref = wl.with_ground_state(s.H)
    e_cm, cd = spectra.spectrum(corr, 1.0, omega_ref_cm=omega_ref)
    dw = (e_cm[1] - e_cm[0]) * spectra.TWO_PI_C
    assert abs(np.sum(cd) * dw / (2 * np.pi)) <= 1e-12 * np.sum(np.abs(cd)) * dw
    assert np.max(np.abs(cd)) > 1.0  # not trivially zero


def test_boltzmann_state():
    """exp(-H0/kT)/Z with H0 = H minus the reorganisation energies: trace 1, commutes with H0, and for a
    diagonal H0 the populations are the Boltzmann factors."""
    pop, _ = wl.fmo_like()
    s = pop.system
    rho = spectra.boltzmann_state(s)
    H0 = s.H - np.diag(s.lambda_cm)
    assert abs(np.trace(rho) - 1.0) <= 1e-14
    assert np.max(np.abs(rho @ H0 - H0 @ rho)) <= 1e-10
    d = wl.System("diag", np.diag([0.0, 100.0, 250.0]), [0, 1, 2], [35.0] * 3, [50.0] * 3, [300.0] * 3, K=0, D=1)
    p = np.exp(-np.array([0.0, 100.0, 250.0]) / (0.6950348004 * 300.0))
    assert np.allclose(np.diag(spectra.boltzmann_state(d)), p / p.sum(), rtol=1e-13, atol=0)

"""Pins of the oracle's two-exciton space and laser field (section "Optical spectra": Eq. h-field-rwa
with the Gaussian pulse of Eq. probe_pulse; section "Dipole operators and rotational averaging": the
two-exciton states), checked against what the mathematics fixes:

  * the two-exciton Hamiltonian, dipole operator and site-number operators of workloads.two_exciton
    equal those of the full 2^N spin space (hard-core excitons, Kronecker products of 2 x 2 Pauli
    matrices) restricted to at most two excitations;
  * a resonant Gaussian pulse rotates a two-level system by its pulse area: rho(t) = U rho(0) U^+,
    U = exp(i theta(t) K) with theta(t) = int_0^t E(t') dt' (closed form through erf) and
    K = e^{-i phi} M+ + e^{i phi} M- (the Hamiltonian is -E(t) K at every time, so it commutes with
    itself);
  * two uncoupled resonant sites in the two-exciton space rotate independently: every population is
    a product of the single-site ones, sin^2 or cos^2 of w_a theta(t);
  * a zero-amplitude field changes nothing (bit for bit);
  * started in the one-exciton block, the two-exciton model with site-number baths reproduces the
    one-exciton model with a ground state (the pairs stay empty);
  * the right-hand side with diagonal multi-state couplings equals the dense Kronecker Liouvillian
    built from the exported modes and the same diagonals (terminator included), at a time with the
    field on.
"""
from math import erf, sqrt, pi

import numpy as np
import pytest
from scipy.linalg import expm

from helpers import oracle_for, oracle_start
from liouvillian import build_general, from_vec, to_vec
from oracle.oracle import Bath, OracleModel
from paper_1803_03498_gb300 import workloads as wl

TWO_PI_C = 1.8836515673088532e-4


def spin_space(Hs, w, omega_ref):
    """H, M+ and the number operators on the 2^n spin space, restricted to <= 2 excitations in the
    two-exciton order (ground, singles a, pairs (a, b) lexicographic)."""
    n = len(Hs)
    sp = np.array([[0.0, 0.0], [1.0, 0.0]])  # sigma+ on (ground, excited)
    num = np.diag([0.0, 1.0])

    def at(a, o):
        out = np.array([[1.0]])
        for k in range(n):
            out = np.kron(out, o if k == a else np.eye(2))
        return out

    Hf = sum((Hs[a, a] - omega_ref) * at(a, num) for a in range(n))
    Hf = Hf + sum(Hs[a, b] * at(a, sp) @ at(b, sp).T for a in range(n) for b in range(n) if a != b)
    Mf = sum(w[a] * at(a, sp) for a in range(n))
    Nf = [at(a, num) for a in range(n)]

    def state(bits):  # index of a basis vector with the given sites excited (site 0 = leading factor)
        return sum(1 << (n - 1 - a) for a in bits)

    order = [state([])] + [state([a]) for a in range(n)] + [state([a, b]) for a in range(n) for b in range(a + 1, n)]
    sel = np.ix_(order, order)
    return Hf[sel], Mf[sel], [x[sel] for x in Nf]


def test_two_exciton_space_equals_spin_construction():
    rng = np.random.default_rng(7)
    n = 4
    Hs = rng.normal(0, 40, (n, n))
    Hs = (Hs + Hs.T) / 2
    Hs[np.diag_indices(n)] = rng.uniform(12100, 12600, n)
    sysm = wl.System("t", Hs, list(range(n)), [35.0] * n, [100.0] * n, [300.0] * n, K=0, D=1)
    w = rng.normal(size=n)
    g, pairs = wl.two_exciton(sysm, omega_ref=12300.0)
    H2, M2, N2 = spin_space(Hs, w, 12300.0)
    assert g.N == 1 + n + n * (n - 1) // 2 == H2.shape[0]
    assert np.allclose(g.H, H2, atol=1e-9, rtol=0)
    assert np.array_equal(wl.two_exciton_dipole(n, w), M2)
    for b in range(n):
        assert np.array_equal(np.diag(g.bath_mask[b]).astype(float), N2[b])
    assert g.bath_state == [1 + b for b in range(n)]


def area(t, amp_cm, tc, sig):
    """int_0^t amp exp(-(t' - tc)^2 / (2 sig^2)) dt' in rad."""
    a = amp_cm * TWO_PI_C
    return a * sig * sqrt(pi / 2) * (erf((t - tc) / (sig * sqrt(2))) + erf(tc / (sig * sqrt(2))))


@pytest.mark.parametrize("phase", [0.0, 0.7])
def test_resonant_pulse_rotates_two_level_system(phase):
    H = np.zeros((2, 2))  # ground and one site at the reference energy
    m = OracleModel(H, [Bath(1, 0.0, 100.0, 300.0)], K=0, D=1)  # lambda = 0: unitary
    Mp = np.array([[0.0, 0.0], [1.0, 0.0]])
    amp, tc, sig = 150.0, 30.0, 10.0
    m.set_field(Mp, amp, tc, sig, phase=phase)
    re, im = oracle_start(m, np.diag([1.0, 0.0]), np.zeros((2, 2)))
    dt, steps = 0.1, 800
    obs = m.rk4(re, im, dt, steps, obs_stride=100)
    K = np.exp(-1j * phase) * Mp + np.exp(1j * phase) * Mp.T
    rho0 = np.diag([1.0, 0.0]).astype(complex)
    for k in range(obs.shape[0]):
        th = area(k * 100 * dt, amp, tc, sig)
        U = expm(1j * th * K)
        rho = U @ rho0 @ U.conj().T
        assert np.max(np.abs(obs[k, :2] - rho.diagonal().real)) <= 1e-9
    U = expm(1j * area(steps * dt, amp, tc, sig) * K)
    rho = U @ rho0 @ U.conj().T
    assert np.max(np.abs((re[0] + 1j * im[0]) - rho)) <= 1e-9
    assert abs(area(steps * dt, amp, tc, sig)) > 0.5  # a large rotation, not a small-angle check


def test_two_uncoupled_sites_rotate_independently():
    Hs = np.diag([12300.0, 12300.0])
    sysm = wl.System("pair", Hs, [0, 1], [0.0, 0.0], [100.0, 100.0], [300.0, 300.0], K=0, D=1)
    g, _ = wl.two_exciton(sysm, omega_ref=12300.0)
    m = oracle_for(g)
    w = np.array([0.8, 0.5])
    amp, tc, sig = 200.0, 30.0, 10.0
    m.set_field(wl.two_exciton_dipole(2, w), amp, tc, sig)
    r0 = np.zeros((4, 4))
    r0[0, 0] = 1.0
    re, im = oracle_start(m, r0, np.zeros((4, 4)))
    obs = m.rk4(re, im, 0.1, 800, obs_stride=200)
    for k in range(obs.shape[0]):
        th = area(k * 200 * 0.1, amp, tc, sig)
        e1, e2 = np.sin(w * th) ** 2
        g1, g2 = 1 - e1, 1 - e2
        expect = [g1 * g2, e1 * g2, g1 * e2, e1 * e2]  # ground, site 1, site 2, pair (1, 2)
        assert np.max(np.abs(obs[k, :4] - expect)) <= 1e-9
    assert obs[-1, 3] > 0.05


def test_zero_amplitude_field_changes_nothing():
    prop, pulse = wl.fmo_two_exciton(n_sites=3, D=2)
    a = oracle_for(prop.system)
    b = oracle_for(prop.system)
    b.set_field(pulse.mu_plus, 0.0, pulse.t_center_fs, pulse.sigma_fs)
    ra, ia = oracle_start(a, prop.rho0_re, prop.rho0_im)
    rb, ib = oracle_start(b, prop.rho0_re, prop.rho0_im)
    ra[0] = np.diag(np.arange(a.N, dtype=float)) / a.N
    rb[0] = ra[0]
    oa = a.rk4(ra, ia, 0.5, 20)
    ob = b.rk4(rb, ib, 0.5, 20)
    assert np.array_equal(oa, ob) and np.array_equal(ra, rb) and np.array_equal(ia, ib)


def test_two_exciton_reduces_to_one_exciton():
    pop, _ = wl.fmo_like()
    s = pop.system
    n = 3
    sites = wl.System("3 sites", np.asarray(s.H)[:n, :n], list(range(n)), [35.0] * n, [166.0] * n, [77.0] * n, K=1, D=2)
    g, _ = wl.two_exciton(sites)
    Hg, _ = wl.with_ground_state(sites.H, omega_ref=float(np.mean(np.diag(sites.H))))
    one = wl.System("one", Hg, [1 + b for b in range(n)], sites.lambda_cm, sites.tau_fs, sites.T_K, K=1, D=2)
    m2, m1 = oracle_for(g), oracle_for(one)
    r2 = np.zeros((g.N, g.N))
    r2[1, 1] = 1.0
    r1 = np.zeros((n + 1, n + 1))
    r1[1, 1] = 1.0
    re2, im2 = oracle_start(m2, r2, np.zeros_like(r2))
    re1, im1 = oracle_start(m1, r1, np.zeros_like(r1))
    o2 = m2.rk4(re2, im2, 0.5, 200, obs_stride=20)
    o1 = m1.rk4(re1, im1, 0.5, 200, obs_stride=20)
    assert np.max(np.abs(o2[:, :n + 1] - o1[:, :n + 1])) <= 1e-12
    assert np.max(np.abs(o1[-1, 2:n + 1])) > 1e-4  # energy moved between the sites
    assert not np.any(re2[:, n + 1:, :]) and not np.any(re2[:, :, n + 1:])  # the pairs stay empty
    assert np.max(np.abs((re2[:, :n + 1, :n + 1] - re1) + 1j * (im2[:, :n + 1, :n + 1] - im1))) <= 1e-12


@pytest.mark.parametrize("terminator", [True, False])
def test_masked_rhs_equals_dense_liouvillian(terminator):
    prop, pulse = wl.fmo_two_exciton(n_sites=3, D=2)
    s = prop.system
    m = OracleModel(s.H, [Bath(st, l, t, T) for st, l, t, T in zip(s.bath_state, s.lambda_cm, s.tau_fs, s.T_K)],
                    K=s.K, D=s.D, terminator=terminator, bath_mask=s.bath_mask)
    t_eval = 37.0
    m.set_field(pulse.mu_plus, pulse.amp_cm, pulse.t_center_fs, pulse.sigma_fs, phase=0.3, detuning_cm=25.0)
    m.set_time(t_eval)
    md = m.modes()
    K1 = s.K + 1
    mode_v = [s.bath_mask[l // K1] for l in range(m.M)]
    bath_terms = [(md["delta"][b], s.bath_mask[b]) for b in range(len(s.bath_state))]
    # H(t) written out here from the pulse definition
    x = (t_eval - pulse.t_center_fs) / pulse.sigma_fs
    gt = pulse.amp_cm * np.exp(-0.5 * x * x) * np.exp(-1j * (25.0 * TWO_PI_C * t_eval + 0.3))
    Ht = (np.asarray(s.H) - gt * pulse.mu_plus - np.conj(gt) * pulse.mu_plus.T) * TWO_PI_C
    L, tuples, index = build_general(Ht, mode_v, md["gamma"], md["c"], md["lamnu"], bath_terms, s.D,
                                     terminator=terminator)
    t, _, _ = m.hierarchy()
    rng = np.random.default_rng(3)
    re, im = rng.standard_normal((m.n_ado, m.N, m.N)), rng.standard_normal((m.n_ado, m.N, m.N))
    ore, oim = m.rhs(re, im)
    ref = from_vec(L @ to_vec(re, im, t, index), t, index, m.N)
    assert np.max(np.abs((ore + 1j * oim) - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the sandwich part of the terminator matters here: pairs sharing a site
    if terminator:
        assert any(s.bath_mask[b].sum() > 1 for b in range(len(s.bath_state)))

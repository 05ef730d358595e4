"""Pins of the oracle's Pade bath decomposition (section "HEOM formalism": the Pade expansion that
replaces the Matsubara frequencies), checked against what the mathematics fixes, not against the
oracle's own formulas:

  * K = 1 closed form: the [0/1] Pade approximant of g(y) = (f(x) - 1/x - 1/2) / x, y = x^2,
    f = 1/(1 - e^-x), is (1/12) / (1 + y/60): xi^2 = 60, eta = 5/2;
  * the defining property of the [K-1/K] approximant: sum_i 2 eta_i / (y + xi_i^2) reproduces the
    first 2K Taylor coefficients of g(y), which are B_{2m+2} / (2m+2)! (Bernoulli numbers, exact
    rationals computed here by their recurrence);
  * convergence to the exact Bose function (numpy exp) as K grows;
  * for t >= 10 fs the Pade correlation function sum_k c_k exp(-gamma_k t) of a Drude-Lorentz bath
    converges to the exact one (the Matsubara series summed to convergence, an independent route) as
    K grows, and beats the Matsubara series truncated at the same K;
  * the product's host-side modes (heom_bath_modes, eigenvalues by Sturm bisection) equal the
    oracle's (dense Jacobi rotations) to rounding;
  * the oracle's Pade right-hand side equals the dense Liouvillian built from its exported modes.
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

from liouvillian import build_from_oracle, from_vec, to_vec
from oracle.oracle import Bath, OracleModel, pade

KB_RAD = 1.8836515673088532e-4 * 0.6950348004  # k_B in rad/fs per K


def bernoulli(n):
    """B_0..B_n as exact fractions (B_1 = -1/2 convention), from sum_k C(m+1, k) B_k = 0."""
    B = [Fraction(1)]
    for m in range(1, n + 1):
        B.append(-sum(comb(m + 1, k) * B[k] for k in range(m)) / (m + 1))
    return B


def test_pade_k1_closed_form():
    xi, eta = pade(1)
    assert abs(xi[0] ** 2 - 60.0) <= 1e-12 * 60
    assert abs(eta[0] - 2.5) <= 1e-13


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6])
def test_pade_matches_taylor_coefficients(K):
    """(f(x) - 1/x - 1/2)/x = sum_m B_{2m+2}/(2m+2)! y^m; the approximant's expansion in y = x^2 is
    sum_m (-1)^m (sum_i 2 eta_i / xi_i^(2m+2)) y^m.  A [K-1/K] Pade approximant in y matches 2K terms."""
    xi, eta = pade(K)
    B = bernoulli(4 * K + 2)
    for m in range(2 * K):
        exact = float(B[2 * m + 2] / factorial(2 * m + 2))
        approx = (-1) ** m * float(np.sum(2 * eta / xi ** (2 * m + 2)))
        assert abs(approx - exact) <= 1e-9 * abs(exact), (K, m, approx, exact)
    # and not the next one (the approximant is not the function; its mismatch there shrinks fast
    # with K, so check it where it is well above rounding)
    if K <= 4:
        m = 2 * K
        exact = float(B[2 * m + 2] / factorial(2 * m + 2))
        approx = (-1) ** m * float(np.sum(2 * eta / xi ** (2 * m + 2)))
        assert abs(approx - exact) > 1e-9 * abs(exact)


def test_pade_converges_to_bose_function():
    x = np.linspace(0.01, 30.0, 3000)
    exact = 1.0 / (1.0 - np.exp(-x))
    errs = []
    for K in (1, 2, 3, 4, 6, 8):
        xi, eta = pade(K)
        approx = 1.0 / x + 0.5 + np.sum(2 * eta[:, None] * x / (x ** 2 + xi[:, None] ** 2), axis=0)
        errs.append(np.max(np.abs(approx - exact) / exact))
        assert np.all(eta > 0) and np.all(np.diff(xi) > 0)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6


def corr(model, t):
    m = model.modes()
    return np.sum(m["c"][:, None] * np.exp(-m["gamma"][:, None] * t), axis=0)


def test_pade_correlation_converges_to_exact():
    lam, tau, T = 35.0, 50.0, 77.0
    H = np.zeros((1, 1))
    # t >= 10 fs: at shorter times the 1/omega tail of the Drude density needs many exponentials with
    # either expansion at 77 K
    t = np.linspace(10.0, 200.0, 100)
    # exact Re C(t): the Matsubara series summed to convergence (20000 terms)
    lam_r = 1.8836515673088532e-4 * lam
    nu = 1.0 / tau
    beta = 1.0 / (KB_RAD * T)
    exact = lam_r * nu / np.tan(beta * nu / 2) * np.exp(-nu * t)
    k = np.arange(1, 20001)[:, None]
    g = 2 * np.pi * k / beta
    exact = exact + np.sum(4 * lam_r * nu / beta * g / (g ** 2 - nu ** 2) * np.exp(-g * t), axis=0)
    err_p, err_m = [], []
    for K in (1, 2, 3, 4, 6):
        mp = OracleModel(H, [Bath(0, lam, tau, T)], K=K, D=0, decomposition="pade")
        mm = OracleModel(H, [Bath(0, lam, tau, T)], K=K, D=0)
        err_p.append(np.max(np.abs(corr(mp, t) - exact)) / np.max(np.abs(exact)))
        err_m.append(np.max(np.abs(corr(mm, t) - exact)) / np.max(np.abs(exact)))
    assert all(b < a for a, b in zip(err_p, err_p[1:]))
    assert all(p < m for p, m in zip(err_p, err_m))
    assert err_p[-1] < 5e-4


def test_product_modes_equal_oracle_modes():
    from helpers import oracle_for
    from paper_1803_03498_gb300 import heom
    from paper_1803_03498_gb300 import workloads as wl
    pop, _ = wl.fmo_like()
    s = pop.system
    for K in (0, 1, 3, 6):
        s.K, s.decomposition = K, "pade"
        g = heom.bath_modes(s)
        o = oracle_for(s).modes()
        for key in ("gamma", "c", "lamnu"):
            assert np.allclose(g[key], o[key], rtol=1e-13, atol=0), (K, key)
        tb = np.zeros(s.N)
        for b, st in enumerate(s.bath_state):
            tb[st] += o["delta"][b]
        assert np.allclose(g["term"], tb, rtol=1e-12, atol=1e-20)


def test_pade_model_rhs_equals_dense_liouvillian():
    """The right-hand side with Pade modes is the same superoperator with other coefficients: the
    oracle's RHS of a random state equals the dense Liouvillian built from its exported modes."""
    H = np.array([[0.0, 50.0], [50.0, 100.0]])
    m = OracleModel(H, [Bath(0, 35.0, 50.0, 77.0), Bath(1, 35.0, 50.0, 77.0)], K=2, D=2, decomposition="pade")
    L, tuples, index = build_from_oracle(m)
    t, _, _ = m.hierarchy()
    rng = np.random.default_rng(11)
    re, im = rng.standard_normal((m.n_ado, 2, 2)), rng.standard_normal((m.n_ado, 2, 2))
    ore, oim = m.rhs(re, im)
    ref = from_vec(L @ to_vec(re, im, t, index), t, index, m.N)
    assert np.max(np.abs((ore + 1j * oim) - ref)) <= 1e-13 * np.max(np.abs(ref))

"""Pins of the oracle's bath coefficients (Matsubara gamma(b,k), c(b,k) and the terminator of
Eq. HEOM, section "HEOM formalism") against closed forms that do not restate the definitions:

* the units: beta in fs equals hbar / (k_B T) with SI hbar and k_B;
* the Matsubara sum rule sum_{k>=0} c_k / gamma_k = 2 lambda / (beta nu) (the partial-fraction
  expansion of cot), so the terminator of K terms vanishes like lambda nu beta / (pi^2 K);
* the high-temperature limit c_0 -> 2 lambda / beta when beta nu -> 0;
* gamma_k = nu (Matsubara resonance) is rejected.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Bath, OracleModel

HBAR_SI = 1.054571817e-34   # J s
KB_SI = 1.380649e-23        # J / K
CM_TO_RAD_FS = 2 * math.pi * 2.99792458e-5


def model(lam=35.0, tau=50.0, T=300.0, K=0, D=1, terminator=True):
    H = np.array([[0.0]])
    return OracleModel(H, [Bath(0, lam, tau, T)], K=K, D=D, terminator=terminator)


def test_beta_units():
    for T in (30.0, 77.0, 300.0):
        md = model(T=T, K=1).modes()
        beta_fs = 2 * math.pi / md["gamma"][1]          # gamma_1 = 2 pi / beta
        assert beta_fs == pytest.approx(HBAR_SI / (KB_SI * T) * 1e15, rel=1e-9)


def test_drude_mode():
    md = model(lam=35.0, tau=50.0, T=300.0, K=0).modes()
    assert md["gamma"][0] == pytest.approx(1 / 50.0, rel=1e-15)
    assert md["lamnu"][0] == pytest.approx(35.0 * CM_TO_RAD_FS / 50.0, rel=1e-14)


@pytest.mark.parametrize("T,tau", [(300.0, 50.0), (77.0, 166.0), (30.0, 50.0)])
def test_sum_rule_and_tail(T, tau):
    lam = 35.0
    lam_r = lam * CM_TO_RAD_FS
    nu = 1.0 / tau
    beta = HBAR_SI / (KB_SI * T) * 1e15
    deltas = []
    for K in (0, 1, 4, 16, 200):
        md = model(lam, tau, T, K=K, D=0).modes()
        deltas.append(md["delta"][0])
        # terminator = 2 lambda/(beta nu) - partial sum; all terms positive -> decreasing, positive
    assert all(d > 0 for d in deltas)
    assert all(a > b for a, b in zip(deltas, deltas[1:]))
    # tail of the partial-fraction series: sum_{k>K} 4 lam nu beta / (4 pi^2 k^2 - beta^2 nu^2)
    K = 200
    tail = sum(4 * lam_r * nu * beta / (4 * math.pi ** 2 * k ** 2 - beta ** 2 * nu ** 2) for k in range(K + 1, 200000))
    tail += lam_r * nu * beta / (math.pi ** 2 * 200000)  # integral estimate of the remainder
    assert deltas[-1] == pytest.approx(tail, rel=1e-4)
    assert deltas[-1] * (K + 0.5) == pytest.approx(lam_r * nu * beta / math.pi ** 2, rel=1e-3)


def test_high_temperature_limit():
    lam_r = 35.0 * CM_TO_RAD_FS
    for T in (3000.0, 30000.0):
        beta = HBAR_SI / (KB_SI * T) * 1e15
        nu = 1 / 50.0
        c0 = model(T=T).modes()["c"][0]
        x = beta * nu
        assert c0 == pytest.approx(2 * lam_r / beta, rel=x * x / 12 * 1.1 + 1e-12)
        assert abs(c0 / (2 * lam_r / beta) - 1) > 0  # not identically the limit


def test_resonance_rejected():
    # choose T so that gamma_1 = 2 pi / beta equals nu = 1/tau
    tau = 50.0
    beta = 2 * math.pi * tau
    T = HBAR_SI / (KB_SI * beta * 1e-15)
    with pytest.raises(ValueError):
        model(tau=tau, T=T, K=1)

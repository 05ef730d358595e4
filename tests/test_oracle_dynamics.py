"""Pins of the oracle's right-hand side (Eq. HEOM with the rescaling) and its classic RK4.

(i)   one RHS call equals the dense Kronecker Liouvillian times the state; n RK4 steps equal the
      degree-4 Taylor polynomial of h L to the n-th power; RK4 converges to expm(tL) at order 4;
(ii)  lambda = 0 reduces to unitary evolution exp(-iHt) (and the dipole correlation to
      d^T exp(-i H_e t) d);
(iii) trace of sigma_0 is conserved and every ADO stays Hermitian in the paper's gauge;
(iv)  a dimer relaxes to the null vector of L, close to the Boltzmann populations of H;
gauge: the paper's form (up +iV^x, down n(icV^x + lambda nu V^o), rescaled) and the textbook
      form (up -iV^x, down -in(c~ V . - c~* . V) with complex c~_0) give the same sigma_0.
Mutation checks plant plausible mistakes in the dense Liouvillian (which the RHS test ties to the
oracle) and show that the physics pins reject them.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import liouvillian as lv
from oracle.oracle import Bath, OracleModel
from paper_1803_03498_gb300 import workloads as wl

CM = 1.8836515673088532e-4


def dimer_model(**kw):
    p = wl.dimer()
    s = p.system
    baths = [Bath(st, l, t, T) for st, l, t, T in zip(s.bath_state, s.lambda_cm, s.tau_fs, s.T_K)]
    args = dict(K=s.K, D=s.D)
    args.update(kw)
    return OracleModel(s.H, baths, **args), p


def ground_model(K=1, D=3, rescale=True, terminator=True):
    """3 states: 0 = ground (no bath), sites 1, 2; complex Hermitian H."""
    H = np.array([[0.0, 0, 0], [0, 80.0, 40.0 + 15.0j], [0, 40.0 - 15.0j, 0.0]])
    baths = [Bath(1, 35.0, 50.0, 300.0), Bath(2, 60.0, 100.0, 300.0)]
    return OracleModel(H, baths, K=K, D=D, rescale=rescale, terminator=terminator)


def shared_state_model():
    """Two baths on state 0 and one on state 1 (several baths per site)."""
    H = np.array([[0.0, 30.0], [30.0, 150.0]])
    baths = [Bath(0, 20.0, 60.0, 200.0), Bath(0, 50.0, 120.0, 200.0), Bath(1, 35.0, 50.0, 200.0)]
    return OracleModel(H, baths, K=0, D=3)


def random_state(m, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m.n_ado, m.N, m.N)), rng.standard_normal((m.n_ado, m.N, m.N))


@pytest.mark.parametrize("builder", [lambda: dimer_model()[0], ground_model, shared_state_model,
                                     lambda: ground_model(rescale=False, terminator=False),
                                     lambda: dimer_model(K=1, D=3)[0]])
def test_rhs_equals_dense_liouvillian(builder):
    m = builder()
    L, tuples, index = lv.build_from_oracle(m)
    t, _, _ = m.hierarchy()
    re, im = random_state(m, 7)
    ore, oim = m.rhs(re, im)
    ref = lv.from_vec(L @ lv.to_vec(re, im, t, index), t, index, m.N)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs((ore + 1j * oim) - ref)) <= 1e-13 * scale


def taylor4(L, h):
    A = h * L
    I = np.eye(L.shape[0])
    return I + A + A @ A / 2 + A @ A @ A / 6 + A @ A @ A @ A / 24


def start(m, rho_re, rho_im):
    re = np.zeros((m.n_ado, m.N, m.N))
    im = np.zeros_like(re)
    re[0], im[0] = rho_re, rho_im
    return re, im


def test_rk4_is_taylor_polynomial():
    m, p = dimer_model()
    L, tuples, index = lv.build_from_oracle(m)
    t, _, _ = m.hierarchy()
    re, im = start(m, p.rho0_re, p.rho0_im)
    v = lv.to_vec(re, im, t, index)
    n = 200
    m.rk4(re, im, p.dt_fs, n, obs_stride=n)
    P = np.linalg.matrix_power(taylor4(L, p.dt_fs), n)
    ref = lv.from_vec(P @ v, t, index, m.N)
    assert np.max(np.abs((re + 1j * im) - ref)) <= 1e-12


def test_rk4_fourth_order():
    m = ground_model(K=0, D=3)
    L, tuples, index = lv.build_from_oracle(m)
    t, _, _ = m.hierarchy()
    rho = np.zeros((3, 3)); rho[1, 1] = 1.0
    T = 200.0
    exact = lv.from_vec(sla.expm(T * L) @ lv.to_vec(*start(m, rho, 0 * rho), t, index), t, index, m.N)[0]
    errs = []
    for dt in (4.0, 2.0, 1.0):
        re, im = start(m, rho, 0 * rho)
        m.rk4(re, im, dt, int(round(T / dt)), obs_stride=1000000)
        errs.append(np.max(np.abs(re[0] + 1j * im[0] - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, (errs, r1, r2)


@pytest.mark.parametrize("make", [lambda: dimer_model(K=1, D=3)[0], lambda: ground_model(K=1, D=3)])
def test_gauge_textbook_form(make):
    m = make()
    Lp, tp_, ip = lv.build_from_oracle(m, form="paper")
    Lc, tc_, ic = lv.build_from_oracle(m, form="common", rescale=False)
    N = m.N
    rho = np.zeros((N, N), complex); rho[N - 1, N - 1] = 1.0
    rho[N - 1, 0] = 0.3
    for T in (20.0, 150.0):
        vp = np.zeros(Lp.shape[0], complex); vp[ip[tuple([0] * m.M)] * N * N:][:N * N] = rho.reshape(-1)
        vc = np.zeros(Lc.shape[0], complex); vc[ic[tuple([0] * m.M)] * N * N:][:N * N] = rho.reshape(-1)
        sp = (sla.expm(T * Lp) @ vp)[ip[tuple([0] * m.M)] * N * N:][:N * N]
        sc = (sla.expm(T * Lc) @ vc)[ic[tuple([0] * m.M)] * N * N:][:N * N]
        assert np.max(np.abs(sp - sc)) <= 1e-12


def test_rescaling_is_a_gauge():
    a = ground_model(rescale=True)
    b = ground_model(rescale=False)
    rho = np.zeros((3, 3)); rho[2, 2] = 1.0; rho[1, 0] = 0.5
    ra, ia = start(a, rho, 0 * rho)
    rb, ib = start(b, rho, 0 * rho)
    a.rk4(ra, ia, 0.5, 400, obs_stride=400)
    b.rk4(rb, ib, 0.5, 400, obs_stride=400)
    assert np.max(np.abs((ra[0] - rb[0]) + 1j * (ia[0] - ib[0]))) <= 1e-13


def test_unitary_limit():
    H = np.array([[0.0, 0, 0], [0, 100.0, 45.0], [0, 45.0, -20.0]])
    m = OracleModel(H, [Bath(1, 0.0, 50.0, 300.0), Bath(2, 0.0, 70.0, 300.0)], K=1, D=3)
    w = np.array([0.0, 0.8, -0.6])
    rho = np.zeros((3, 3)); rho[:, 0] = w
    re, im = start(m, rho, 0 * rho)
    dt, n = 0.25, 4000
    obs = m.rk4(re, im, dt, n, obs_stride=n // 4, w=w)
    E, U = np.linalg.eigh(H * CM)
    assert np.max(np.abs(re[1:])) == 0 and np.max(np.abs(im[1:])) == 0   # ADOs never fed
    for r, t in enumerate(np.arange(0, n + 1, n // 4) * dt):
        Ut = U @ np.diag(np.exp(-1j * E * t)) @ U.conj().T
        corr = w @ Ut @ w
        # RK4 phase error per step ~ (omega h)^5 / 120
        tol = (np.max(np.abs(E)) * dt) ** 5 / 120 * (t / dt) * 2 + 1e-13
        assert abs(obs[r, 5] + 1j * obs[r, 6] - corr) <= tol
    sig = Ut @ rho @ Ut.conj().T
    assert np.max(np.abs(re[0] + 1j * im[0] - sig)) <= tol


def test_trace_and_hermiticity_population_run():
    pop, _ = wl.fmo_like()
    s = pop.system
    m = OracleModel(s.H, [Bath(st, l, t, T) for st, l, t, T in zip(s.bath_state, s.lambda_cm, s.tau_fs, s.T_K)],
                    K=0, D=2)
    re, im = start(m, pop.rho0_re, pop.rho0_im)
    obs = m.rk4(re, im, pop.dt_fs, 400, obs_stride=50)
    assert np.max(np.abs(obs[:, m.N] - 1.0)) <= 1e-13
    assert np.max(np.abs(obs[:, m.N + 1])) <= 1e-13
    sig = re + 1j * im
    herm = np.max(np.abs(sig - np.conj(np.transpose(sig, (0, 2, 1)))))
    assert herm <= 1e-13
    assert np.max(np.abs(sig[1:])) > 1e-4     # the ADOs are populated


def null_state(L, index, M, N):
    w, V = np.linalg.eig(L)
    k = np.argmin(np.abs(w))
    v = V[:, k]
    root = index[tuple([0] * M)]
    rho = v[root * N * N:(root + 1) * N * N].reshape(N, N)
    return rho / np.trace(rho), np.sort(np.abs(w))[:2]


def boltzmann_sites(H, T):
    E, U = np.linalg.eigh(H)
    p = np.exp(-(E - E.min()) / (0.6950348004 * T))
    p /= p.sum()
    return np.real(np.diag(U @ np.diag(p) @ U.T))


def test_thermal_relaxation_dimer():
    m, p = dimer_model()
    L, tuples, index = lv.build_from_oracle(m)
    rho_inf, evs = null_state(L, index, m.M, m.N)
    assert evs[0] < 1e-12 < evs[1]
    re, im = start(m, p.rho0_re, p.rho0_im)
    m.rk4(re, im, 1.0, 20000, obs_stride=20000)
    assert np.max(np.abs(re[0] + 1j * im[0] - rho_inf)) <= 1e-6
    pb = boltzmann_sites(p.system.H, 300.0)
    assert pb == pytest.approx([0.6155, 0.3845], abs=5e-4)
    assert np.real(np.diag(rho_inf)) == pytest.approx(pb, abs=0.03)


# --- planted mistakes: each one must be caught by a physics pin --------------------------------

def _mutant(m, kind):
    md = m.modes()
    N = m.N
    H = np.asarray(m.H, complex) * CM
    delta = np.zeros(N)
    for b, bath in enumerate(m.baths):
        delta[bath.state] += md["delta"][b]
    c, ln = md["c"].copy(), md["lamnu"].copy()
    if kind == "lamnu_sign":
        ln = -ln
    elif kind == "c_sign":
        c = -c
    elif kind == "no_terminator_factor2":
        delta = 2 * delta
    return lv.build(H, md["state"], md["gamma"], c, ln, delta, m.D, terminator=True, rescale=True)


@pytest.mark.parametrize("kind", ["lamnu_sign", "c_sign"])
def test_planted_mistakes_break_detailed_balance(kind):
    m, p = dimer_model()
    L, tuples, index = _mutant(m, kind)
    rho_inf, _ = null_state(L, index, m.M, m.N)
    pb = boltzmann_sites(p.system.H, 300.0)
    bad = np.max(np.abs(np.real(np.diag(rho_inf)) - pb)) > 0.03 or np.max(np.abs(rho_inf - rho_inf.conj().T)) > 1e-6
    assert bad


def test_planted_terminator_mistake_breaks_gauge_and_rhs():
    m = ground_model(K=0, D=2)
    L_good, tuples, index = lv.build_from_oracle(m)
    L_bad, _, _ = _mutant(m, "no_terminator_factor2")
    t, _, _ = m.hierarchy()
    re, im = random_state(m, 3)
    ore, oim = m.rhs(re, im)
    v = lv.to_vec(re, im, t, index)
    ref_bad = lv.from_vec(L_bad @ v, t, index, m.N)
    assert np.max(np.abs(ore + 1j * oim - ref_bad)) > 1e-6

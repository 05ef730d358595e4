"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle on the same seeded
inputs.  FP64: max |difference| <= 1e-12 on every element of every ADO.  FP32-mixed: max
population error <= 1e-6 (the precision target), with the element-wise error reported.

Sizes: the dimer (15 ADOs, full 2000 steps), the FMO-like system (3060 ADOs of 7x7 and 8x8: several
CTA chunks and a ragged tail) over 40 steps with the full state compared, edge cases (one state, depth
0, no Matsubara term, complex H, unbathed ground state, several baths on one state, rescaling and
terminator off) and, at the LHCII-like size (1,344,904 ADOs of 14x14, the benchmark's launch
configuration), one right-hand-side evaluation of a random state on sampled ADOs.
"""
import numpy as np
import pytest

from helpers import gpu_run, oracle_for, oracle_propagate, oracle_start
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
POP_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_03498_gb300.build import build
    build()


def full_state(r):
    re, im = r.get_ados(0, r.n_ado)
    return re + 1j * im


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_dimer_full_run(precision):
    p = wl.dimer()
    m, ore, oim, oobs = oracle_propagate(p, p.n_steps, stride=1)
    r, gobs = gpu_run(p, precision, stride=1)
    assert gobs.shape[0] == p.n_steps + 1
    N = p.system.N
    pop_err = np.max(np.abs(gobs[:, :N] - oobs[:, :N]))
    if precision == "fp64":
        assert np.max(np.abs(full_state(r) - (ore + 1j * oim))) <= FP64_TOL
        assert pop_err <= FP64_TOL
        assert np.max(np.abs(gobs[:, N:N + 4] - oobs[:, N:N + 4])) <= FP64_TOL
    else:
        assert pop_err <= POP_TOL
    assert np.max(np.abs(gobs[:, N] - 1.0)) <= (1e-13 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("which", ["pop", "dip0", "dip2"])
def test_fmo_like_full_state(precision, which):
    pop, dips = wl.fmo_like()
    p = {"pop": pop, "dip0": dips[0], "dip2": dips[2]}[which]
    steps = 40
    m, ore, oim, oobs = oracle_propagate(p, steps, stride=4)
    r, gobs = gpu_run(p, precision, n_steps=steps, stride=4)
    N = p.system.N
    ref = ore + 1j * oim
    err = np.max(np.abs(full_state(r) - ref))
    if precision == "fp64":
        assert err <= FP64_TOL, err
        assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= FP64_TOL
    else:
        assert np.max(np.abs(gobs[:, :N] - oobs[:, :N])) <= POP_TOL
        assert np.max(np.abs(gobs[:, N + 2:N + 4] - oobs[:, N + 2:N + 4])) <= 1e-5
        assert err <= 1e-4 * max(1.0, np.max(np.abs(ref)))


def _edge_cases():
    H2 = np.array([[0.0, 50.0], [50.0, 100.0]])
    Hc = np.array([[0.0, 0, 0], [0, 80.0, 40.0 + 15.0j], [0, 40.0 - 15.0j, 0.0]])
    out = {}
    s = wl.System("one state", np.array([[10.0]]), [0], [35.0], [50.0], [300.0], K=1, D=3)
    out["one-state"] = wl.Propagation(s, np.array([[1.0]]), np.zeros((1, 1)), 1.0, 60)
    s = wl.System("depth 0", H2, [0, 1], [35.0] * 2, [50.0] * 2, [300.0] * 2, K=1, D=0)
    out["depth0"] = wl.Propagation(s, np.diag([1.0, 0.0]), np.zeros((2, 2)), 1.0, 60)
    s = wl.System("K=2", H2, [0, 1], [35.0] * 2, [50.0] * 2, [300.0] * 2, K=2, D=3)
    out["K2"] = wl.Propagation(s, np.diag([1.0, 0.0]), np.zeros((2, 2)), 0.5, 80)
    s = wl.System("complex H + ground", Hc, [1, 2], [35.0, 60.0], [50.0, 100.0], [300.0, 300.0], K=1, D=3)
    rho = np.zeros((3, 3)); rho[2, 2] = 1.0; rho[1, 0] = 0.5
    out["complexH-ground"] = wl.Propagation(s, rho, np.zeros((3, 3)), 0.5, 80, w=np.array([0.0, 0.6, 0.8]))
    s = wl.System("shared state", np.array([[0.0, 30.0], [30.0, 150.0]]), [0, 0, 1], [20.0, 50.0, 35.0],
                  [60.0, 120.0, 50.0], [200.0] * 3, K=0, D=3)
    out["shared-state"] = wl.Propagation(s, np.diag([0.0, 1.0]), np.zeros((2, 2)), 1.0, 80)
    rng = np.random.default_rng(11)
    H5 = rng.normal(0, 60, (5, 5)); H5 = H5 + H5.T
    s = wl.System("N=5 ragged", H5, list(range(5)), [40.0] * 5, [80.0] * 5, [150.0] * 5, K=1, D=3)
    out["N5-ragged"] = wl.Propagation(s, np.diag([1.0, 0, 0, 0, 0]), np.zeros((5, 5)), 0.5, 40)
    H24 = rng.normal(0, 30, (24, 24)); H24 = H24 + H24.T
    s = wl.System("N=24", H24, list(range(24)), [35.0] * 24, [50.0] * 24, [300.0] * 24, K=0, D=1)
    rho = np.zeros((24, 24)); rho[3, 3] = 1.0
    out["N24"] = wl.Propagation(s, rho, np.zeros((24, 24)), 1.0, 30)
    H17 = rng.normal(0, 30, (17, 17)); H17 = H17 + H17.T
    s = wl.System("N=17", H17, list(range(1, 17)), [35.0] * 16, [70.0] * 16, [77.0] * 16, K=1, D=2)
    rho = np.zeros((17, 17)); rho[:, 0] = rng.normal(size=17); rho[0, 0] = 0
    out["N17-dipole"] = wl.Propagation(s, rho, np.zeros((17, 17)), 0.5, 30, w=rho[:, 0].copy())
    return out


EDGE = _edge_cases()


@pytest.mark.parametrize("name", list(EDGE))
@pytest.mark.parametrize("flags", [(True, True), (False, False)])
def test_edge_cases_fp64(name, flags):
    p = EDGE[name]
    term, resc = flags
    m, ore, oim, oobs = oracle_propagate(p, p.n_steps, stride=5, terminator=term, rescale=resc)
    r, gobs = gpu_run(p, "fp64", stride=5, terminator=term, rescale=resc)
    err = np.max(np.abs(full_state(r) - (ore + 1j * oim)))
    assert err <= FP64_TOL * max(1.0, np.max(np.abs(ore + 1j * oim))), err
    N = p.system.N
    assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= FP64_TOL


@pytest.mark.parametrize("name", ["complexH-ground", "N5-ragged", "N24", "N17-dipole"])
def test_edge_cases_mixed(name):
    p = EDGE[name]
    m, ore, oim, oobs = oracle_propagate(p, p.n_steps, stride=5)
    r, gobs = gpu_run(p, "fp32_mixed", stride=5)
    N = p.system.N
    assert np.max(np.abs(gobs[:, :N] - oobs[:, :N])) <= POP_TOL


def test_rhs_eval_small_random_state():
    """One RHS evaluation of a dense random state, every ADO, FP64."""
    pop, dips = wl.fmo_like()
    p = dips[1]
    m = oracle_for(p.system)
    re, im = wl.random_state(m.n_ado, m.N, seed=5)
    ore, oim = m.rhs(re, im)
    from paper_1803_03498_gb300 import heom
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision="fp64", w=p.w, max_records=2)
    r.set_ados(0, re, im)
    gre, gim = r.rhs_eval(0, m.n_ado)
    scale = np.max(np.abs(ore + 1j * oim))
    assert np.max(np.abs((gre - ore) + 1j * (gim - oim))) <= 1e-14 * scale * 10
    # the state itself is untouched
    sre, sim = r.get_ados(0, m.n_ado)
    assert np.array_equal(sre, re) and np.array_equal(sim, im)


def hermitian(re, im):
    """Hermitian part of every tile: (A + A^dagger) / 2."""
    return 0.5 * (re + np.transpose(re, (0, 2, 1))), 0.5 * (im - np.transpose(im, (0, 2, 1)))


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_rhs_eval_hermitian_random_state(precision):
    """A dense random Hermitian state takes the Hermitian kernels (row-only gathers, s H = (H s)^dagger);
    every ADO of one RHS evaluation against the oracle's general formula."""
    pop, dips = wl.fmo_like()
    m = oracle_for(pop.system)
    re, im = hermitian(*wl.random_state(m.n_ado, m.N, seed=15))
    from paper_1803_03498_gb300 import heom
    r = heom.Run(pop.system, pop.rho0_re, pop.rho0_im, precision=precision, max_records=2)
    r.set_ados(0, re, im)
    if precision == "fp32_mixed":
        re, im = r.get_ados(0, m.n_ado)
    ore, oim = m.rhs(re, im)
    gre, gim = r.rhs_eval(0, m.n_ado)
    scale = np.max(np.abs(ore + 1j * oim))
    tol = 1e-14 * scale * 10 if precision == "fp64" else 2e-5 * scale
    assert np.max(np.abs((gre - ore) + 1j * (gim - oim))) <= tol
    # the result is exactly Hermitian
    g = gre + 1j * gim
    assert np.array_equal(g, np.conj(np.transpose(g, (0, 2, 1))))


def sample_ados(level_offsets, n_ado, rng, n_random=300):
    us = set()
    for off in level_offsets[:-1]:
        for d in (0, 1, 2):
            if 0 <= off + d < n_ado:
                us.add(int(off + d))
            if 0 <= off - 1 - d < n_ado:
                us.add(int(off - 1 - d))
    us.update(int(x) for x in rng.integers(0, n_ado, n_random))
    us.add(n_ado - 1)
    return np.array(sorted(us), dtype=np.int64)


@pytest.mark.parametrize("herm", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_lhcii_full_size_rhs_sampled(precision, herm):
    """Full LHCII-like hierarchy (1,344,904 ADOs of 14 x 14): one RHS evaluation of a dense random
    state with the benchmark's kernels and launch configuration, checked on sampled ADOs (every
    level boundary and 300 random ADOs) against the oracle's per-ADO right-hand side."""
    from paper_1803_03498_gb300 import heom
    p = wl.lhcii_like()
    m = oracle_for(p.system)
    re, im = wl.random_state(m.n_ado, m.N, seed=9, scale=0.1)
    if herm:
        re, im = hermitian(re, im)
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision=precision, max_records=2)
    r.set_ados(0, re, im)
    if precision == "fp32_mixed":
        # the oracle sees the same (rounded) state the GPU holds
        gre, gim = r.get_ados(0, m.n_ado)
        re, im = gre, gim
    us = sample_ados(r.hier.level_offsets, m.n_ado, np.random.default_rng(3))
    ore, oim = m.rhs_list(us, re, im)
    gre, gim = r.rhs_eval(0, m.n_ado)
    ref = ore + 1j * oim
    err = np.max(np.abs(gre[us] + 1j * gim[us] - ref))
    scale = np.max(np.abs(ref))
    if precision == "fp64":
        assert err <= 1e-13 * scale * 10, (err, scale)
    else:
        assert err <= 2e-5 * scale, (err, scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_lhcii_invariants_few_steps(precision):
    """A few RK4 steps at full size: trace of sigma_0 stays 1 and sigma_0 stays Hermitian (paper
    gauge, population run); the FP64 and mixed runs agree on the populations."""
    p = wl.lhcii_like(n_steps=3)
    r, obs = gpu_run(p, precision, stride=1)
    N = p.system.N
    assert np.max(np.abs(obs[:, N] - 1.0)) <= (1e-13 if precision == "fp64" else 1e-6)
    assert np.max(np.abs(obs[:, N + 1])) <= (1e-13 if precision == "fp64" else 1e-6)
    assert np.max(obs[:, N + 4]) <= (1e-13 if precision == "fp64" else 1e-6)
    assert obs[-1, 0] < 1.0 - 1e-4  # population moved


def test_state_roundtrip_and_errors():
    from paper_1803_03498_gb300 import heom
    pop, dips = wl.fmo_like()
    p = dips[0]
    for prec in ("fp64", "fp32_mixed"):
        r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision=prec, w=p.w, max_records=3)
        re, im = wl.random_state(r.n_ado, r.N, seed=1)
        r.set_ados(0, re, im)
        gre, gim = r.get_ados(0, r.n_ado)
        if prec == "fp64":
            assert np.array_equal(gre, re) and np.array_equal(gim, im)
        else:
            split = 1 + p.system.n_modes
            assert np.array_equal(gre[:split], re[:split])
            assert np.array_equal(gre[split:], re[split:].astype(np.float32).astype(np.float64))
        with pytest.raises(heom.HeomError) as ei:
            r.propagate(p.dt_fs, 10, 2)   # 5 more records but room for 2
        assert ei.value.code == heom.HEOM_E_NOMEM
        with pytest.raises(heom.HeomError) as ei:
            r.propagate(50.0, 1, 0)       # dt far above 1/gamma
        assert ei.value.code == heom.HEOM_E_ARG
        with pytest.raises(heom.HeomError):
            r.get_ados(r.n_ado - 1, 2)


@pytest.mark.parametrize("N,K,D", [(8, 1, 3), (9, 0, 4), (11, 1, 2), (13, 0, 3), (16, 1, 2)])
def test_column_kernel_sizes_fp64(N, K, D):
    """FP64 Hermitian runs with 8 <= N <= 16 take the column-form stage kernel (every lane owns one
    column of one part of an ADO's result).  Seeded symmetric H, one bath per site, population run from
    the first site: every element of every ADO after 30 steps within 1e-12 of the oracle.  The sizes
    give ragged last chunks, ADOs with more links than one record batch (up to 2M up links at the
    root) and one-ADO chunks (N = 16)."""
    rng = np.random.default_rng(1803100 + N)
    H = _sym(rng, N)
    s = wl.System(f"column N={N}", H, list(range(N)), [35.0] * N, [60.0] * N, [300.0] * N, K=K, D=D)
    rho = np.zeros((N, N))
    rho[0, 0] = 1.0
    p = wl.Propagation(s, rho, np.zeros((N, N)), 1.0, 30)
    m, ore, oim, oobs = oracle_propagate(p, p.n_steps, stride=3)
    r, gobs = gpu_run(p, "fp64", stride=3)
    ref = ore + 1j * oim
    assert np.max(np.abs(full_state(r) - ref)) <= FP64_TOL
    assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= FP64_TOL
    assert np.max(np.abs(ref[-1])) > 0  # the deepest ADOs were reached


def _sym(rng, N):
    H = np.diag(rng.uniform(0.0, 400.0, N)) + np.triu(rng.normal(0.0, 40.0, (N, N)), 1)
    return H + np.triu(H, 1).T


@pytest.mark.parametrize("N", [17, 19, 20, 24])
def test_fp32_owner_path_large_n(N):
    """FP32 body kernels for 17 <= N <= 24 (one ADO per warp, N of 32 lanes) on Hermitian runs take the
    owner-lane form: S = s H from each lane's own row, the links added in registers, Q + Q^dagger at
    the end.  K = 0, D = 3 (levels 2 and 3 in the FP32 body, ragged last chunks).  (1) One right-hand
    side of a dense Hermitian random state, every ADO, against the oracle (2e-5 of the largest
    element: FP32 rounding of an N-term sum per element); (2) 30 RK4 steps from the first site on
    populations (1e-6)."""
    from paper_1803_03498_gb300 import heom
    rng = np.random.default_rng(1803200 + N)
    H = _sym(rng, N)
    s = wl.System(f"owner N={N}", H, list(range(N)), [35.0] * N, [60.0] * N, [300.0] * N, K=0, D=3)
    rho = np.zeros((N, N))
    rho[0, 0] = 1.0
    p = wl.Propagation(s, rho, np.zeros((N, N)), 1.0, 30)
    m = oracle_for(s)
    re, im = hermitian(*wl.random_state(m.n_ado, N, seed=N, scale=0.1))
    r = heom.Run(s, p.rho0_re, p.rho0_im, precision="fp32_mixed", max_records=2)
    r.set_ados(0, re, im)
    gre0, gim0 = r.get_ados(0, m.n_ado)  # the state as the GPU holds it (body rounded to FP32)
    ore, oim = m.rhs(gre0, gim0)
    gre, gim = r.rhs_eval(0, m.n_ado)
    ref = ore + 1j * oim
    assert np.max(np.abs(gre + 1j * gim - ref)) <= 2e-5 * np.max(np.abs(ref))
    r.close()
    m2, ore2, oim2, oobs = oracle_propagate(p, p.n_steps, stride=3)
    r2, gobs = gpu_run(p, "fp32_mixed", stride=3)
    assert np.max(np.abs(gobs[:, :N] - oobs[:, :N])) <= POP_TOL
    assert np.max(np.abs(ore2[-1] + 1j * oim2[-1])) > 0  # the deepest ADOs were reached

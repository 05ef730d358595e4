"""The split-TF32 precision: the FP32 body stage of Hermitian runs with real H and N <= 16 computes
the commutator's s H on the tensor cores (tcgen05, TF32 high/low parts, FP32 accumulation).

Checks against the CPU oracle (the oracle sees the same FP32-rounded state the GPU holds):
  * one RHS evaluation of dense random Hermitian states for N = 2..16 (every padding of the 16-wide
    tensor-core tiles, A = floor(32 / N) ADOs per warp), every ADO, within the mixed precision's
    tolerance; the result is exactly Hermitian and differs from the CUDA-core FP32 kernel's (so the
    tensor-core kernel ran), by no more than the TF32 split allows;
  * the full LHCII-like hierarchy (1,344,904 ADOs of 14 x 14) on sampled ADOs;
  * the 4000-step FMO-like population run against the stored oracle trajectory (population error
    <= 1e-6, the mixed precision's target);
  * a non-Hermitian run at this precision is bit-identical to fp32_mixed (same kernel).
"""
import os

import numpy as np
import pytest

from helpers import gpu_run, oracle_for
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def heom():
    from paper_1803_03498_gb300.build import build
    build()
    from paper_1803_03498_gb300 import heom as h
    h.load()
    return h


def hermitian(re, im):
    return 0.5 * (re + np.transpose(re, (0, 2, 1))), 0.5 * (im - np.transpose(im, (0, 2, 1)))


def small_system(N, K, D, seed):
    rng = np.random.default_rng(seed)
    H = np.zeros((N, N))
    H[np.diag_indices(N)] = rng.uniform(12100.0, 12600.0, N)
    iu = np.triu_indices(N, 1)
    H[iu] = rng.normal(0.0, 40.0, len(iu[0]))
    H = H + np.triu(H, 1).T
    lam = list(rng.uniform(20.0, 100.0, N))
    tau = list(rng.uniform(50.0, 200.0, N))
    return wl.System(f"tc N={N}", H, list(range(N)), lam, tau, [300.0] * N, K=K, D=D)


def rhs_of(heom, sysm, precision, re, im):
    rho = np.zeros((sysm.N, sysm.N))
    rho[0, 0] = 1.0
    r = heom.Run(sysm, rho, np.zeros_like(rho), precision=precision, max_records=2)
    r.set_ados(0, re, im)
    sre, sim = r.get_ados(0, sysm.n_ado)
    gre, gim = r.rhs_eval(0, sysm.n_ado)
    r.close()
    return sre, sim, gre, gim


@pytest.mark.parametrize("N,K,D", [(2, 1, 4), (5, 1, 3), (7, 1, 3), (8, 0, 4), (11, 0, 3), (14, 0, 3), (16, 0, 3)])
def test_split_tf32_rhs_hermitian_random_state(heom, N, K, D):
    sysm = small_system(N, K, D, seed=100 + N)
    re, im = hermitian(*wl.random_state(sysm.n_ado, N, seed=200 + N))
    sre, sim, gre, gim = rhs_of(heom, sysm, "split_tf32", re, im)
    m = oracle_for(sysm)
    ore, oim = m.rhs(sre, sim)
    ref = ore + 1j * oim
    scale = np.max(np.abs(ref))
    g = gre + 1j * gim
    assert np.max(np.abs(g - ref)) <= 2e-5 * scale
    assert np.array_equal(g, np.conj(np.transpose(g, (0, 2, 1))))
    # the CUDA-core FP32 kernel on the same state: close, but not the same arithmetic
    _, _, fre, fim = rhs_of(heom, sysm, "fp32_mixed", re, im)
    f = fre + 1j * fim
    d = np.max(np.abs(g - f))
    assert 0 < d <= 2e-5 * scale


def test_split_tf32_lhcii_full_size_rhs_sampled(heom):
    p = wl.lhcii_like()
    m = oracle_for(p.system)
    re, im = hermitian(*wl.random_state(m.n_ado, m.N, seed=9, scale=0.1))
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision="split_tf32", max_records=2)
    r.set_ados(0, re, im)
    re, im = r.get_ados(0, m.n_ado)
    rng = np.random.default_rng(3)
    us = set(int(x) for x in rng.integers(0, m.n_ado, 300))
    for off in r.hier.level_offsets[:-1]:
        us.update(int(x) for x in (off, off + 1, off - 1) if 0 <= x < m.n_ado)
    us.add(m.n_ado - 1)
    us = np.array(sorted(us), dtype=np.int64)
    ore, oim = m.rhs_list(us, re, im)
    gre, gim = r.rhs_eval(0, m.n_ado)
    ref = ore + 1j * oim
    err = np.max(np.abs(gre[us] + 1j * gim[us] - ref))
    assert err <= 2e-5 * np.max(np.abs(ref)), err


def test_split_tf32_fmo_like_4000_steps(heom):
    pop, _ = wl.fmo_like()
    ref = np.loadtxt(os.path.join(GOLDEN, "fmo_like_pop.txt"))
    r, obs = gpu_run(pop, "split_tf32", stride=10)
    N = pop.system.N
    assert obs.shape[0] == ref.shape[0] == pop.n_steps // 10 + 1
    assert np.max(np.abs(obs[:, :N] - ref[:, :N])) <= 1e-6
    assert np.max(np.abs(obs[:, N] - 1.0)) <= 1e-6


def test_split_tf32_non_hermitian_run_is_fp32_mixed(heom):
    _, dips = wl.fmo_like()
    p = dips[0]
    _, a = gpu_run(p, "split_tf32", n_steps=200, stride=10)
    _, b = gpu_run(p, "fp32_mixed", n_steps=200, stride=10)
    assert np.array_equal(a, b)

"""Multi-step parity of the LHCII-like system against the CPU FP64 oracle.

The benchmark propagates the 14-site LHCII-like system (K = 1: 28 modes) at depth 6.  This test runs
the same system at depth 4 (35,960 ADOs of 14 x 14: a persistent grid whose warps stride over many
chunks, ragged last chunk) for 12 RK4 steps of 1 fs through the same kernels the benchmark times:
``stage_kernel<14, double, double>`` for FP64, and for the mixed precision the FP32 body kernel
``stage_kernel<14, float, float>`` with the FP64 head kernel of levels 0 and 1 on the library's side
stream.  The Horner form of RK4 on the GPU is compared with the oracle's classic four-copy tableau
(Eq. HEOM, RK4 of section "HEOM memory and compute requirements").

Two starts:
  * rho(0) = |1><1| (first site): every ADO stays Hermitian, so the GPU takes its Hermitian fast path
    (row-only gathers; in FP32 the owner-lane link form and S = sigma H from the lane's own row);
  * a seeded random non-Hermitian rho(0) (unit trace): the general path (row and column gathers,
    links applied through shared memory).

Bars: FP64 within 1e-12 of the oracle on every element of every ADO after the last step and on every
observable record; mixed precision within 1e-6 on the populations of every record.
"""
import threading

import numpy as np
import pytest

from helpers import gpu_run, oracle_for, oracle_start
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
POP_TOL = 1e-6
STEPS = 12
DEPTH = 4


def _non_hermitian_rho(N, seed=1803014):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    z /= np.trace(z)  # unit trace, not Hermitian
    return np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)


def _case(which):
    p = wl.lhcii_like(n_steps=STEPS)
    p.system.D = DEPTH
    p.system.name = p.system.name.replace("D=6", f"D={DEPTH}")
    if which == "nonherm":
        p.rho0_re, p.rho0_im = _non_hermitian_rho(p.system.N)
    return p


@pytest.fixture(scope="module")
def oracle_runs():
    """Both oracle trajectories, computed in two threads (the ctypes calls release the GIL)."""
    out = {}

    def work(which):
        p = _case(which)
        m = oracle_for(p.system)
        re, im = oracle_start(m, p.rho0_re, p.rho0_im)
        obs = m.rk4(re, im, p.dt_fs, STEPS, obs_stride=1)
        out[which] = (re + 1j * im, obs)

    ts = [threading.Thread(target=work, args=(w,)) for w in ("herm", "nonherm")]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return out


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_03498_gb300.build import build
    build()


@pytest.mark.parametrize("which", ["herm", "nonherm"])
def test_lhcii_family_fp64_every_ado(oracle_runs, which):
    p = _case(which)
    assert p.system.n_ado == 35960
    ref, oobs = oracle_runs[which]
    r, gobs = gpu_run(p, "fp64", stride=1)
    # GPU records carry a Hermiticity column after the oracle's N + 4 values
    assert gobs.shape == (STEPS + 1, p.system.N + 5) and oobs.shape == (STEPS + 1, p.system.N + 4)
    re, im = r.get_ados(0, r.n_ado)
    err = np.max(np.abs(re + 1j * im - ref))
    assert err <= FP64_TOL, err
    N = p.system.N
    assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= FP64_TOL
    # the run really moved: the root ADO and the deepest level changed measurably
    assert np.max(np.abs(ref[0] - (p.rho0_re + 1j * p.rho0_im))) > 1e-3
    assert np.max(np.abs(ref[-1])) > 0
    r.close()


@pytest.mark.parametrize("which", ["herm", "nonherm"])
def test_lhcii_family_mixed_populations(oracle_runs, which):
    p = _case(which)
    ref, oobs = oracle_runs[which]
    r, gobs = gpu_run(p, "fp32_mixed", stride=1)
    N = p.system.N
    pop_err = np.max(np.abs(gobs[:, :N] - oobs[:, :N]))
    assert pop_err <= POP_TOL, pop_err
    # the FP64 root ADO of the mixed run against the oracle (reported scale of the FP32 bulk error)
    s0 = r.sigma0()
    assert np.max(np.abs(s0 - ref[0])) <= 1e-5
    r.close()

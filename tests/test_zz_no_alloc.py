"""heom_propagate_static: the entry point for callers that cannot allocate device memory (code that
runs while its stream is being captured into a CUDA graph, plug-ins whose host application owns
all device allocations, latency-critical paths that cannot take the implicit synchronisation of
cudaMalloc/cudaFree).  Its device workspace is the library's static 32 MiB array, so this test
allocates nothing on the device for those calls either.

Checks, through the C ABI: several calls in a row (different sizes and precisions, so whatever an
earlier call left in the shared array must not leak into the next) give the same records and final
sigma_0 as the allocating path heom_run_create + heom_propagate + heom_observables, within the
tolerance the parity tests use; a run above the 32 MiB limit is rejected with HEOM_E_NOMEM.
"""
import numpy as np
import pytest

from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
POP_TOL = 1e-6


@pytest.fixture(scope="module")
def heom():
    from paper_1803_03498_gb300.build import build
    build()
    from paper_1803_03498_gb300 import heom as h
    h.load()
    return h


def allocating_path(heom, p, precision, steps, stride):
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision=precision, w=p.w, max_records=steps // stride + 1)
    r.propagate(p.dt_fs, steps, stride)
    obs = r.observables()
    s0 = r.sigma0()
    r.close()
    return obs, s0


def static_path(heom, p, precision, steps, stride):
    return heom.propagate_static(p.system, p.rho0_re, p.rho0_im, precision=precision, w=p.w, dt_fs=p.dt_fs,
                                 n_steps=steps, obs_stride=stride)


def test_static_matches_allocating_path_on_consecutive_calls(heom):
    pop, dips = wl.fmo_like()
    cases = [(dips[0], "fp64", 40, 4), (wl.dimer(), "fp32_mixed", 300, 10), (pop, "fp32_mixed", 40, 5),
             (dips[0], "fp64", 40, 4)]
    first = None
    for p, prec, steps, stride in cases:
        ref_obs, ref_s0 = allocating_path(heom, p, prec, steps, stride)
        obs, s0 = static_path(heom, p, prec, steps, stride)
        assert obs.shape == ref_obs.shape == (steps // stride + 1, p.system.N + 5)
        tol = FP64_TOL if prec == "fp64" else POP_TOL
        assert np.max(np.abs(obs - ref_obs)) <= tol
        assert np.max(np.abs(s0 - ref_s0)) <= tol
        if first is None:
            first = (obs, s0)
    # the repeated first case reproduces the first call exactly
    assert np.array_equal(first[0], obs) and np.array_equal(first[1], s0)


def test_static_rejects_runs_above_the_limit(heom):
    p = wl.lhcii_like()
    with pytest.raises(heom.HeomError) as ei:
        static_path(heom, p, "fp32_mixed", 1, 1)
    assert ei.value.code == heom.HEOM_E_NOMEM
    assert "32 MiB" in str(ei.value)

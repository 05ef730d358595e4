"""The Pade bath decomposition on the GPU path: same kernels, other mode coefficients (computed by
the library's own Sturm-bisection eigenvalues; the oracle uses Jacobi rotations).  FP64 runs match
the oracle's classic RK4 to 1e-12 in every ADO; the mixed precision matches the populations to 1e-6.
"""
import copy

import numpy as np
import pytest

from helpers import gpu_run, oracle_propagate
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_03498_gb300.build import build
    build()


def pade_case(which):
    if which == "dimer-K2":
        p = copy.deepcopy(wl.dimer())
        p.system.K, p.system.D, p.system.T_K = 2, 4, [77.0, 77.0]
        p.n_steps = 400
    else:
        pop, dips = wl.fmo_like()
        p = copy.deepcopy(pop if which == "fmo-pop" else dips[1])
        p.n_steps = 300
    p.system.decomposition = "pade"
    return p


@pytest.mark.parametrize("which", ["dimer-K2", "fmo-pop", "fmo-dip1"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_pade_run_matches_oracle(which, precision):
    p = pade_case(which)
    N = p.system.N
    m, ore, oim, oobs = oracle_propagate(p, p.n_steps, stride=10)
    r, gobs = gpu_run(p, precision, stride=10)
    assert gobs.shape[0] == oobs.shape[0]
    if precision == "fp64":
        gre, gim = r.get_ados(0, m.n_ado)
        assert np.max(np.abs((gre - ore) + 1j * (gim - oim))) <= 1e-12
        assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= 1e-12
    else:
        assert np.max(np.abs(gobs[:, :N] - oobs[:, :N])) <= 1e-6
    # the decomposition matters: the Matsubara run differs
    q = copy.deepcopy(p)
    q.system.decomposition = "matsubara"
    _, mobs = gpu_run(q, "fp64", stride=10)
    assert np.max(np.abs(mobs[:, :N + 4] - gobs[:, :N + 4])) > 1e-6

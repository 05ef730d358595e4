"""The coherence-block layout (heom_run_layout 1): linear-absorption runs store and propagate each
ADO as its column 0, because every term of Eq. HEOM keeps ADOs of the form sum_a x_a |a><0| in that
form when state 0 has no bath and H does not couple it to the other states.

  * dipole runs take the column layout, population runs the matrix layout;
  * a dipole run equals the oracle's full-matrix propagation to 1e-12 (FP64) in every element of
    every ADO -- the elements outside column 0 are exactly zero on both sides;
  * uploading data outside the block moves the run to the matrix layout: the state is kept exactly,
    and the propagation continues to agree with the oracle to 1e-12.
"""
import numpy as np
import pytest

from helpers import gpu_run, oracle_for, oracle_start
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def heom():
    from paper_1803_03498_gb300.build import build
    build()
    from paper_1803_03498_gb300 import heom as h
    h.load()
    return h


def test_layout_choice(heom):
    pop, dips = wl.fmo_like()
    r1, _ = gpu_run(dips[0], "fp32_mixed", n_steps=2)
    r2, _ = gpu_run(pop, "fp32_mixed", n_steps=2)
    assert r1.layout() == 1 and r2.layout() == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_column_run_matches_oracle(heom, precision):
    _, dips = wl.fmo_like()
    p = dips[2]
    r, gobs = gpu_run(p, precision, n_steps=200, stride=10)
    assert r.layout() == 1
    m = oracle_for(p.system)
    re, im = oracle_start(m, p.rho0_re, p.rho0_im)
    oobs = m.rk4(re, im, p.dt_fs, 200, obs_stride=10, w=p.w)
    N = p.system.N
    if precision == "fp64":
        gre, gim = r.get_ados(0, m.n_ado)
        assert np.max(np.abs((gre - re) + 1j * (gim - im))) <= 1e-12
        off = np.ones((N, N), bool)
        off[1:, 0] = False
        assert not np.any(gre[:, off]) and not np.any(gim[:, off])
        assert np.max(np.abs(gobs[:, :N + 4] - oobs[:, :N + 4])) <= 1e-12
    else:
        assert np.max(np.abs(gobs[:, N + 2:N + 4] - oobs[:, N + 2:N + 4])) <= 1e-5


def test_leaving_the_column_layout(heom):
    _, dips = wl.fmo_like()
    p = dips[1]
    m = oracle_for(p.system)
    r = heom.Run(p.system, p.rho0_re, p.rho0_im, precision="fp64", w=p.w, max_records=4)
    assert r.layout() == 1
    r.propagate(p.dt_fs, 50, 0)
    re, im = r.get_ados(0, m.n_ado)
    re2, im2 = re.copy(), im.copy()
    re2[3, 1, 2] = 1e-3   # outside column 0
    im2[3, 2, 1] = -2e-3
    r.set_ados(3, re2[3:4], im2[3:4])
    assert r.layout() == 0
    gre, gim = r.get_ados(0, m.n_ado)
    assert np.array_equal(gre, re2) and np.array_equal(gim, im2)
    r.propagate(p.dt_fs, 50, 0)
    gre, gim = r.get_ados(0, m.n_ado)
    ore, oim = re2.copy(), im2.copy()
    m.rk4(ore, oim, p.dt_fs, 50, obs_stride=0, w=p.w)
    assert np.max(np.abs((gre - ore) + 1j * (gim - oim))) <= 1e-12

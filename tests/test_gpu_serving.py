"""The continuous-batching server (paper_1803_03498_gb300.serving): every result is the same alone and
in the mix (bitwise: separate workspaces, deterministic kernels), requests larger than the memory
budget are rejected, and mixed-precision results stay within 1e-6 of the FP64 oracle on populations."""
import numpy as np
import pytest

from helpers import oracle_propagate
from paper_1803_03498_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1803_03498_gb300.build import build
    build()


def small_stream(n=16, rate=200.0):
    return wl.serving_stream(rate, n, seed=77, n_max=8, d_max=4, steps_lo=20, steps_hi=120, max_ado_steps=2e5)


def test_alone_equals_in_mix():
    from paper_1803_03498_gb300.serving import Server
    reqs = small_stream()
    srv = Server(budget_bytes=2e9, quantum=16, max_active=6, obs_stride=4, keep_sigma0=True)
    mix = srv.serve(reqs, real_time=True)
    summ = mix.summary()
    assert summ["completed"] == len(reqs) and summ["rejected"] == 0
    # overlap happened: some request was admitted before an earlier one finished
    res = mix.results
    assert any(b.admitted_s < a.done_s for a in res for b in res if b.rid > a.rid)
    for r in reqs[::3]:
        alone = Server(budget_bytes=2e9, quantum=16, max_active=1, obs_stride=4, keep_sigma0=True).serve([r], False)
        a = alone.results[0]
        m = [x for x in res if x.rid == r.rid][0]
        assert np.array_equal(a.observables, m.observables)
        assert np.array_equal(a.sigma0, m.sigma0)


def test_rejects_above_budget_and_keeps_serving():
    from paper_1803_03498_gb300.serving import Server
    reqs = small_stream(6)
    big = wl.serving_stream(1.0, 1, seed=5, n_max=24, d_max=6, steps_lo=200, steps_hi=200)[0]
    big.rid = 999
    srv = Server(budget_bytes=64e6, quantum=32, max_active=4)
    stats = srv.serve(reqs + [big], real_time=False)
    rej = [r for r in stats.results if r.rejected]
    assert [r.rid for r in rej] == [999] or all(r.workspace_bytes > 64e6 for r in rej)
    assert stats.summary()["completed"] == len(stats.results) - len(rej)


def test_mixed_precision_results_against_oracle():
    from paper_1803_03498_gb300.serving import Server
    reqs = [r for r in small_stream(10) if r.prop.system.n_ado * r.prop.n_steps <= 2e4][:4]
    assert reqs
    stats = Server(budget_bytes=2e9, quantum=25, max_active=4, obs_stride=1).serve(reqs, real_time=False)
    for r, res in zip(reqs, stats.results):
        m, ore, oim, oobs = oracle_propagate(r.prop, r.prop.n_steps, stride=1)
        N = r.prop.system.N
        assert np.max(np.abs(res.observables[:, :N] - oobs[:, :N])) <= 1e-6

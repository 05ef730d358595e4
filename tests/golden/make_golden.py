"""Write the oracle's trajectories of the FMO-like workload to tests/golden/ (text).

Calls only the CPU oracle (oracle/) on inputs from the seeded workload generator; nothing here
touches the CUDA library.  Four runs of 4000 RK4 steps, dt = 0.5 fs, one record every 10 steps:
the population run (7 sites, rho(0) = |1><1|) and the three linear-absorption runs (ground state
+ 7 sites, sigma_0(0) = mu_p^+ |0><0|, p = x, y, z).  Each record: populations, Re/Im trace,
Re/Im dipole correlation.  Runs in parallel processes (spawn); about half an hour on 4 cores.

    python tests/golden/make_golden.py
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
STRIDE = 10


def _run(tag):
    sys.path.insert(0, ROOT)
    from oracle.oracle import Bath, OracleModel
    from paper_1803_03498_gb300 import workloads as wl

    pop, dips = wl.fmo_like()
    p = {"pop": pop, "dip0": dips[0], "dip1": dips[1], "dip2": dips[2]}[tag]
    s = p.system
    m = OracleModel(s.H, [Bath(st, l, t, T) for st, l, t, T in zip(s.bath_state, s.lambda_cm, s.tau_fs, s.T_K)],
                    K=s.K, D=s.D)
    re = np.zeros((m.n_ado, m.N, m.N))
    im = np.zeros_like(re)
    re[0], im[0] = p.rho0_re, p.rho0_im
    t0 = time.time()
    obs = m.rk4(re, im, p.dt_fs, p.n_steps, obs_stride=STRIDE, w=p.w)
    path = os.path.join(HERE, f"fmo_like_{tag}.txt")
    hdr = (f"oracle trajectory, fmo-like {tag}: N={m.N} M={m.M} D={s.D} n_ado={m.n_ado} dt={p.dt_fs} fs "
           f"steps={p.n_steps} stride={STRIDE}; columns: pop[0..N-1], tr_re, tr_im, corr_re, corr_im; "
           f"written by tests/golden/make_golden.py in {time.time() - t0:.0f} s")
    np.savetxt(path, obs, fmt="%.17g", header=hdr)
    return tag


if __name__ == "__main__":
    tags = sys.argv[1:] or ["pop", "dip0", "dip1", "dip2"]
    with mp.get_context("spawn").Pool(len(tags)) as pool:
        for t in pool.imap_unordered(_run, tags):
            print("done", t, flush=True)

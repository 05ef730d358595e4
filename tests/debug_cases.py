"""Small parity cases run in a child process against the bounds-checked debug build of libheom
(HEOM_LIB points at it; see test_gpu_debug_build.py).  Every kernel family runs once: the row-form
stage kernels (FP64, FP32 owner-lane and shared-memory link paths, the FP64 head), the column-form FP64
kernel, the split-TF32 tensor-core kernel, the column-0 kernels (alone and batched) and the general
kernel.  Each case is compared with the oracle; heom_observables would raise HEOM_E_BOUNDS if a bounds
check had failed.  Prints one line per case and exits non-zero on the first failure."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

from helpers import gpu_run, oracle_propagate  # noqa: E402
from paper_1803_03498_gb300 import heom  # noqa: E402
from paper_1803_03498_gb300 import workloads as wl  # noqa: E402


def check(name, p, precision, steps, stride=1):
    m, ore, oim, oobs = oracle_propagate(p, steps, stride=stride)
    r, gobs = gpu_run(p, precision, n_steps=steps, stride=stride)
    N = p.system.N
    if precision == "fp64":
        re, im = r.get_ados(0, r.n_ado)
        err = float(np.max(np.abs(re + 1j * im - (ore + 1j * oim))))
        ok = err <= 1e-12 * max(1.0, float(np.max(np.abs(ore + 1j * oim))))
    else:
        err = float(np.max(np.abs(gobs[:, :N] - oobs[:, :N])))
        ok = err <= 1e-6
    r.close()
    print(f"{name} {precision}: max error {err:.2e} {'ok' if ok else 'FAIL'}", flush=True)
    if not ok:
        raise SystemExit(1)


def main():
    print("library", heom.LIB_PATH, flush=True)
    heom.load()
    pop, dips = wl.fmo_like()
    dimer = wl.dimer()
    lh = wl.lhcii_like(n_steps=4)
    lh.system.D = 3
    H = np.array([[0.0, 0, 0], [0, 80.0, 40.0 + 15.0j], [0, 40.0 - 15.0j, 0.0]])
    s = wl.System("complex H + ground", H, [1, 2], [35.0, 60.0], [50.0, 100.0], [300.0, 300.0], K=1, D=3)
    rho = np.zeros((3, 3))
    rho[2, 2] = 1.0
    rho[1, 0] = 0.5
    cplx = wl.Propagation(s, rho, np.zeros((3, 3)), 0.5, 40, w=np.array([0.0, 0.6, 0.8]))
    sub = wl.System("fmo-like 3 sites", np.asarray(pop.system.H)[:3, :3], [0, 1, 2], [35.0] * 3, [166.0] * 3,
                    [77.0] * 3, K=1, D=3)
    g, _ = wl.two_exciton(sub)
    rho = np.zeros((g.N, g.N))
    rho[1, 1] = 1.0
    twox = wl.Propagation(g, rho, np.zeros_like(rho), 0.5, 20)
    check("dimer", dimer, "fp64", 40)
    check("dimer", dimer, "fp32_mixed", 40)
    check("fmo-like pop", pop, "fp64", 10)
    check("fmo-like pop", pop, "fp32_mixed", 10)
    check("fmo-like pop", pop, "split_tf32", 10)
    check("fmo-like dipole (column 0)", dips[0], "fp32_mixed", 10)
    check("fmo-like dipole (column 0)", dips[0], "fp64", 10)
    check("lhcii-like D=3 (column-form FP64)", lh, "fp64", 4)
    check("lhcii-like D=3", lh, "fp32_mixed", 4)
    check("complex H, unbathed ground", cplx, "fp64", 20)
    check("complex H, unbathed ground", cplx, "fp32_mixed", 20)
    check("two-exciton space (general kernel)", twox, "fp64", 20)
    check("two-exciton space (general kernel)", twox, "fp32_mixed", 20)
    # batched column-0 launches: three dipole runs in one graph, against their single runs
    runs = [heom.Run(p.system, p.rho0_re, p.rho0_im, precision="fp32_mixed", w=p.w, max_records=4) for p in dips]
    b = heom.Batch(runs, dips[0].dt_fs, 10, 10)
    b.launch(1)
    for p, r in zip(dips, runs):
        obs = r.observables()
        alone, aobs = gpu_run(p, "fp32_mixed", n_steps=10, stride=10)
        if not np.array_equal(obs, aobs):
            print("batched column-0 runs differ from single runs FAIL", flush=True)
            raise SystemExit(1)
        alone.close()
    b.close()
    print("batched column-0 runs: equal to single runs ok", flush=True)
    print("ALL OK", flush=True)


if __name__ == "__main__":
    main()

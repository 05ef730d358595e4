"""Shared test helpers: oracle models from workload systems, GPU runs through the C ABI."""
import numpy as np

from oracle.oracle import Bath, OracleModel


def oracle_for(system, terminator=True, rescale=True):
    baths = [Bath(st, l, t, T) for st, l, t, T in zip(system.bath_state, system.lambda_cm, system.tau_fs, system.T_K)]
    return OracleModel(system.H, baths, K=system.K, D=system.D, terminator=terminator, rescale=rescale,
                       decomposition=getattr(system, "decomposition", "matsubara"),
                       bath_mask=getattr(system, "bath_mask", None))


def oracle_start(m, rho_re, rho_im):
    re = np.zeros((m.n_ado, m.N, m.N))
    im = np.zeros_like(re)
    re[0], im[0] = rho_re, rho_im
    return re, im


def oracle_propagate(prop, n_steps, stride=1, terminator=True, rescale=True):
    m = oracle_for(prop.system, terminator, rescale)
    re, im = oracle_start(m, prop.rho0_re, prop.rho0_im)
    obs = m.rk4(re, im, prop.dt_fs, n_steps, obs_stride=stride, w=prop.w)
    return m, re, im, obs


def gpu_run(prop, precision="fp64", n_steps=None, stride=1, terminator=True, rescale=True, max_records=None):
    from paper_1803_03498_gb300 import heom

    n_steps = prop.n_steps if n_steps is None else n_steps
    mr = max_records or (n_steps // max(stride, 1) + 2)
    r = heom.Run(prop.system, prop.rho0_re, prop.rho0_im, precision=precision, w=prop.w, max_records=mr,
                 terminator=terminator, rescale=rescale)
    r.propagate(prop.dt_fs, n_steps, stride)
    return r, r.observables()

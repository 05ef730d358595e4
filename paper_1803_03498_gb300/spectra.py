"""Linear absorption, circular dichroism and static fluorescence spectra from the dipole correlation
functions that the propagation records (host post-processing and run set-up; every propagation runs
in libheom's kernels).

Section "Linear absorption spectra", Eq. lin_abs_mukamel: with all ADOs zero and
sigma_0(0) = mu_p^+ |0><0|, the rotationally averaged spectrum is
    LA(omega) = Re sum_p int_0^inf dt exp(i omega t) C_p(t),   C_p(t) = Tr[mu_p^- sigma_0(t)]
              = sum_a (e_p . d_a) sigma_0(t)[a, 0],
the correlation column a run records when its dipole weights are w_a = e_p . d_a.  Section
"Circular dichroism spectra": the same with the excitation vector replaced by the rotational
strengths (R_a x d_a) . e_p (the trace weights stay e_p . d_a).  The three Cartesian e_p give the
rotational average (section "Dipole operators and rotational averaging").  The correlation decays
at finite temperature, so it is padded with zeros before the transform (same section).

Section "Static Fluorescence Spectra": the emission runs start from the thermal state sigma_u(inf)
of every ADO, obtained by a long propagation from the Boltzmann state of the zero-phonon site
Hamiltonian (thermal_state), with the dipole applied to every ADO (emission_start).

The integral is the trapezoid sum over the recorded samples t_k = k dt_s:
    S(omega_j) = Re dt_s [C_0 / 2 + sum_{k>=1} exp(i omega_j t_k) C_k],  omega_j = 2 pi j / (n dt_s),
evaluated for all j at once by one FFT of length n (numpy's inverse FFT carries exp(+2 pi i jk/n)).
"""
from __future__ import annotations

import numpy as np

TWO_PI_C = 1.8836515673088532e-4  # rad/fs per cm^-1


def spectrum(corr, dt_fs: float, omega_ref_cm: float = 0.0, n_fft: int | None = None):
    """Spectrum of correlation samples.

    corr: complex array [n_t] or [n_p, n_t] (summed over the first axis), samples at t_k = k dt_fs.
    omega_ref_cm: the rotating-frame shift that was subtracted from the excited states (it is added
    back to the energy axis).  n_fft: transform length (>= n_t; zero padding), default 8 n_t rounded
    up to a power of two.
    Returns (energy_cm, S): energy_cm ascending over one period of width 2 pi / dt_fs, S real.
    """
    c = np.asarray(corr, dtype=complex)
    if c.ndim == 2:
        c = c.sum(axis=0)
    n_t = c.shape[0]
    if n_t < 2:
        raise ValueError("need at least two correlation samples")
    n = n_fft or 1 << int(np.ceil(np.log2(8 * n_t)))
    if n < n_t:
        raise ValueError("n_fft shorter than the correlation")
    w = c.copy()
    w[0] *= 0.5  # trapezoid weight of t = 0
    buf = np.zeros(n, dtype=complex)
    buf[:n_t] = w
    s = (dt_fs * n * np.fft.ifft(buf)).real  # S_j for omega_j = 2 pi j / (n dt)
    omega = 2.0 * np.pi * np.fft.fftfreq(n, d=dt_fs)  # signed angular frequencies, rad/fs
    order = np.argsort(omega)
    return omega[order] / TWO_PI_C + omega_ref_cm, s[order]


def correlations(obs, n_states: int):
    """The recorded correlation column of a run's observable records [n_rec, n_states + 5]."""
    obs = np.asarray(obs)
    return obs[:, n_states + 2] + 1j * obs[:, n_states + 3]


def rotational_strengths(positions, dipoles):
    """(R_a x d_a) for every site: [n_sites, 3] (section "Circular dichroism spectra")."""
    return np.cross(np.asarray(positions, dtype=float), np.asarray(dipoles, dtype=float))


# ---- static fluorescence (section "Static Fluorescence Spectra") -------------------------------

KB_CM = 0.6950348004  # cm^-1 per K


def boltzmann_state(system):
    """rho = exp(-H0 / k_B T) / Tr[...] with H0 = H minus the reorganisation energies of the baths on
    each site (the zero-phonon Hamiltonian of the site basis); the start of the thermal-state
    propagation.  All baths of the system share T (the first one's is used)."""
    H0 = np.array(system.H, dtype=float).copy()
    for st, lam in zip(system.bath_state, system.lambda_cm):
        H0[st, st] -= lam
    w, U = np.linalg.eigh(H0)
    p = np.exp(-(w - w.min()) / (KB_CM * float(system.T_K[0])))
    rho = (U * (p / p.sum())) @ U.T
    return 0.5 * (rho + rho.T)


def propagate_state(system, re, im, dt_fs, n_steps, stride=1, w=None, precision="fp64"):
    """Propagate a full hierarchy state (every ADO, [n_ado, N, N]) on the GPU; returns
    (observable records, final re, final im, |L sigma| / |sigma| of the final state)."""
    from . import heom

    # created with the state's own sigma_0, so that the record at creation is the first sample
    r = heom.Run(system, np.asarray(re[0]), np.asarray(im[0]), precision=precision, w=w,
                 max_records=(n_steps // stride if stride > 0 else 0) + 2)
    try:
        r.set_ados(0, re, im)
        r.propagate(dt_fs, n_steps, stride)
        obs = r.observables()
        fre, fim = r.get_ados(0, system.n_ado)
        lre, lim = r.rhs_eval(0, system.n_ado)
        resid = float(np.sqrt(np.sum(lre ** 2 + lim ** 2) / max(np.sum(fre ** 2 + fim ** 2), 1e-300)))
    finally:
        r.close()
    return obs, fre, fim, resid


def thermal_state(system, dt_fs, n_steps, precision="fp64"):
    """sigma_u(infinity) of every ADO by propagating the Boltzmann state (all other ADOs zero) for
    n_steps: returns (re, im, residual |L sigma| / |sigma| in 1/fs)."""
    n = system.n_ado
    re = np.zeros((n, system.N, system.N))
    im = np.zeros_like(re)
    re[0] = boltzmann_state(system)
    _, fre, fim, resid = propagate_state(system, re, im, dt_fs, n_steps, stride=0, precision=precision)
    return fre, fim, resid


def emission_start(thermal_re, thermal_im, dip_p):
    """Start of the emission run of polarisation p on the (N+1)-state space (state 0 = ground):
    every ADO X_u = sigma_u(infinity) mu_p^+, i.e. column 0 holds sigma_u(infinity) (e_p . d) and the
    rest is zero.  (The paper's Tr[mu_p^-(t) mu_p^+(infinity) sigma_0^*(infinity)] is read as the
    propagation of this coherence, the Hermitian conjugate of mu_p^- sigma(infinity), so that
    emission appears at positive frequency like absorption.)"""
    s = np.asarray(thermal_re) + 1j * np.asarray(thermal_im)
    n, N, _ = s.shape
    x = np.zeros((n, N + 1, N + 1), dtype=complex)
    x[:, 1:, 0] = s @ np.asarray(dip_p, dtype=float)
    return x.real.copy(), x.imag.copy()

"""Linear absorption and circular dichroism spectra from the dipole correlation functions that the
propagation records (host post-processing; the propagation itself runs in libheom's kernels).

Section "Linear absorption spectra", Eq. lin_abs_mukamel: with all ADOs zero and
sigma_0(0) = mu_p^+ |0><0|, the rotationally averaged spectrum is
    LA(omega) = Re sum_p int_0^inf dt exp(i omega t) C_p(t),   C_p(t) = Tr[mu_p^- sigma_0(t)]
              = sum_a (e_p . d_a) sigma_0(t)[a, 0],
the correlation column a run records when its dipole weights are w_a = e_p . d_a.  Section
"Circular dichroism spectra": the same with the excitation vector replaced by the rotational
strengths (R_a x d_a) . e_p (the trace weights stay e_p . d_a).  The three Cartesian e_p give the
rotational average (section "Dipole operators and rotational averaging").  The correlation decays
at finite temperature, so it is padded with zeros before the transform (same section).

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

"""Seeded synthetic inputs shaped like the paper's light-harvesting workloads.

This module only draws numbers: Hamiltonians, bath parameters, dipole directions, initial density
matrices, request streams and random hierarchy states.  It holds none of the HEOM arithmetic, so
both the CUDA path and the CPU oracle can take their inputs from it.

Energies are in cm^-1, times in fs, temperatures in K.  The workloads:

* ``dimer``      -- 2 sites, E = (0, 100), J = 50; lambda = 35, 1/nu = 50 fs, 300 K, K = 0, D = 4
                    (15 ADOs); rho(0) = |1><1|; dt = 1 fs, 2000 steps.
* ``fmo_like``   -- 7 sites, energies U[12100, 12600], couplings N(0, 40); lambda = 35,
                    1/nu = 166 fs, 77 K, K = 1 (14 modes), D = 4 (3060 ADOs); dt = 0.5 fs, 4000 steps;
                    populations from |1><1| and three dipole runs (state 0 = ground).
* ``lhcii_like`` -- 14 sites, energies U[14800, 15300], couplings N(0, 30); lambda = 35,
                    1/nu = 50 fs, 300 K, K = 1 (28 modes), D = 6 (1,344,904 ADOs); dt = 1 fs.
* ``ragged_batch`` -- 64 systems, N in {2..16}, D in {3..5}, K in {0, 1}, lambda U[20, 100],
                    1/nu U[50, 200], T in {77, 300}; three dipole orientations each.
* ``serving_stream`` -- Poisson arrivals of requests, N in {2..24}, D in {2..6}, K in {0, 1},
                    200..5000 steps.
* ``cd_runs``    -- three circular-dichroism runs of a site system, pigment centres from
                    ``site_positions`` (uniform in a 30 Angstrom cube; FMO-like: seed 1803022).
The FMO Hamiltonian printed in the paper (section "Results", FMO seven-pigment model) is
available as a fixed extra input from ``tests/golden``; it is not used by the benchmarks.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from math import comb

import numpy as np


@dataclass
class System:
    """A Frenkel-exciton system with one Drude-Lorentz bath per coupled state."""
    name: str
    H: np.ndarray                 # [N, N] real symmetric, cm^-1
    bath_state: list              # state index of each bath
    lambda_cm: list
    tau_fs: list
    T_K: list
    K: int                        # modes per bath beyond the Drude mode (modes per bath = K + 1)
    D: int                        # hierarchy depth
    decomposition: str = "matsubara"  # expansion of the Bose function: "matsubara" or "pade"
    bath_mask: np.ndarray | None = None  # [n_baths, N] 0/1: diagonal of V_b (None: |bath_state><bath_state|)

    @property
    def N(self) -> int:
        return int(self.H.shape[0])

    @property
    def n_modes(self) -> int:
        return len(self.bath_state) * (self.K + 1)

    @property
    def n_ado(self) -> int:
        return comb(self.n_modes + self.D, self.D)


@dataclass
class Propagation:
    system: System
    rho0_re: np.ndarray
    rho0_im: np.ndarray
    dt_fs: float
    n_steps: int
    w: np.ndarray | None = None   # dipole-correlation weights e_p . d_a per state (None: populations)
    tag: str = ""


def _sym_random_H(rng, n_sites, lo, hi, sd):
    H = np.zeros((n_sites, n_sites))
    H[np.diag_indices(n_sites)] = rng.uniform(lo, hi, n_sites)
    iu = np.triu_indices(n_sites, 1)
    H[iu] = rng.normal(0.0, sd, len(iu[0]))
    H = H + np.triu(H, 1).T
    return H


def _pure(N, s):
    re = np.zeros((N, N))
    re[s, s] = 1.0
    return re, np.zeros((N, N))


def dimer() -> Propagation:
    H = np.array([[0.0, 50.0], [50.0, 100.0]])
    sysm = System("dimer N=2 K=0 D=4", H, [0, 1], [35.0] * 2, [50.0] * 2, [300.0] * 2, K=0, D=4)
    re, im = _pure(2, 0)
    return Propagation(sysm, re, im, dt_fs=1.0, n_steps=2000, tag="dimer")


def with_ground_state(H_sites: np.ndarray, omega_ref: float | None = None):
    """State space 0 = ground, 1..N = sites.  The excited block is shifted by -omega_ref (a rotating
    frame; exact for the ground/one-exciton coherences that a linear-absorption run populates)."""
    n = H_sites.shape[0]
    if omega_ref is None:
        omega_ref = float(np.mean(np.diag(H_sites)))
    H = np.zeros((n + 1, n + 1))
    H[1:, 1:] = H_sites - omega_ref * np.eye(n)
    return H, omega_ref


def unit_dipoles(rng, n_sites):
    d = rng.normal(size=(n_sites, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def dipole_runs(sysm_sites: System, dip: np.ndarray, dt_fs: float, n_steps: int, tag: str):
    """Three linear-absorption runs (Cartesian e_p) on the (N+1)-state space."""
    Hg, _ = with_ground_state(sysm_sites.H)
    n = sysm_sites.N
    g = System(sysm_sites.name + " +ground", Hg, [s + 1 for s in sysm_sites.bath_state], list(sysm_sites.lambda_cm),
               list(sysm_sites.tau_fs), list(sysm_sites.T_K), sysm_sites.K, sysm_sites.D)
    out = []
    for p in range(3):
        w = np.zeros(n + 1)
        w[1:] = dip[:, p]
        re = np.zeros((n + 1, n + 1))
        re[:, 0] = w            # sigma_0(0) = mu_p^+ |0><0|
        out.append(Propagation(g, re, np.zeros_like(re), dt_fs, n_steps, w=w, tag=f"{tag}-dip{p}"))
    return out


def two_exciton(sysm_sites: System, omega_ref: float | None = None):
    """The system on the zero-, one- and two-exciton states of its N sites (section "Dipole operators
    and rotational averaging": N_states = 1 + N + N (N - 1) / 2).  State 0 is the ground state,
    state 1 + a has site a excited, and the pairs (a, b), a < b, follow in lexicographic order from
    N + 1.  The sites are hard-core excitons: a pair has energy E_a + E_b and couples to the pair
    (c, b) by J_ac (one excitation hops, the other stays).  Every excitation is counted from omega_ref
    (default: the mean site energy), so singles are shifted by -omega_ref and pairs by -2 omega_ref:
    the frame that rotates with a carrier at omega_ref.  The bath of site b couples through the site's
    number operator: V_b is 1 at the single b and at every pair that contains b (bath_mask).
    Returns (System, pairs)."""
    n = sysm_sites.N
    Hs = np.asarray(sysm_sites.H, dtype=float)
    if omega_ref is None:
        omega_ref = float(np.mean(np.diag(Hs)))
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    N = 1 + n + len(pairs)
    idx = {p: 1 + n + k for k, p in enumerate(pairs)}
    H = np.zeros((N, N))
    H[1:n + 1, 1:n + 1] = Hs - omega_ref * np.eye(n)
    for (a, b), i in idx.items():
        H[i, i] = Hs[a, a] + Hs[b, b] - 2.0 * omega_ref
        for (c, d), j in idx.items():
            shared = {a, b} & {c, d}
            if i != j and len(shared) == 1:
                x = ({a, b} - shared).pop()
                y = ({c, d} - shared).pop()
                H[i, j] = Hs[x, y]
    mask = np.zeros((len(sysm_sites.bath_state), N), np.uint8)
    for k, site in enumerate(sysm_sites.bath_state):
        mask[k, 1 + site] = 1
        for (a, b), i in idx.items():
            if site in (a, b):
                mask[k, i] = 1
    g = System(sysm_sites.name + " two-exciton", H, [1 + s for s in sysm_sites.bath_state],
               list(sysm_sites.lambda_cm), list(sysm_sites.tau_fs), list(sysm_sites.T_K), sysm_sites.K,
               sysm_sites.D, sysm_sites.decomposition, bath_mask=mask)
    return g, pairs


def two_exciton_dipole(n_sites: int, w) -> np.ndarray:
    """M+ = e . mu^+ on the two-exciton space of n_sites (order of two_exciton) for the weights
    w_a = e . d_a: site a is excited from the ground state (|a><0|) or on top of site b (|ab><b|)."""
    pairs = [(a, b) for a in range(n_sites) for b in range(a + 1, n_sites)]
    N = 1 + n_sites + len(pairs)
    Mp = np.zeros((N, N))
    for a in range(n_sites):
        Mp[1 + a, 0] = w[a]
    for k, (a, b) in enumerate(pairs):
        i = 1 + n_sites + k
        Mp[i, 1 + b] = w[a]
        Mp[i, 1 + a] = w[b]
    return Mp


@dataclass
class Pulse:
    """A Gaussian laser pulse in the rotating-wave approximation (Eq. h-field-rwa with Eq. probe_pulse):
    H(t) = H - g(t) M+ - conj(g(t)) M+^T, g(t) = amp exp(-(t - t_c)^2 / (2 sigma^2)) exp(-i (Delta t + phi)),
    amp (the coupling mu E in cm^-1 for unit dipole weights) and the detuning Delta of the carrier
    from the frame's reference frequency in cm^-1."""
    mu_plus: np.ndarray
    amp_cm: float
    t_center_fs: float
    sigma_fs: float
    phase: float = 0.0
    detuning_cm: float = 0.0


def fmo_two_exciton(n_sites: int = 7, D: int = 3, seed: int = 1803002, dip_seed: int = 1803012, amp_cm: float = 60.0):
    """The FMO-like system (first n_sites sites, K = 1) in the two-exciton space (29 states for
    7 sites) under one Gaussian pump pulse (sigma 15 fs, centred at 40 fs, resonant, x-polarised),
    from the ground state: returns (Propagation, Pulse)."""
    pop, _ = fmo_like(seed, dip_seed)
    s = pop.system
    sub = System(f"fmo-like {n_sites} sites", np.asarray(s.H)[:n_sites, :n_sites], list(range(n_sites)),
                 [35.0] * n_sites, [166.0] * n_sites, [77.0] * n_sites, K=1, D=D)
    g, _ = two_exciton(sub)
    dip = unit_dipoles(np.random.default_rng(dip_seed), 7)[:n_sites]
    Mp = two_exciton_dipole(n_sites, dip[:, 0])
    re = np.zeros((g.N, g.N))
    re[0, 0] = 1.0
    prop = Propagation(g, re, np.zeros_like(re), dt_fs=0.5, n_steps=200, tag=f"fmo-2x-{n_sites}")
    return prop, Pulse(Mp, amp_cm, 40.0, 15.0)


def site_positions(rng, n_sites, box_angstrom: float = 30.0):
    """Pigment centres R_a, uniform in a cube of the given edge (Angstrom), centred at the origin."""
    return rng.uniform(-0.5 * box_angstrom, 0.5 * box_angstrom, (n_sites, 3))


def cd_runs(sysm_sites: System, dip: np.ndarray, pos: np.ndarray, dt_fs: float, n_steps: int, tag: str):
    """Three circular-dichroism runs (Cartesian e_p) on the (N+1)-state space: sigma_0(0) has the
    rotational strengths (R_a x d_a) . e_p in column 0, the recorded correlation weights are
    e_p . d_a (mu_p^-)."""
    Hg, _ = with_ground_state(sysm_sites.H)
    n = sysm_sites.N
    g = System(sysm_sites.name + " +ground", Hg, [s + 1 for s in sysm_sites.bath_state], list(sysm_sites.lambda_cm),
               list(sysm_sites.tau_fs), list(sysm_sites.T_K), sysm_sites.K, sysm_sites.D)
    rot = np.cross(pos, dip)
    out = []
    for p in range(3):
        w = np.zeros(n + 1)
        w[1:] = dip[:, p]
        re = np.zeros((n + 1, n + 1))
        re[1:, 0] = rot[:, p]
        out.append(Propagation(g, re, np.zeros_like(re), dt_fs, n_steps, w=w, tag=f"{tag}-cd{p}"))
    return out


def fmo_like(seed: int = 1803002, dip_seed: int = 1803012):
    """Returns (population run, [3 dipole runs])."""
    rng = np.random.default_rng(seed)
    H = _sym_random_H(rng, 7, 12100.0, 12600.0, 40.0)
    sysm = System("fmo-like N=7 K=1 D=4", H, list(range(7)), [35.0] * 7, [166.0] * 7, [77.0] * 7, K=1, D=4)
    re, im = _pure(7, 0)
    pop = Propagation(sysm, re, im, dt_fs=0.5, n_steps=4000, tag="fmo-pop")
    dip = unit_dipoles(np.random.default_rng(dip_seed), 7)
    return pop, dipole_runs(sysm, dip, 0.5, 4000, "fmo")


def lhcii_like(seed: int = 1803003, n_steps: int = 1000) -> Propagation:
    rng = np.random.default_rng(seed)
    H = _sym_random_H(rng, 14, 14800.0, 15300.0, 30.0)
    sysm = System("lhcii-like N=14 K=1 D=6", H, list(range(14)), [35.0] * 14, [50.0] * 14, [300.0] * 14, K=1, D=6)
    re, im = _pure(14, 0)
    return Propagation(sysm, re, im, dt_fs=1.0, n_steps=n_steps, tag="lhcii-pop")


def _random_system(rng, n_sites, D, K, name):
    H = _sym_random_H(rng, n_sites, 12100.0, 12600.0, 40.0)
    lam = list(rng.uniform(20.0, 100.0, n_sites))
    tau = list(rng.uniform(50.0, 200.0, n_sites))
    T = float(rng.choice([77.0, 300.0]))
    return System(name, H, list(range(n_sites)), lam, tau, [T] * n_sites, K=K, D=D)


def ragged_batch(seed: int = 1803004, n_systems: int = 64, n_steps: int = 1000, dt_fs: float = 0.5):
    """64 systems x 3 dipole orientations = 192 propagations on (N+1)-state spaces."""
    rng = np.random.default_rng(seed)
    props = []
    for s in range(n_systems):
        n = int(rng.integers(2, 17))
        D = int(rng.integers(3, 6))
        K = int(rng.integers(0, 2))
        sysm = _random_system(rng, n, D, K, f"batch{s} N={n} K={K} D={D}")
        dip = unit_dipoles(rng, n)
        props += dipole_runs(sysm, dip, dt_fs, n_steps, f"batch{s}")
    return props


@dataclass
class Request:
    arrival_s: float
    prop: Propagation
    rid: int = 0
    meta: dict = field(default_factory=dict)


def serving_stream(rate_per_s: float, n_requests: int, seed: int = 1803005, dt_fs: float = 0.5,
                   n_max: int = 24, d_max: int = 6, steps_lo: int = 200, steps_hi: int = 5000,
                   max_ado_steps: float | None = None):
    """Poisson arrivals; population runs from |1><1| of random systems.  With max_ado_steps, draws
    whose ADO count times step count exceeds it are redrawn (a bounded sample of the same mix)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        while True:
            n = int(rng.integers(2, n_max + 1))
            D = int(rng.integers(2, d_max + 1))
            K = int(rng.integers(0, 2))
            steps = int(rng.integers(steps_lo, steps_hi + 1))
            if max_ado_steps is None or comb(n * (K + 1) + D, D) * steps <= max_ado_steps:
                break
        sysm = _random_system(rng, n, D, K, f"req{r} N={n} K={K} D={D}")
        re, im = _pure(n, 0)
        out.append(Request(t, Propagation(sysm, re, im, dt_fs, steps, tag=f"req{r}"), rid=r))
    return out


def random_state(n_ado: int, N: int, seed: int, scale: float = 1.0):
    """A dense random hierarchy state (re, im) [n_ado, N, N], float64, for single-stage checks."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n_ado, N, N)) * scale
    im = rng.standard_normal((n_ado, N, N)) * scale
    return re, im

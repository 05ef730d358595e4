"""ctypes front end of the plain CPU FP64 HEOM oracle (``heom_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py``.  The CUDA library never imports or links it, and it imports nothing
from the CUDA package.

State arrays use the canonical host layout shared with the library's host API: ADO-major,
then row-major N x N, real and imaginary parts in separate float64 arrays of shape [n_ado, N, N].
Energies in cm^-1, times in fs, temperatures in K.

Parity status of each function (against the paper, arXiv 1803.03498):
  hierarchy      pinned (counts of Eq. Nmatrices incl. the paper's printed 12,271,512; colex
                 closed-form rank; exhaustive link invariants)
  coefficients   pinned (Matsubara sum rule, high-temperature limit, resonance rejection)
  rhs / rk4      pinned (dense Kronecker Liouvillian, textbook-gauge equivalence, unitary limit,
                 trace/Hermiticity invariants, thermal relaxation, RK4 order)
  bath masks     pinned (dense Kronecker Liouvillian with diagonal V_b; the two-exciton space started
                 in the one-exciton block equals the one-exciton model)
  laser field    pinned (Rabi rotation of a two-level system by a resonant Gaussian pulse: closed form
                 through the pulse area; two uncoupled sites in the two-exciton space: the product of
                 two such rotations; a zero-amplitude field changes nothing)
  the paper prints its dynamics as figures only (no tabulated values), so no pin compares with
  printed numbers; every function above is pinned as listed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heom_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libheom_oracle.so")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        P = ctypes.POINTER
        d, i32, i64, u8, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint8, ctypes.c_void_p
        L.orc_hier_count.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_hier_count.restype = i64
        L.orc_hier_export.argtypes = [ctypes.c_int, ctypes.c_int, i64, P(u8), P(i32), P(i32)]
        L.orc_hier_export.restype = ctypes.c_int
        L.orc_create.argtypes = [ctypes.c_int, P(d), P(d), ctypes.c_int, P(ctypes.c_int), P(d), P(d), P(d),
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_pade.argtypes = [ctypes.c_int, P(d), P(d)]
        L.orc_pade.restype = ctypes.c_int
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_destroy.restype = None
        L.orc_n_ado.argtypes = [vp]
        L.orc_n_ado.restype = i64
        L.orc_n_modes.argtypes = [vp]
        L.orc_n_modes.restype = ctypes.c_int
        L.orc_export_modes.argtypes = [vp, P(d), P(d), P(d), P(ctypes.c_int), P(d)]
        L.orc_export_modes.restype = None
        L.orc_export_hierarchy.argtypes = [vp, P(u8), P(i32), P(i32)]
        L.orc_export_hierarchy.restype = None
        L.orc_rhs.argtypes = [vp, P(d), P(d), P(d), P(d)]
        L.orc_rhs.restype = None
        L.orc_rhs_list.argtypes = [vp, P(i64), i64, P(d), P(d), P(d), P(d)]
        L.orc_rhs_list.restype = None
        L.orc_record_len.argtypes = [vp]
        L.orc_record_len.restype = ctypes.c_int
        L.orc_rk4.argtypes = [vp, P(d), P(d), d, i64, i64, P(d), P(d)]
        L.orc_rk4.restype = ctypes.c_int
        L.orc_rk4_t.argtypes = [vp, P(d), P(d), d, d, i64, i64, P(d), P(d)]
        L.orc_rk4_t.restype = ctypes.c_int
        L.orc_set_bath_mask.argtypes = [vp, P(u8)]
        L.orc_set_bath_mask.restype = ctypes.c_int
        L.orc_set_field.argtypes = [vp, P(d), d, d, d, d, d]
        L.orc_set_field.restype = ctypes.c_int
        L.orc_set_time.argtypes = [vp, d]
        L.orc_set_time.restype = None
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def hier_count(M: int, D: int) -> int:
    """Brute-force count of tuples n in N^M with |n| <= D."""
    return int(lib().orc_hier_count(M, D))


def hier_export(M: int, D: int):
    """(tuples uint8 [n, M], plus int32 [n, M], minus int32 [n, M]) in the oracle's order."""
    n = hier_count(M, D)
    t = np.zeros((n, M), np.uint8)
    p = np.zeros((n, M), np.int32)
    m = np.zeros((n, M), np.int32)
    rc = lib().orc_hier_export(M, D, n, _ptr(t, ctypes.c_uint8), _ptr(p, ctypes.c_int32), _ptr(m, ctypes.c_int32))
    if rc != 0:
        raise RuntimeError(f"orc_hier_export failed ({rc})")
    return t, p, m


@dataclass
class Bath:
    state: int          # state index coupled through V = |state><state|
    lambda_cm: float    # reorganisation energy, cm^-1
    tau_fs: float       # bath correlation time 1/nu, fs
    T_K: float          # temperature, K


def pade(K):
    """Pade poles xi and weights eta of the Bose function (orc_pade): 1/(1 - e^-x) ~ 1/x + 1/2 +
    sum_i 2 eta_i x / (x^2 + xi_i^2)."""
    xi = np.zeros(K)
    eta = np.zeros(K)
    if lib().orc_pade(int(K), _ptr(xi, ctypes.c_double), _ptr(eta, ctypes.c_double)):
        raise ValueError("K must be >= 1")
    return xi, eta


@dataclass
class OracleModel:
    H: np.ndarray                 # [N, N] complex or real, cm^-1
    baths: list                   # list[Bath]
    K: int                        # modes per bath beyond the Drude mode (Matsubara terms or Pade poles)
    D: int                        # hierarchy depth
    terminator: bool = True
    rescale: bool = True
    decomposition: str = "matsubara"  # or "pade"
    bath_mask: np.ndarray | None = None  # [B, N] 0/1 diagonal of each V_b (None: |state><state|)
    _h: int = field(default=0, init=False, repr=False)

    def __post_init__(self):
        H = np.asarray(self.H)
        self.N = H.shape[0]
        hr = np.ascontiguousarray(H.real, dtype=np.float64)
        hi = np.ascontiguousarray(H.imag if np.iscomplexobj(H) else np.zeros_like(hr), dtype=np.float64)
        B = len(self.baths)
        st = np.array([b.state for b in self.baths], dtype=np.intc)
        la = np.array([b.lambda_cm for b in self.baths], dtype=np.float64)
        ta = np.array([b.tau_fs for b in self.baths], dtype=np.float64)
        Ta = np.array([b.T_K for b in self.baths], dtype=np.float64)
        h = lib().orc_create(self.N, _ptr(hr, ctypes.c_double), _ptr(hi, ctypes.c_double), B,
                             _ptr(st, ctypes.c_int), _ptr(la, ctypes.c_double), _ptr(ta, ctypes.c_double),
                             _ptr(Ta, ctypes.c_double), self.K, self.D, int(self.terminator), int(self.rescale),
                             {"matsubara": 0, "pade": 1}[self.decomposition])
        if not h:
            raise ValueError("oracle rejected the model (bad shape, state index or Matsubara resonance)")
        self._h = h
        self.n_ado = int(lib().orc_n_ado(h))
        self.M = int(lib().orc_n_modes(h))
        if self.bath_mask is not None:
            mk = np.ascontiguousarray(self.bath_mask, dtype=np.uint8)
            assert mk.shape == (B, self.N)
            if lib().orc_set_bath_mask(h, _ptr(mk, ctypes.c_uint8)):
                raise ValueError("bath mask entries must be 0 or 1")

    def set_field(self, mu_plus, amp_cm: float, t_center_fs: float, sigma_fs: float, phase: float = 0.0,
                  detuning_cm: float = 0.0):
        """H(t) = H - g(t) M+ - conj(g(t)) M+^T, g(t) = E0 exp(-(t - t_c)^2 / (2 sigma^2)) exp(-i (Delta t + phi));
        mu_plus None removes the field."""
        if mu_plus is None:
            lib().orc_set_field(self._h, None, 0.0, 0.0, 1.0, 0.0, 0.0)
            return
        self._mup = np.ascontiguousarray(mu_plus, dtype=np.float64)
        assert self._mup.shape == (self.N, self.N)
        if lib().orc_set_field(self._h, _ptr(self._mup, ctypes.c_double), float(amp_cm), float(t_center_fs),
                               float(sigma_fs), float(phase), float(detuning_cm)):
            raise ValueError("sigma_fs must be > 0")

    def set_time(self, t_fs: float):
        """rhs() uses H(t_fs) from now on."""
        lib().orc_set_time(self._h, float(t_fs))

    def __del__(self):
        if getattr(self, "_h", 0):
            lib().orc_destroy(self._h)
            self._h = 0

    def hierarchy(self):
        t = np.zeros((self.n_ado, self.M), np.uint8)
        p = np.zeros((self.n_ado, self.M), np.int32)
        m = np.zeros((self.n_ado, self.M), np.int32)
        lib().orc_export_hierarchy(self._h, _ptr(t, ctypes.c_uint8), _ptr(p, ctypes.c_int32), _ptr(m, ctypes.c_int32))
        return t, p, m

    def modes(self):
        """dict of per-mode gamma [1/fs], c [(rad/fs)^2], lamnu, state and per-bath terminator delta."""
        M, B = self.M, len(self.baths)
        g, c, ln = np.zeros(M), np.zeros(M), np.zeros(M)
        ms = np.zeros(M, np.intc)
        db = np.zeros(B)
        lib().orc_export_modes(self._h, _ptr(g, ctypes.c_double), _ptr(c, ctypes.c_double), _ptr(ln, ctypes.c_double),
                               _ptr(ms, ctypes.c_int), _ptr(db, ctypes.c_double))
        return {"gamma": g, "c": c, "lamnu": ln, "state": ms.astype(int), "delta": db}

    def zeros(self):
        return np.zeros((self.n_ado, self.N, self.N)), np.zeros((self.n_ado, self.N, self.N))

    def rhs(self, re: np.ndarray, im: np.ndarray):
        re = np.ascontiguousarray(re, dtype=np.float64)
        im = np.ascontiguousarray(im, dtype=np.float64)
        assert re.shape == (self.n_ado, self.N, self.N) and im.shape == re.shape
        ore, oim = np.empty_like(re), np.empty_like(im)
        lib().orc_rhs(self._h, _ptr(re, ctypes.c_double), _ptr(im, ctypes.c_double),
                      _ptr(ore, ctypes.c_double), _ptr(oim, ctypes.c_double))
        return ore, oim

    def rhs_list(self, us, re: np.ndarray, im: np.ndarray):
        us = np.ascontiguousarray(us, dtype=np.int64)
        re = np.ascontiguousarray(re, dtype=np.float64)
        im = np.ascontiguousarray(im, dtype=np.float64)
        assert re.shape == (self.n_ado, self.N, self.N)
        ore = np.empty((len(us), self.N, self.N))
        oim = np.empty_like(ore)
        lib().orc_rhs_list(self._h, _ptr(us, ctypes.c_int64), len(us), _ptr(re, ctypes.c_double),
                           _ptr(im, ctypes.c_double), _ptr(ore, ctypes.c_double), _ptr(oim, ctypes.c_double))
        return ore, oim

    def rk4(self, re: np.ndarray, im: np.ndarray, dt_fs: float, n_steps: int, obs_stride: int = 1, w=None,
            t0: float = 0.0):
        """Classic RK4 in place on (re, im) from time t0 (stage times t, t + h/2, t + h/2, t + h).
        Returns records [n_rec, N+4]: populations[N], trace re, trace im, correlation re, correlation im."""
        assert re.flags.c_contiguous and im.flags.c_contiguous and re.dtype == np.float64
        rl = int(lib().orc_record_len(self._h))
        n_rec = (n_steps // obs_stride + 1) if obs_stride > 0 else 1
        obs = np.zeros((n_rec, rl))
        wp = None
        if w is not None:
            w = np.ascontiguousarray(w, dtype=np.float64)
            wp = _ptr(w, ctypes.c_double)
        rc = lib().orc_rk4_t(self._h, _ptr(re, ctypes.c_double), _ptr(im, ctypes.c_double), float(t0), float(dt_fs),
                             int(n_steps), int(obs_stride), wp, _ptr(obs, ctypes.c_double))
        if rc != 0:
            raise MemoryError("oracle RK4 workspace allocation failed")
        return obs

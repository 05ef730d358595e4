"""Thin Python binding of libheom's C ABI (include/heom.h): argument marshalling only.

Every step of the propagation runs in the CUDA library; this module converts numpy arrays to
pointers, takes device memory for the workspace from PyTorch's caching allocator and passes the
current torch CUDA stream.  There is no fallback: ``load()`` raises if ``libheom.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HEOM_LIB selects another build of the same library (the bounds-checked debug build of build(debug=True))
LIB_PATH = os.environ.get("HEOM_LIB") or os.path.join(_HERE, "_build", "libheom.so")

HEOM_OK = 0
(HEOM_E_ARG, HEOM_E_OVERFLOW, HEOM_E_NOMEM, HEOM_E_CUDA, HEOM_E_TIMEOUT, HEOM_E_NUMERIC, HEOM_E_STATE,
 HEOM_E_BOUNDS) = range(-1, -9, -1)
FP64, FP32_MIXED, SPLIT_TF32 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32_mixed": FP32_MIXED, "split_tf32": SPLIT_TF32}

# every symbol include/heom.h declares
ABI_SYMBOLS = [
    "heom_last_error", "heom_build_hierarchy", "heom_hier_destroy", "heom_hier_info", "heom_hier_export",
    "heom_run_bytes", "heom_run_create", "heom_run_destroy", "heom_propagate", "heom_record_len",
    "heom_observables", "heom_get_sigma0", "heom_get_ados", "heom_set_ados", "heom_rhs_eval", "heom_run_info",
    "heom_run_launches", "heom_run_set_timing", "heom_run_kernel_time", "heom_propagate_static",
    "heom_batch_create", "heom_batch_launch", "heom_batch_destroy", "heom_bath_modes", "heom_run_layout",
    "heom_schedule_candidates", "heom_tune", "heom_set_autotune", "heom_get_schedule", "heom_set_schedule",
    "heom_tune_cache_clear", "heom_batch_schedule", "heom_set_default_schedule", "heom_run_set_field",
    "heom_group_propagate",
]
MATSUBARA, PADE = 0, 1
DECOMPOSITIONS = {"matsubara": MATSUBARA, "pade": PADE}


class HeomError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libheom error {code}: {msg}")
        self.code = code


class _System(ctypes.Structure):
    _fields_ = [
        ("n_states", ctypes.c_int),
        ("H_re", ctypes.POINTER(ctypes.c_double)),
        ("H_im", ctypes.POINTER(ctypes.c_double)),
        ("n_baths", ctypes.c_int),
        ("bath_state", ctypes.POINTER(ctypes.c_int)),
        ("lambda_cm", ctypes.POINTER(ctypes.c_double)),
        ("tau_fs", ctypes.POINTER(ctypes.c_double)),
        ("T_K", ctypes.POINTER(ctypes.c_double)),
        ("n_matsubara", ctypes.c_int),
        ("terminator", ctypes.c_int),
        ("rescale", ctypes.c_int),
        ("decomposition", ctypes.c_int),
        ("bath_mask", ctypes.POINTER(ctypes.c_uint8)),
        ("time_dependent", ctypes.c_int),
    ]


class _Field(ctypes.Structure):
    _fields_ = [
        ("mu_plus", ctypes.POINTER(ctypes.c_double)),
        ("amp_cm", ctypes.c_double),
        ("t_center_fs", ctypes.c_double),
        ("sigma_fs", ctypes.c_double),
        ("phase", ctypes.c_double),
        ("detuning_cm", ctypes.c_double),
    ]


class _Schedule(ctypes.Structure):
    _fields_ = [("occupancy_pct", ctypes.c_int), ("chunks_per_warp", ctypes.c_int)]


def _sched_tuple(s):
    return (int(s.occupancy_pct), int(s.chunks_per_warp))


_lib = None


def load():
    """Load libheom.so (built by ``paper_1803_03498_gb300.build.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libheom.so not found at {LIB_PATH}: build it with paper_1803_03498_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    i, i64, d, vp, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    L.heom_last_error.restype = ctypes.c_char_p
    L.heom_last_error.argtypes = []
    L.heom_build_hierarchy.argtypes = [i, i, P(vp)]
    L.heom_hier_destroy.argtypes = [vp]
    L.heom_hier_info.argtypes = [vp, P(i64), P(i64)]
    L.heom_hier_export.argtypes = [vp, P(ctypes.c_uint8), P(ctypes.c_int32), P(ctypes.c_int32)]
    L.heom_run_bytes.argtypes = [P(_System), vp, i, i64, P(sz)]
    L.heom_run_create.argtypes = [P(_System), vp, i, i64, P(d), P(d), P(d), vp, sz, vp, P(vp)]
    L.heom_run_destroy.argtypes = [vp]
    L.heom_propagate.argtypes = [vp, d, i64, i64]
    L.heom_record_len.argtypes = [vp]
    L.heom_observables.argtypes = [vp, P(d), i64, P(i64)]
    L.heom_get_sigma0.argtypes = [vp, P(d), P(d)]
    L.heom_get_ados.argtypes = [vp, i64, i64, P(d), P(d)]
    L.heom_set_ados.argtypes = [vp, i64, i64, P(d), P(d)]
    L.heom_rhs_eval.argtypes = [vp, i64, i64, P(d), P(d)]
    L.heom_run_info.argtypes = [vp, P(i64), P(i), P(i), P(i64), P(d)]
    L.heom_run_launches.argtypes = [vp]
    L.heom_run_launches.restype = i64
    L.heom_run_set_timing.argtypes = [vp, i]
    L.heom_run_kernel_time.argtypes = [vp, P(d), P(i64), P(d), P(d)]
    L.heom_batch_create.argtypes = [P(vp), i, d, i64, i64, P(vp)]
    L.heom_batch_launch.argtypes = [vp, i64]
    L.heom_batch_destroy.argtypes = [vp]
    L.heom_group_propagate.argtypes = [P(vp), i, d, P(i64), i64, vp]
    L.heom_propagate_static.argtypes = [P(_System), vp, i, P(d), P(d), P(d), d, i64, i64, vp, P(d), i64, P(i64),
                                        P(d), P(d)]
    S = _Schedule
    L.heom_schedule_candidates.argtypes = [i, P(S), i]
    L.heom_tune.argtypes = [vp, i, i, P(S), P(d), i, P(i), P(S)]
    L.heom_set_autotune.argtypes = [i]
    L.heom_get_schedule.argtypes = [vp, i, P(S)]
    L.heom_set_schedule.argtypes = [vp, i, P(S)]
    L.heom_tune_cache_clear.argtypes = []
    L.heom_set_default_schedule.argtypes = [i, P(S)]
    L.heom_run_set_field.argtypes = [vp, P(_Field)]
    L.heom_batch_schedule.argtypes = [vp, i, i, P(S), P(i)]
    for name in ABI_SYMBOLS:
        if name not in ("heom_last_error", "heom_run_launches"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != HEOM_OK:
        msg = load().heom_last_error()
        raise HeomError(rc, msg.decode() if msg else "")


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Hierarchy:
    """heom_build_hierarchy: multi-indices |n| <= depth over n_modes modes and their +/- links."""

    def __init__(self, n_modes: int, depth: int):
        L = load()
        self._h = ctypes.c_void_p()
        _check(L.heom_build_hierarchy(int(n_modes), int(depth), ctypes.byref(self._h)))
        self.n_modes, self.depth = int(n_modes), int(depth)
        n = ctypes.c_int64()
        offs = (ctypes.c_int64 * (depth + 2))()
        _check(L.heom_hier_info(self._h, ctypes.byref(n), offs))
        self.n_ado = int(n.value)
        self.level_offsets = np.array(list(offs), dtype=np.int64)

    def export(self):
        t = np.zeros((self.n_ado, self.n_modes), np.uint8)
        p = np.zeros((self.n_ado, self.n_modes), np.int32)
        m = np.zeros((self.n_ado, self.n_modes), np.int32)
        _check(load().heom_hier_export(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                       p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return t, p, m

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            load().heom_hier_destroy(self._h)
            self._h = ctypes.c_void_p()


class _SysArgs:
    """Keeps the numpy arrays behind a heom_system alive."""

    def __init__(self, system, terminator=True, rescale=True, time_dependent=False):
        H = np.asarray(system.H)
        self.H_re = np.ascontiguousarray(H.real, dtype=np.float64)
        self.H_im = np.ascontiguousarray(H.imag, dtype=np.float64) if np.iscomplexobj(H) else None
        self.bath_state = np.ascontiguousarray(system.bath_state, dtype=np.intc)
        self.lam = np.ascontiguousarray(system.lambda_cm, dtype=np.float64)
        self.tau = np.ascontiguousarray(system.tau_fs, dtype=np.float64)
        self.T = np.ascontiguousarray(system.T_K, dtype=np.float64)
        s = _System()
        s.n_states = int(H.shape[0])
        s.H_re = _dp(self.H_re)
        s.H_im = _dp(self.H_im)
        s.n_baths = len(self.bath_state)
        s.bath_state = self.bath_state.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        s.lambda_cm = _dp(self.lam)
        s.tau_fs = _dp(self.tau)
        s.T_K = _dp(self.T)
        s.n_matsubara = int(system.K)
        s.terminator = int(bool(terminator))
        s.rescale = int(bool(rescale))
        s.decomposition = DECOMPOSITIONS[getattr(system, "decomposition", "matsubara")]
        mask = getattr(system, "bath_mask", None)
        self.mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        s.bath_mask = None if self.mask is None else self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        s.time_dependent = int(bool(time_dependent))
        self.s = s


def schedule_candidates(layout: int):
    """heom_schedule_candidates (host only): the (occupancy_pct, chunks_per_warp) pairs the tuner
    times for layout 0 (matrix), 1 (column-0 run) or 2 (column-0 batch group)."""
    L = load()
    n = L.heom_schedule_candidates(int(layout), None, 0)
    if n < 0:
        _check(n)
    buf = (_Schedule * n)()
    L.heom_schedule_candidates(int(layout), buf, n)
    return [_sched_tuple(x) for x in buf]


def set_autotune(reps: int) -> int:
    """heom_set_autotune: timed launches per candidate when runs and batches are created (0: off);
    returns the previous value (a negative argument only queries)."""
    return int(load().heom_set_autotune(int(reps)))


def tune_cache_clear():
    _check(load().heom_tune_cache_clear())


def set_default_schedule(layout: int, schedule=None):
    """heom_set_default_schedule: the schedule (occupancy_pct, chunks_per_warp) that parts of a layout
    take without a cache entry or tuning; None restores (100, 1)."""
    s = None if schedule is None else ctypes.byref(_Schedule(int(schedule[0]), int(schedule[1])))
    _check(load().heom_set_default_schedule(int(layout), s))


def bath_modes(system, terminator=True):
    """Bath modes the library uses for `system` (host only): dict of gamma, c, lamnu [rad/fs units],
    mode_state (per mode) and term (per state)."""
    L = load()
    sa = _SysArgs(system, terminator=terminator)
    M = len(system.bath_state) * (system.K + 1)
    g, c, ln = (np.zeros(M) for _ in range(3))
    ms = np.zeros(M, dtype=np.intc)
    term = np.zeros(system.N)
    _check(L.heom_bath_modes(ctypes.byref(sa.s), _dp(g), _dp(c), _dp(ln),
                             ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(term)))
    return {"gamma": g, "c": c, "lamnu": ln, "mode_state": ms, "term": term}


def run_bytes(system, hier: Hierarchy, precision="fp64", max_records=1, terminator=True, rescale=True,
              time_dependent=False) -> int:
    sa = _SysArgs(system, terminator, rescale, time_dependent)
    b = ctypes.c_size_t()
    _check(load().heom_run_bytes(ctypes.byref(sa.s), hier._h, PRECISIONS[precision], int(max_records), ctypes.byref(b)))
    return int(b.value)


class Run:
    """One propagation (heom_run_create) on a torch-allocated device workspace and torch stream."""

    def __init__(self, system, rho0_re, rho0_im=None, precision="fp64", w=None, max_records=1024,
                 terminator=True, rescale=True, hier: Hierarchy | None = None, stream=None, workspace=None,
                 time_dependent=False):
        import torch

        L = load()
        self.system = system
        self.hier = hier if hier is not None else Hierarchy(system.n_modes, system.D)
        self.precision = precision
        self._sa = _SysArgs(system, terminator, rescale, time_dependent)
        nbytes = ctypes.c_size_t()
        _check(L.heom_run_bytes(ctypes.byref(self._sa.s), self.hier._h, PRECISIONS[precision], int(max_records),
                                ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device="cuda")
        self._ws = workspace
        base = workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        avail = workspace.numel() - (aligned - base)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        r0 = np.ascontiguousarray(rho0_re, dtype=np.float64)
        i0 = None if rho0_im is None else np.ascontiguousarray(rho0_im, dtype=np.float64)
        wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        self._r = ctypes.c_void_p()
        _check(L.heom_run_create(ctypes.byref(self._sa.s), self.hier._h, PRECISIONS[precision], int(max_records),
                                 _dp(r0), _dp(i0), _dp(wv), ctypes.c_void_p(aligned), ctypes.c_size_t(avail),
                                 ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(self._r)))
        self.N = int(np.asarray(system.H).shape[0])
        self.n_ado = self.hier.n_ado
        self.record_len = int(L.heom_record_len(self._r))

    def layout(self) -> int:
        """0: ADOs stored as N x N matrices; 1: as their column 0 (coherence block)."""
        return int(load().heom_run_layout(self._r))

    def set_field(self, pulse):
        """heom_run_set_field: a Gaussian RWA pulse (workloads.Pulse or any object with mu_plus, amp_cm,
        t_center_fs, sigma_fs, phase, detuning_cm); None removes it.  Needs time_dependent=True."""
        if pulse is None:
            _check(load().heom_run_set_field(self._r, None))
            return
        self._mup = np.ascontiguousarray(pulse.mu_plus, dtype=np.float64)
        f = _Field(_dp(self._mup), float(pulse.amp_cm), float(pulse.t_center_fs), float(pulse.sigma_fs),
                   float(getattr(pulse, "phase", 0.0)), float(getattr(pulse, "detuning_cm", 0.0)))
        _check(load().heom_run_set_field(self._r, ctypes.byref(f)))

    def propagate(self, dt_fs: float, n_steps: int, obs_stride: int = 0):
        _check(load().heom_propagate(self._r, float(dt_fs), int(n_steps), int(obs_stride)))

    def observables(self, cap: int | None = None) -> np.ndarray:
        cap = cap if cap is not None else 1 << 20
        buf = np.zeros((cap, self.record_len))
        written = ctypes.c_int64()
        _check(load().heom_observables(self._r, _dp(buf), cap, ctypes.byref(written)))
        return buf[: written.value].copy()

    def sigma0(self) -> np.ndarray:
        re = np.zeros((self.N, self.N))
        im = np.zeros((self.N, self.N))
        _check(load().heom_get_sigma0(self._r, _dp(re), _dp(im)))
        return re + 1j * im

    def get_ados(self, u0: int, count: int):
        re = np.zeros((count, self.N, self.N))
        im = np.zeros((count, self.N, self.N))
        _check(load().heom_get_ados(self._r, int(u0), int(count), _dp(re), _dp(im)))
        return re, im

    def set_ados(self, u0: int, re: np.ndarray, im: np.ndarray):
        re = np.ascontiguousarray(re, dtype=np.float64)
        im = np.ascontiguousarray(im, dtype=np.float64)
        _check(load().heom_set_ados(self._r, int(u0), int(re.shape[0]), _dp(re), _dp(im)))

    def rhs_eval(self, u0: int, count: int):
        re = np.zeros((count, self.N, self.N))
        im = np.zeros((count, self.N, self.N))
        _check(load().heom_rhs_eval(self._r, int(u0), int(count), _dp(re), _dp(im)))
        return re, im

    def info(self) -> dict:
        n_ado, n, m, steps, t = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_double()
        _check(load().heom_run_info(self._r, ctypes.byref(n_ado), ctypes.byref(n), ctypes.byref(m), ctypes.byref(steps),
                                    ctypes.byref(t)))
        return {"n_ado": n_ado.value, "n_states": n.value, "n_modes": m.value, "steps": steps.value, "t_fs": t.value}

    def launches(self) -> int:
        return int(load().heom_run_launches(self._r))

    def tune(self, part: int = 0, reps: int = 3):
        """heom_tune: time every candidate schedule of a part (0 body, 1 FP64 head); returns
        (chosen, [(schedule, ms per launch), ...])."""
        cap = 16
        tried = (_Schedule * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        ch = _Schedule()
        _check(load().heom_tune(self._r, int(part), int(reps), tried, ms, cap, ctypes.byref(n), ctypes.byref(ch)))
        return _sched_tuple(ch), [(_sched_tuple(tried[k]), float(ms[k])) for k in range(min(n.value, cap))]

    def schedule(self, part: int = 0):
        s = _Schedule()
        _check(load().heom_get_schedule(self._r, int(part), ctypes.byref(s)))
        return _sched_tuple(s)

    def set_schedule(self, occupancy_pct: int, chunks_per_warp: int = 1, part: int = 0):
        s = _Schedule(int(occupancy_pct), int(chunks_per_warp))
        _check(load().heom_set_schedule(self._r, int(part), ctypes.byref(s)))

    def set_timing(self, enable: bool):
        _check(load().heom_run_set_timing(self._r, int(bool(enable))))

    def kernel_time(self) -> dict:
        ms, n, b, f = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(load().heom_run_kernel_time(self._r, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b), ctypes.byref(f)))
        return {"ms": ms.value, "launches": n.value, "alg_bytes": b.value, "alg_flops": f.value}

    def close(self):
        if getattr(self, "_r", None) is not None and self._r.value:
            load().heom_run_destroy(self._r)
            self._r = ctypes.c_void_p()

    def __del__(self):
        self.close()


class Batch:
    """heom_batch_create: one CUDA graph advancing every run by steps_per_launch RK4 steps."""

    def __init__(self, runs, dt_fs: float, steps_per_launch: int, obs_stride: int = 1):
        L = load()
        self.runs = list(runs)  # keeps the runs (and their workspaces) alive
        arr = (ctypes.c_void_p * len(self.runs))(*[r._r.value for r in self.runs])
        self._b = ctypes.c_void_p()
        _check(L.heom_batch_create(arr, len(self.runs), float(dt_fs), int(steps_per_launch), int(obs_stride),
                                   ctypes.byref(self._b)))
        self.steps_per_launch = int(steps_per_launch)

    def launch(self, n_launches: int = 1):
        _check(load().heom_batch_launch(self._b, int(n_launches)))

    def schedules(self):
        """heom_batch_schedule: per group of batched column-0 launches, (body, FP64 head) schedules."""
        L = load()
        ng = ctypes.c_int()
        _check(L.heom_batch_schedule(self._b, -1, 0, None, ctypes.byref(ng)))
        out = []
        for g in range(ng.value):
            pair = []
            for part in (0, 1):
                s = _Schedule()
                _check(L.heom_batch_schedule(self._b, g, part, ctypes.byref(s), None))
                pair.append(_sched_tuple(s))
            out.append(tuple(pair))
        return out

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            load().heom_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        self.close()


def group_propagate(runs, dt_fs: float, n_steps, obs_stride: int = 0, stream=None):
    """heom_group_propagate: advance runs[i] by n_steps[i] RK4 steps (an int applies to every run),
    small mixed-precision runs of equal size sharing work-list launches; enqueued on `stream`
    (default: torch's current stream)."""
    import torch

    L = load()
    runs = list(runs)
    steps = [int(n_steps)] * len(runs) if np.isscalar(n_steps) else [int(x) for x in n_steps]
    if len(steps) != len(runs):
        raise ValueError("one step count per run")
    arr = (ctypes.c_void_p * len(runs))(*[r._r.value for r in runs])
    st = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    sarr = (ctypes.c_int64 * len(runs))(*steps)
    _check(L.heom_group_propagate(arr, len(runs), float(dt_fs), sarr, int(obs_stride), ctypes.c_void_p(st)))


def propagate_static(system, rho0_re, rho0_im=None, precision="fp64", w=None, dt_fs=1.0, n_steps=0, obs_stride=1,
                     terminator=True, rescale=True, hier: Hierarchy | None = None, stream=None):
    """heom_propagate_static: a whole propagation whose device workspace is the library's static
    array (no device allocation by the library or by this binding).  Returns (records, sigma_0)."""
    L = load()
    hier = hier if hier is not None else Hierarchy(system.n_modes, system.D)
    sa = _SysArgs(system, terminator, rescale)
    N = int(np.asarray(system.H).shape[0])
    cap = 1 + (n_steps // obs_stride if obs_stride > 0 else 0)
    rec = np.zeros((cap, N + 5))
    s_re = np.zeros((N, N))
    s_im = np.zeros((N, N))
    r0 = np.ascontiguousarray(rho0_re, dtype=np.float64)
    i0 = None if rho0_im is None else np.ascontiguousarray(rho0_im, dtype=np.float64)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    written = ctypes.c_int64()
    if stream is None:  # the same default as Run: torch's current stream on the current device
        import torch
        stream = torch.cuda.current_stream()
    st = ctypes.c_void_p(stream.cuda_stream)
    _check(L.heom_propagate_static(ctypes.byref(sa.s), hier._h, PRECISIONS[precision], _dp(r0), _dp(i0), _dp(wv),
                                   float(dt_fs), int(n_steps), int(obs_stride), st, _dp(rec), cap,
                                   ctypes.byref(written), _dp(s_re), _dp(s_im)))
    return rec[: written.value].copy(), s_re + 1j * s_im

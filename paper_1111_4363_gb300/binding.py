"""ctypes binding of the C ABI in include/leastaction.h (argument marshalling only).

Every numerical step runs in the CUDA library; this module converts Python/torch/numpy
arguments to pointers and sizes and raises ``LeastActionError`` on a non-zero status.
Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libleastaction.so")

LA_OK, LA_EINVAL, LA_ENOMEM, LA_ECUDA, LA_ENOTCONV, LA_ESTATE, LA_ETIMEOUT = range(7)
STATUS_NAMES = {0: "LA_OK", 1: "LA_EINVAL", 2: "LA_ENOMEM", 3: "LA_ECUDA", 4: "LA_ENOTCONV", 5: "LA_ESTATE",
                6: "LA_ETIMEOUT"}
WEIGHTS = {"dual": 0, "literal": 1, "identity": 2}
LOCAL_FORMS = {"lsq": 0, "square": 1}

EXPORTS = ["la_init", "la_set_hamiltonian", "la_step", "la_action", "la_solve_step", "la_residual",
           "la_relax_colour", "la_time_matrices", "la_backward", "la_step_batch", "la_profile_enable", "la_profile_read", "la_action_noalloc",
           "la_lfa_maps", "la_wait_selftest", "la_fma_peaks",
           "la_finalize", "la_last_error", "la_version"]
NOALLOC_MAX_POINTS = 1 << 22


class LeastActionError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class la_config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3), ("nt", C.c_int), ("dt", C.c_double),
                ("sub", C.c_int * 3), ("levels", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("coarse_sweeps", C.c_int), ("max_cycles", C.c_int), ("tol", C.c_double), ("weight", C.c_int),
                ("precision", C.c_int), ("laser_axis", C.c_int), ("ckpt_every", C.c_int),
                ("coarse_sub", C.c_int * 3), ("trial", C.c_int), ("coarse_cycle", C.c_int),
                ("coarse_nu1", C.c_int), ("coarse_nu2", C.c_int), ("cache_factors", C.c_int),
                ("local_form", C.c_int), ("factor_group", C.c_int)]


class la_pulse(C.Structure):
    _fields_ = [("ncomp", C.c_int), ("amp", C.POINTER(C.c_double)), ("omega", C.POINTER(C.c_double)),
                ("t_center", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double))]


class la_step_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("fine_sweeps", C.c_int), ("action", C.c_double), ("rel_action", C.c_double)]


class la_profile(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("n_factor", C.c_int), ("ms_factor", C.c_double),
                ("flops_factor", C.c_double), ("n_sweep", C.c_int), ("ms_sweep", C.c_double),
                ("flops_sweep", C.c_double), ("n_resid", C.c_int), ("ms_resid", C.c_double),
                ("bytes_resid", C.c_double), ("n_resid32", C.c_int), ("ms_resid32", C.c_double),
                ("bytes_resid32", C.c_double), ("n_restrict", C.c_int), ("ms_restrict", C.c_double),
                ("bytes_restrict", C.c_double), ("n_prolong", C.c_int), ("ms_prolong", C.c_double),
                ("bytes_prolong", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.la_init.argtypes = [C.POINTER(la_config), vp, C.POINTER(vp)]
        L.la_set_hamiltonian.argtypes = [vp, vp, C.POINTER(la_pulse)]
        L.la_step.argtypes = [vp, vp, i, d, C.POINTER(la_step_stats)]
        L.la_action.argtypes = [vp, C.POINTER(d), C.POINTER(d)]
        L.la_solve_step.argtypes = [vp, vp, d, i, vp, C.POINTER(la_step_stats)]
        L.la_residual.argtypes = [vp, vp, d, vp, vp, C.POINTER(d)]
        L.la_relax_colour.argtypes = [vp, vp, d, i, vp]
        L.la_time_matrices.argtypes = [vp, d, C.POINTER(d)]
        L.la_backward.argtypes = [vp, vp, C.POINTER(d), vp]
        L.la_step_batch.argtypes = [C.POINTER(vp), i, C.POINTER(vp), i, C.POINTER(d), C.POINTER(la_step_stats)]
        L.la_profile_enable.argtypes = [vp, i]
        L.la_profile_read.argtypes = [vp, C.POINTER(la_profile)]
        L.la_action_noalloc.argtypes = [C.POINTER(la_config), vp, C.POINTER(la_pulse), vp, d, vp, C.POINTER(d), vp]
        L.la_fma_peaks.argtypes = [C.POINTER(d), C.POINTER(d), C.POINTER(C.c_int), vp]
        L.la_finalize.argtypes = [vp]
        L.la_last_error.argtypes = [vp]
        L.la_last_error.restype = C.c_char_p
        L.la_version.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("la_last_error", "la_version"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def config_from_workload(w, precision: int = 0, **overrides) -> la_config:
    cfg = la_config()
    cfg.dim = w.dim
    for a in range(3):
        cfg.n[a] = w.n[a] if a < w.dim else 1
        cfg.h[a] = w.h[a]
        cfg.sub[a] = w.sub[a] if a < w.dim else 1
    cfg.nt, cfg.dt = w.nt, w.dt
    cfg.levels, cfg.nu1, cfg.nu2 = w.levels, w.nu1, w.nu2
    cfg.coarse_sweeps, cfg.max_cycles, cfg.tol = max(w.coarse_sweeps, 1), w.max_cycles, w.tol
    cfg.weight = WEIGHTS[w.weight]
    cfg.precision = precision
    cfg.laser_axis = w.pulse.axis if w.pulse is not None else 0
    if getattr(w, "coarse_sub", None) is not None:
        for a in range(w.dim):
            cfg.coarse_sub[a] = w.coarse_sub[a]
    cfg.trial = getattr(w, "trial", 0)
    if getattr(w, "coarse_nu", None) is not None:
        cfg.coarse_cycle, cfg.coarse_nu1, cfg.coarse_nu2 = 1, int(w.coarse_nu[0]), int(w.coarse_nu[1])
    cfg.local_form = LOCAL_FORMS[getattr(w, "local_form", "lsq")]
    cfg.factor_group = int(getattr(w, "factor_group", 0))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def _pulse_struct(pulse):
    p = la_pulse()
    keep = []
    if pulse is not None and pulse.ncomp > 0:
        for name, src in (("amp", pulse.amp), ("omega", pulse.omega), ("t_center", pulse.t_center),
                          ("sigma", pulse.sigma)):
            a = np.ascontiguousarray(np.asarray(src, dtype=np.float64))
            keep.append(a)
            setattr(p, name, a.ctypes.data_as(C.POINTER(C.c_double)))
        p.ncomp = pulse.ncomp
    return p, keep


class la_lfa_case(C.Structure):
    _fields_ = [("method", C.c_int), ("nx", C.c_int), ("nt", C.c_int), ("kappa", C.c_double), ("nu", C.c_double)]


LFA_METHODS = {"one": 0, "two": 1, "transfer": 2}


def lfa_maps(cases, k, w, out=None, stream=None) -> np.ndarray:
    """la_lfa_maps: cases = [(method, nx, nt, kappa, nu)], method a name of LFA_METHODS; returns (or fills
    ``out``, host or device, shaped [ncases, 2, len(w), len(k)]) log10 ratios after / before of N and |S|."""
    L = lib()
    arr = (la_lfa_case * len(cases))()
    for c, (method, nx, nt, kappa, nu) in enumerate(cases):
        arr[c] = la_lfa_case(LFA_METHODS[method], nx, nt, kappa, nu)
    k = np.ascontiguousarray(k, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    if out is None:
        out = np.zeros((len(cases), 2, len(w), len(k)))
    st = L.la_lfa_maps(arr, len(cases), k.ctypes.data_as(C.POINTER(C.c_double)), len(k),
                       w.ctypes.data_as(C.POINTER(C.c_double)), len(w), _ptr(out), _stream_handle(stream))
    if st != LA_OK:
        raise LeastActionError(st, L.la_last_error(None).decode())
    return out


def wait_selftest(polls: int, stream=None) -> int:
    """la_wait_selftest: the status word after one bounded wait on an mbarrier nothing completes."""
    L = lib()
    st = C.c_int(0)
    rc = L.la_wait_selftest(int(polls), C.byref(st), _stream_handle(stream))
    if rc != LA_OK:
        raise LeastActionError(rc, "la_wait_selftest failed")
    return st.value


def fma_peaks(stream=None):
    """la_fma_peaks: measured (FP64 TFLOP/s, FP32 TFLOP/s, SM count) of the current device."""
    L = lib()
    a, b, n = C.c_double(), C.c_double(), C.c_int()
    rc = L.la_fma_peaks(C.byref(a), C.byref(b), C.byref(n), _stream_handle(stream))
    if rc != LA_OK:
        raise LeastActionError(rc, "la_fma_peaks failed")
    return a.value, b.value, n.value


def action_noalloc(cfg: la_config, V0, pulse, psi0, t0: float, c, stream=None) -> float:
    """la_action_noalloc: residual norm N of device coefficients c without any device allocation."""
    L = lib()
    p, keep = _pulse_struct(pulse)
    N = C.c_double()
    st = L.la_action_noalloc(C.byref(cfg), _ptr(V0), C.byref(p), _ptr(psi0), float(t0), _ptr(c), C.byref(N),
                             _stream_handle(stream))
    if st != LA_OK:
        raise LeastActionError(st, L.la_last_error(None).decode())
    return N.value


def step_batch(contexts, psis, nsteps: int, t0s=None, allow_notconv: bool = False):
    """la_step_batch over Context objects; returns per-context lists of (cycles, sweeps, N, rel)."""
    L = lib()
    n = len(contexts)
    hs = (C.c_void_p * n)(*[c.handle.value for c in contexts])
    ps = (C.c_void_p * n)(*[_ptr(p).value for p in psis])
    t0 = (C.c_double * n)(*([0.0] * n if t0s is None else [float(t) for t in t0s]))
    rec = (la_step_stats * max(n * nsteps, 1))()
    st = L.la_step_batch(hs, n, ps, int(nsteps), t0, rec)
    if st != LA_OK and not (allow_notconv and st == LA_ENOTCONV):
        msgs = "; ".join(L.la_last_error(c.handle).decode() for c in contexts[:3])
        raise LeastActionError(st, msgs)
    return [[(r.cycles, r.fine_sweeps, r.action, r.rel_action) for r in rec[i * nsteps:(i + 1) * nsteps]]
            for i in range(n)]


class Context:
    """One least-action propagator context (la_init ... la_finalize)."""

    def __init__(self, cfg: la_config, stream=None):
        self._lib = lib()
        self.cfg = cfg
        h = C.c_void_p()
        st = self._lib.la_init(C.byref(cfg), _stream_handle(stream), C.byref(h))
        if st != LA_OK:
            raise LeastActionError(st, self._lib.la_last_error(None).decode())
        self.handle = h
        self.K = cfg.nt
        self.npoints = int(np.prod([cfg.n[a] for a in range(cfg.dim)]))
        self._keep = []

    def _check(self, st, allow=()):
        if st != LA_OK and st not in allow:
            raise LeastActionError(st, self._lib.la_last_error(self.handle).decode())
        return st

    def set_hamiltonian(self, V0, pulse=None):
        arrs = []
        p = la_pulse()
        if pulse is not None and pulse.ncomp > 0:
            for name, src in (("amp", pulse.amp), ("omega", pulse.omega), ("t_center", pulse.t_center),
                              ("sigma", pulse.sigma)):
                a = np.ascontiguousarray(np.asarray(src, dtype=np.float64))
                arrs.append(a)
                setattr(p, name, a.ctypes.data_as(C.POINTER(C.c_double)))
            p.ncomp = pulse.ncomp
        self._keep = arrs
        return self._check(self._lib.la_set_hamiltonian(self.handle, _ptr(V0), C.byref(p)))

    def step(self, psi, nsteps: int, t0: float = 0.0, stats: bool = False, allow_notconv: bool = False):
        rec = (la_step_stats * max(nsteps, 1))()
        st = self._check(self._lib.la_step(self.handle, _ptr(psi), int(nsteps), float(t0), rec),
                         allow=(LA_ENOTCONV,) if allow_notconv else ())
        if stats:
            return st, [(r.cycles, r.fine_sweeps, r.action, r.rel_action) for r in rec[:nsteps]]
        return st

    def action(self):
        N, rel = C.c_double(), C.c_double()
        self._check(self._lib.la_action(self.handle, C.byref(N), C.byref(rel)))
        return N.value, rel.value

    def solve_step(self, psi0, t0: float, c_out, ncycles: int = 0):
        rec = la_step_stats()
        st = self._check(self._lib.la_solve_step(self.handle, _ptr(psi0), float(t0), int(ncycles), _ptr(c_out),
                                                 C.byref(rec)), allow=(LA_ENOTCONV,))
        return st, (rec.cycles, rec.fine_sweeps, rec.action, rec.rel_action)

    def backward(self, dJ_dpsiT, ncomp: int, dJ_dpsi0=None) -> np.ndarray:
        """la_backward: dJ/d(amplitudes) (numpy) and, if given, dJ/dpsi_0^* written into dJ_dpsi0."""
        g = np.zeros(max(ncomp, 1))
        self._check(self._lib.la_backward(self.handle, _ptr(dJ_dpsiT), g.ctypes.data_as(C.POINTER(C.c_double)),
                                          _ptr(dJ_dpsi0)))
        return g[:ncomp]

    def residual(self, psi0, t0: float, c, r_out=None) -> float:
        N = C.c_double()
        self._check(self._lib.la_residual(self.handle, _ptr(psi0), float(t0), _ptr(c), _ptr(r_out), C.byref(N)))
        return N.value

    def relax_colour(self, psi0, t0: float, colour: int, c):
        return self._check(self._lib.la_relax_colour(self.handle, _ptr(psi0), float(t0), int(colour), _ptr(c)))

    def time_matrices(self, t0: float):
        K = self.K
        out = np.zeros(4 * K * K + 2 * K)
        self._check(self._lib.la_time_matrices(self.handle, float(t0), out.ctypes.data_as(C.POINTER(C.c_double))))
        KK = K * K
        return {"Ub": out[:KK].reshape(K, K), "Qb": out[KK:2 * KK].reshape(K, K),
                "Eb": out[2 * KK:3 * KK].reshape(K, K), "Ub0": out[3 * KK:3 * KK + K],
                "Eb0": out[3 * KK + K:3 * KK + 2 * K], "Wt": out[3 * KK + 2 * K:].reshape(K, K)}

    def profile_enable(self, on: bool = True):
        return self._check(self._lib.la_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self) -> dict:
        p = la_profile()
        self._check(self._lib.la_profile_read(self.handle, C.byref(p)))
        return {k: getattr(p, k) for k, _ in la_profile._fields_}

    def last_error(self) -> str:
        """la_last_error of this context."""
        return self._lib.la_last_error(self.handle).decode()

    def close(self):
        if getattr(self, "handle", None):
            self._lib.la_finalize(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

"""Thin ctypes binding of libpit.so (include/pit.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The C functions are exposed under their own names (``pit_problem_create``,
``pit_phi_batch``, ...); ``Problem`` wraps a problem handle and accepts torch
tensors (device memory, passed by ``data_ptr()``) or numpy arrays (host
memory, staged by the library where the header allows host pointers).

If libpit.so is missing or cannot be loaded, importing the binding's loader
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpit.so")
MAX_DIM = 6
MAX_HIST = 64

PIT_OK, PIT_ERR_INVALID_ARG, PIT_ERR_CUDA, PIT_ERR_OOM = 0, 1, 2, 3
PIT_ERR_NOCONV, PIT_ERR_BREAKDOWN, PIT_ERR_NONFINITE, PIT_ERR_TIMEOUT, PIT_ERR_UNSUPPORTED = 4, 5, 6, 7, 8
STATUS_NAMES = {0: "PIT_OK", 1: "PIT_ERR_INVALID_ARG", 2: "PIT_ERR_CUDA", 3: "PIT_ERR_OOM",
                4: "PIT_ERR_NOCONV", 5: "PIT_ERR_BREAKDOWN", 6: "PIT_ERR_NONFINITE", 7: "PIT_ERR_TIMEOUT",
                8: "PIT_ERR_UNSUPPORTED"}
PIT_OP_HEAT, PIT_OP_VARHEAT, PIT_OP_OU, PIT_OP_LSDE, PIT_OP_CME = 0, 1, 2, 3, 4
PIT_DRIFT_UPWIND, PIT_DRIFT_CENTRAL = 0, 1
PIT_PREC_FP64, PIT_PREC_MIXED, PIT_PREC_FP32, PIT_PREC_MIXED_PAIR = 0, 1, 2, 3
PIT_COARSE_IMPLICIT, PIT_COARSE_EXACT, PIT_COARSE_LEARNED, PIT_COARSE_SDIRK2, PIT_COARSE_EXTRAP = 0, 1, 2, 3, 4
PIT_RELAX_FCF, PIT_RELAX_F, PIT_RELAX_F_ALL = 0, 1, 2

EXPORTED = ["pit_problem_create", "pit_problem_destroy", "pit_problem_info", "pit_sample_initial", "pit_apply",
            "pit_phi_batch", "pit_sequential_solve", "pit_mgrit_solve", "pit_combine", "pit_profile_enable",
            "pit_profile_read", "pit_phi_batch_inplace_static", "pit_net_set_params", "pit_net_get_params",
            "pit_net_forward", "pit_net_loss_grad", "pit_train_coarse", "pit_recombine",
            "pit_sequential_solve_forced", "pit_last_error"]
NET_PARAMS = 3094
STATIC_SCRATCH_DOUBLES = 1 << 20


class pit_problem_desc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("level_n", ctypes.c_int), ("level0", ctypes.c_int), ("op", ctypes.c_int),
                ("lo", ctypes.c_double * MAX_DIM), ("hi", ctypes.c_double * MAX_DIM),
                ("theta", ctypes.c_double), ("sigma", ctypes.c_double), ("vamp", ctypes.c_double),
                ("drift", ctypes.c_double * (MAX_DIM * MAX_DIM)), ("diffusion", ctypes.c_double * (MAX_DIM * MAX_DIM)),
                ("drift_scheme", ctypes.c_int),
                ("cme_prod", ctypes.c_double * MAX_DIM), ("cme_sat", ctypes.c_double * MAX_DIM),
                ("cme_exp", ctypes.c_double * MAX_DIM), ("cme_deg", ctypes.c_double * MAX_DIM)]


class pit_solve_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("rtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("inner_rtol", ctypes.c_double), ("ir_maxit", ctypes.c_int), ("precond", ctypes.c_int),
                ("guess", ctypes.c_int)]


class pit_phi_stats(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int), ("n_failed", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("sum_iters", ctypes.c_longlong), ("max_refine", ctypes.c_int), ("status", ctypes.c_int)]


class pit_mgrit_opts(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("t1", ctypes.c_double), ("nsteps", ctypes.c_int), ("m", ctypes.c_int),
                ("levels", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("coarse", ctypes.c_int), ("fas", ctypes.c_int), ("fine", pit_solve_opts), ("crs", pit_solve_opts),
                ("relax", ctypes.c_int), ("lanes", ctypes.c_int), ("init", ctypes.c_int), ("recomb", ctypes.c_int),
                ("forcing", ctypes.c_void_p), ("tmul", ctypes.c_void_p), ("global_every", ctypes.c_int), ("residual", ctypes.c_int)]


class pit_mgrit_stats(ctypes.Structure):
    _fields_ = [("max_cycles", ctypes.c_int), ("n_converged", ctypes.c_int),
                ("res_hist", ctypes.c_double * MAX_HIST), ("phi_items", ctypes.c_longlong),
                ("krylov_iters", ctypes.c_longlong), ("point_iters", ctypes.c_longlong),
                ("learned_used", ctypes.c_int), ("fallback", ctypes.c_int), ("ms", ctypes.c_double)]


class pit_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 4), ("ms", ctypes.c_double * 4), ("phi_items", ctypes.c_longlong),
                ("point_iters", ctypes.c_longlong), ("point_passes", ctypes.c_longlong),
                ("point_steps", ctypes.c_longlong), ("kernels", ctypes.c_longlong * 4),
                ("point_iters_f", ctypes.c_longlong * 2), ("point_passes_f", ctypes.c_longlong * 2),
                ("point_steps_f", ctypes.c_longlong * 2), ("device_allocs", ctypes.c_longlong)]


class pit_train_opts(ctypes.Structure):
    _fields_ = [("dt_fine", ctypes.c_double), ("m", ctypes.c_int), ("n_pairs", ctypes.c_int),
                ("n_holdout", ctypes.c_int), ("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("ic_modes", ctypes.c_int), ("ic_fmax", ctypes.c_int),
                ("traj_len", ctypes.c_int), ("fine", pit_solve_opts), ("crs", pit_solve_opts), ("accept_ratio", ctypes.c_double)]


class pit_train_stats(ctypes.Structure):
    _fields_ = [("loss_first_epoch", ctypes.c_double), ("loss_last_epoch", ctypes.c_double),
                ("holdout_err_learned", ctypes.c_double), ("holdout_err_implicit", ctypes.c_double),
                ("accepted", ctypes.c_int), ("adam_steps", ctypes.c_int), ("ms_data", ctypes.c_double),
                ("ms_train", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads libpit.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libpit.so not found at {path}: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(path)
        vp, ci, cd, cll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        P = ctypes.POINTER
        L.pit_problem_create.argtypes = [P(pit_problem_desc), vp, P(vp)]
        L.pit_problem_destroy.argtypes = [vp]
        L.pit_problem_info.argtypes = [vp, P(ci), P(cll), vp, vp, vp]
        L.pit_sample_initial.argtypes = [vp, ci, vp, ci, vp]
        L.pit_apply.argtypes = [vp, cd, ci, vp, vp]
        L.pit_phi_batch.argtypes = [vp, cd, ci, vp, vp, vp, P(pit_solve_opts), P(pit_phi_stats)]
        L.pit_sequential_solve.argtypes = [vp, vp, cd, ci, P(pit_solve_opts), vp, P(pit_phi_stats)]
        L.pit_mgrit_solve.argtypes = [vp, vp, P(pit_mgrit_opts), vp, P(pit_mgrit_stats)]
        L.pit_combine.argtypes = [vp, vp, ci, vp, vp]
        L.pit_profile_enable.argtypes = [vp, ci]
        L.pit_profile_read.argtypes = [vp, P(pit_profile)]
        L.pit_phi_batch_inplace_static.argtypes = [vp, cd, ci, vp, vp, P(pit_solve_opts), P(pit_phi_stats)]
        L.pit_net_set_params.argtypes = [vp, vp, ci]
        L.pit_net_get_params.argtypes = [vp, vp, ci]
        L.pit_net_forward.argtypes = [vp, cd, ci, vp, vp]
        L.pit_net_loss_grad.argtypes = [vp, cd, ci, vp, vp, P(cd), vp]
        L.pit_train_coarse.argtypes = [vp, P(pit_train_opts), P(pit_train_stats)]
        L.pit_recombine.argtypes = [vp, vp, vp]
        L.pit_sequential_solve_forced.argtypes = [vp, vp, cd, ci, vp, vp, P(pit_solve_opts), vp, P(pit_phi_stats)]
        L.pit_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name != "pit_last_error":
                getattr(L, name).restype = ci
        _lib = L
    return _lib


class PitError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().pit_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != PIT_OK:
        raise PitError(st, where)


def _ptr(x):
    """Address of a torch tensor (device or host) or a numpy array (host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous() and str(x.dtype) == "torch.float64"
    return ctypes.c_void_p(x.data_ptr())


PIT_PRECOND_DEFAULT, PIT_PRECOND_NONE, PIT_PRECOND_JACOBI = 0, 1, 2
PIT_GUESS_DEFAULT, PIT_GUESS_PREVIOUS, PIT_GUESS_EXTRAPOLATE = 0, 1, 2


def solve_opts(prec=PIT_PREC_FP64, rtol=1e-10, maxit=10000, inner_rtol=1e-4, ir_maxit=12,
               precond=PIT_PRECOND_DEFAULT, guess=PIT_GUESS_DEFAULT) -> pit_solve_opts:
    return pit_solve_opts(prec, rtol, maxit, inner_rtol, ir_maxit, precond, guess)


def train_opts(dt_fine, m, n_pairs=4096, n_holdout=256, epochs=20, batch=64, lr=1e-3, seed=0, ic_modes=8,
               ic_fmax=4, traj_len=8, fine=None, crs=None, accept_ratio=1.0) -> pit_train_opts:
    fine = fine or solve_opts(PIT_PREC_MIXED, rtol=1e-10)
    crs = crs or fine
    return pit_train_opts(dt_fine, m, n_pairs, n_holdout, epochs, batch, lr, seed, ic_modes, ic_fmax, traj_len,
                          fine, crs, accept_ratio)


def mgrit_opts(t0, t1, nsteps, m, levels=2, tol=1e-8, maxit=64, coarse=PIT_COARSE_IMPLICIT, fine=None,
               crs=None, fas=False, relax=None, lanes=0, init=False, recomb=0, forcing=None,
               tmul=None, global_every=0, residual=False) -> pit_mgrit_opts:
    """forcing: device tensor of nsteps packed states (kept alive by the
    returned struct's _keep); tmul: per-grid steps per fine step (host)."""
    fine = fine or solve_opts()
    crs = crs or fine
    relax = PIT_RELAX_FCF if relax is None else relax
    keep = []
    fptr = None
    if forcing is not None:
        fptr = _ptr(forcing).value
        keep.append(forcing)
    tptr = None
    if tmul is not None:
        t = np.ascontiguousarray(tmul, dtype=np.int32)
        keep.append(t)
        tptr = t.ctypes.data
    init = int(init)  # False/True or 0, 1, 2 (2: extrapolated initial sweep)
    o = pit_mgrit_opts(t0, t1, nsteps, m, levels, tol, maxit, coarse, 1 if fas else 0, fine, crs, relax, lanes,
                       init, recomb, fptr, tptr, global_every, 1 if residual else 0)
    o._keep = keep
    return o


class Problem:
    """A combination-technique problem on the current CUDA device."""

    def __init__(self, d, n, L0=1, op=PIT_OP_HEAT, lo=None, hi=None, theta=1.0, sigma=1.0, vamp=0.5, stream=None,
                 drift=None, diffusion=None, drift_scheme=0, cme=None):
        """cme: (production, saturation, exponent, degradation) rates of the
        toggle-switch CME operator, scalars or one entry per species."""
        L = load()
        desc = pit_problem_desc()
        desc.d, desc.level_n, desc.level0, desc.op = d, n, L0, op
        lo = lo if lo is not None else [0.0] * d
        hi = hi if hi is not None else [1.0] * d
        for i in range(d):
            desc.lo[i], desc.hi[i] = lo[i], hi[i]
        desc.theta, desc.sigma, desc.vamp = theta, sigma, vamp
        if drift is not None:
            a = np.ascontiguousarray(drift, dtype=np.float64).ravel()
            hm = np.ascontiguousarray(diffusion, dtype=np.float64).ravel()
            for k in range(d * d):
                desc.drift[k], desc.diffusion[k] = a[k], hm[k]
        desc.drift_scheme = drift_scheme
        if cme is not None:
            rates = [np.broadcast_to(np.asarray(c, dtype=np.float64), (d,)) for c in cme]
            for i in range(d):
                desc.cme_prod[i], desc.cme_sat[i], desc.cme_exp[i], desc.cme_deg[i] = (float(r[i]) for r in rates)
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream is not None else None
        _check(L.pit_problem_create(ctypes.byref(desc), s, ctypes.byref(h)), "pit_problem_create")
        self._h = h
        self.d = d
        G, nt = ctypes.c_int(), ctypes.c_longlong()
        _check(L.pit_problem_info(h, ctypes.byref(G), ctypes.byref(nt), None, None, None), "pit_problem_info")
        self.G, self.n_total = G.value, nt.value
        self.levels = np.zeros((self.G, d), dtype=np.int32)
        self.coef = np.zeros(self.G)
        self.offsets = np.zeros(self.G + 1, dtype=np.int64)
        _check(L.pit_problem_info(h, None, None, ctypes.c_void_p(self.levels.ctypes.data),
                                  ctypes.c_void_p(self.coef.ctypes.data), ctypes.c_void_p(self.offsets.ctypes.data)),
               "pit_problem_info")

    def close(self):
        if getattr(self, "_h", None):
            load().pit_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample_initial(self, kind, params, out):
        params = np.ascontiguousarray(params, dtype=np.float64)
        _check(load().pit_sample_initial(self._h, kind, ctypes.c_void_p(params.ctypes.data), params.size, _ptr(out)),
               "pit_sample_initial")
        return out

    def apply(self, dt, p, q, n_batch=None):
        nb = n_batch if n_batch is not None else p.numel() // self.n_total
        _check(load().pit_apply(self._h, dt, nb, _ptr(p), _ptr(q)), "pit_apply")
        return q

    def phi_batch(self, dt, u_prev, u_next, opts=None, f=None, n_batch=None, stats=True):
        nb = n_batch if n_batch is not None else u_prev.numel() // self.n_total
        st = pit_phi_stats() if stats else None
        _check(load().pit_phi_batch(self._h, dt, nb, _ptr(u_prev), _ptr(f), _ptr(u_next),
                                    ctypes.byref(opts or solve_opts()), ctypes.byref(st) if st else None),
               "pit_phi_batch")
        return st

    def phi_batch_inplace_static(self, dt, u, opts=None, f=None, n_batch=None, stats=True):
        """In-place step without any allocation (static scratch inside libpit)."""
        nb = n_batch if n_batch is not None else u.numel() // self.n_total
        st = pit_phi_stats() if stats else None
        _check(load().pit_phi_batch_inplace_static(self._h, dt, nb, _ptr(u), _ptr(f),
                                                   ctypes.byref(opts or solve_opts()),
                                                   ctypes.byref(st) if st else None),
               "pit_phi_batch_inplace_static")
        return st

    def sequential_solve(self, u0, dt, nsteps, uT, opts=None):
        st = pit_phi_stats()
        _check(load().pit_sequential_solve(self._h, _ptr(u0), dt, nsteps, ctypes.byref(opts or solve_opts()),
                                           _ptr(uT), ctypes.byref(st)), "pit_sequential_solve")
        return st

    def sequential_solve_forced(self, u0, dt, nsteps, uT, opts=None, forcing=None, tmul=None):
        st = pit_phi_stats()
        t = np.ascontiguousarray(tmul, dtype=np.int32) if tmul is not None else None
        _check(load().pit_sequential_solve_forced(self._h, _ptr(u0), dt, nsteps, _ptr(forcing),
                                                  ctypes.c_void_p(t.ctypes.data) if t is not None else None,
                                                  ctypes.byref(opts or solve_opts()), _ptr(uT), ctypes.byref(st)),
               "pit_sequential_solve_forced")
        return st

    def mgrit_solve(self, u0, opts, uT, check=True):
        st = pit_mgrit_stats()
        rc = load().pit_mgrit_solve(self._h, _ptr(u0), ctypes.byref(opts), _ptr(uT), ctypes.byref(st))
        if check:
            _check(rc, "pit_mgrit_solve")
        return st if check else (st, rc)

    # learned coarse propagator
    def net_set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().pit_net_set_params(self._h, ctypes.c_void_p(w.ctypes.data), w.size), "pit_net_set_params")

    def net_get_params(self) -> np.ndarray:
        w = np.empty(NET_PARAMS, dtype=np.float32)
        _check(load().pit_net_get_params(self._h, ctypes.c_void_p(w.ctypes.data), w.size), "pit_net_get_params")
        return w

    def net_forward(self, dT, u, out, n_batch=None):
        nb = n_batch if n_batch is not None else u.numel() // self.n_total
        _check(load().pit_net_forward(self._h, dT, nb, _ptr(u), _ptr(out)), "pit_net_forward")
        return out

    def net_loss_grad(self, dT, u, y, n_batch=None):
        nb = n_batch if n_batch is not None else u.numel() // self.n_total
        loss = ctypes.c_double()
        grad = np.empty(NET_PARAMS, dtype=np.float32)
        _check(load().pit_net_loss_grad(self._h, dT, nb, _ptr(u), _ptr(y), ctypes.byref(loss),
                                        ctypes.c_void_p(grad.ctypes.data)), "pit_net_loss_grad")
        return loss.value, grad

    def train_coarse(self, opts) -> pit_train_stats:
        st = pit_train_stats()
        _check(load().pit_train_coarse(self._h, ctypes.byref(opts), ctypes.byref(st)), "pit_train_coarse")
        return st

    def profile_enable(self, on=True):
        _check(load().pit_profile_enable(self._h, 1 if on else 0), "pit_profile_enable")

    def profile_read(self) -> pit_profile:
        pr = pit_profile()
        _check(load().pit_profile_read(self._h, ctypes.byref(pr)), "pit_profile_read")
        return pr

    def recombine(self, u, out):
        _check(load().pit_recombine(self._h, _ptr(u), _ptr(out)), "pit_recombine")
        return out

    def combine(self, u, pts, out):
        n_pts = (pts.size if isinstance(pts, np.ndarray) else pts.numel()) // self.d
        _check(load().pit_combine(self._h, _ptr(u), n_pts, _ptr(pts), _ptr(out)), "pit_combine")
        return out

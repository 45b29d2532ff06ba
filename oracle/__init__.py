"""Plain FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It is a
ctypes wrapper around ``pit_oracle.c`` (plain C, built with gcc), which
restates the method of Griebel, Schweitzer and Troska (arXiv 2509.22156):
backward-Euler propagators (Sec. 2, Eq. "parabolic_problem_time_propagation"),
the combination formula (Eq. "combination_technique_solution"), textbook CG /
BiCGStab (Sec. 4.1) and two- and three-level FAS MGRIT with FCF relaxation
(Sec. 3.3, Alg. 2; per grid as in Alg. 3).  It shares no code with the CUDA
library.  Every function is pinned by the ``-m "not gpu"`` tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pit_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_HEAT, OP_VARHEAT, OP_OU, OP_LSDE, OP_CME = 0, 1, 2, 3, 4
STATUS = {0: "ok", 1: "invalid argument", 4: "no convergence", 5: "breakdown"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-D_DEFAULT_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            c_int, c_double, c_ll, vp = ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p
            L.or_coefficient.restype = c_double
            L.or_coefficient.argtypes = [c_int, c_int]
            L.or_enumerate.restype = c_int
            L.or_enumerate.argtypes = [c_int, c_int, c_int, vp, vp, c_int]
            L.or_grid_points.restype = c_ll
            L.or_grid_points.argtypes = [c_int, vp]
            L.or_create.restype = vp
            L.or_create.argtypes = [c_int, c_int, c_int, c_int, vp, vp, c_double, c_double, c_double]
            L.or_destroy.argtypes = [vp]
            L.or_set_sde.restype = c_int
            L.or_set_sde.argtypes = [vp, vp, vp, c_int]
            L.or_set_cme.restype = c_int
            L.or_set_cme.argtypes = [vp, vp, vp, vp, vp, c_int]
            L.or_info.argtypes = [vp, vp, vp, vp, vp, vp]
            L.or_set_threads.argtypes = [c_int]
            L.or_max_threads.restype = c_int
            L.or_apply.argtypes = [vp, c_double, c_int, vp, vp]
            L.or_phi.restype = c_int
            L.or_phi.argtypes = [vp, c_double, c_int, vp, vp, vp, c_double, c_int, vp]
            L.or_dense_solve.restype = c_int
            L.or_dense_solve.argtypes = [vp, c_int, c_double, vp, vp]
            L.or_sequential.restype = c_int
            L.or_sequential.argtypes = [vp, vp, c_double, c_int, c_double, c_int, vp, vp, vp, vp]
            L.or_mgrit.restype = c_int
            L.or_mgrit.argtypes = [vp, vp, c_double, c_int, c_int, c_int, c_double, c_int, c_int,
                                   vp, c_double, c_int, vp, vp, vp, vp, c_int, c_int, vp, vp]
            L.or_coarse_step.restype = c_int
            L.or_coarse_step.argtypes = [vp, c_double, c_int, c_int, c_int, c_double, vp, vp]
            L.or_combine.argtypes = [vp, vp, c_int, vp, vp]
            L.or_interp.argtypes = [vp, c_int, vp, c_int, vp, vp]
            L.or_hierarchize.restype = c_int
            L.or_hierarchize.argtypes = [vp, vp, vp, c_int]
            L.or_recombine.restype = c_int
            L.or_recombine.argtypes = [vp, vp, vp]
            L.or_initial.restype = c_int
            L.or_initial.argtypes = [vp, c_int, vp, c_int, vp]
            L.or_net_param_count.restype = c_ll
            L.or_net_forward.argtypes = [vp, c_double, vp, c_int, vp, vp]
            L.or_net_loss_grad.restype = c_double
            L.or_net_loss_grad.argtypes = [vp, c_double, vp, c_int, vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def coefficient(d: int, w: int) -> float:
    return lib().or_coefficient(d, w)


def enumerate_grids(d: int, n: int, L0: int = 1):
    """Levels (G x d int array) and layers w (G) of the combination grid set."""
    G = lib().or_enumerate(d, n, L0, None, None, 0)
    if G < 0:
        raise ValueError("invalid (d, n, L0)")
    lev = np.zeros((G, d), dtype=np.int32)
    lay = np.zeros(G, dtype=np.int32)
    lib().or_enumerate(d, n, L0, _p(lev), _p(lay), G)
    return lev, lay


def grid_points(levels) -> int:
    l = np.ascontiguousarray(levels, dtype=np.int32)
    return int(lib().or_grid_points(len(l), _p(l)))


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


class Problem:
    """One combination-technique problem on the CPU (FP64)."""

    def __init__(self, d, n, L0=1, op=OP_HEAT, lo=None, hi=None, theta=1.0, sigma=1.0, vamp=0.5,
                 drift=None, diffusion=None, central=False, cme=None):
        self.d, self.n, self.L0, self.op = d, n, L0, op
        self.lo = _f64(lo if lo is not None else [0.0] * d)
        self.hi = _f64(hi if hi is not None else [1.0] * d)
        self.theta, self.sigma, self.vamp = theta, sigma, vamp
        self._h = lib().or_create(d, n, L0, op, _p(self.lo), _p(self.hi), theta, sigma, vamp)
        if not self._h:
            raise ValueError("invalid problem description")
        if op == OP_LSDE:
            # linear SDE dX = A X dt + sigma dW, H = 2 sigma D sigma^T (Sec. 4.4);
            # drift flux donor cell (first order) or central (second order)
            self.drift = _f64(drift).reshape(d, d)
            self.diffusion = _f64(diffusion).reshape(d, d)
            self.central = bool(central)
            if lib().or_set_sde(self._h, _p(self.drift), _p(self.diffusion), int(self.central)) != 0:
                raise ValueError("invalid linear-SDE parameters")
        if op == OP_CME:
            # toggle-switch chemical master equation (Sec. 4.3): cme = (p, s, b,
            # g), one entry per species each: production p / (s + y^b), y the
            # other species' total, degradation g x_i
            self.cme = [_f64(np.broadcast_to(np.asarray(c, dtype=float), (d,))) for c in cme]
            self.central = bool(central)
            if lib().or_set_cme(self._h, *[_p(c) for c in self.cme], int(self.central)) != 0:
                raise ValueError("invalid CME parameters")
        G = ctypes.c_int()
        nt = ctypes.c_longlong()
        lib().or_info(self._h, ctypes.byref(G), ctypes.byref(nt), None, None, None)
        self.G, self.n_total = G.value, nt.value
        self.levels = np.zeros((self.G, d), dtype=np.int32)
        self.coef = np.zeros(self.G)
        self.offsets = np.zeros(self.G + 1, dtype=np.int64)
        lib().or_info(self._h, None, None, _p(self.levels), _p(self.coef), _p(self.offsets))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def grid_slice(self, g: int) -> slice:
        return slice(int(self.offsets[g]), int(self.offsets[g + 1]))

    def apply(self, dt: float, p) -> np.ndarray:
        p = _f64(p)
        nb = p.size // self.n_total
        q = np.empty_like(p)
        lib().or_apply(self._h, dt, nb, _p(p), _p(q))
        return q

    def phi(self, dt, u_prev, f=None, rtol=1e-14, maxit=100000, return_iters=False):
        u_prev = _f64(u_prev)
        nb = u_prev.size // self.n_total
        out = np.empty_like(u_prev)
        its = np.zeros(nb * self.G, dtype=np.int32)
        fp = _f64(f) if f is not None else None
        st = lib().or_phi(self._h, dt, nb, _p(u_prev), _p(fp), _p(out), rtol, maxit, _p(its))
        if st != 0:
            raise RuntimeError(f"oracle phi: {STATUS.get(st, st)}")
        return (out, its) if return_iters else out

    def dense_solve(self, g: int, dt: float, b) -> np.ndarray:
        b = _f64(b)
        x = np.empty_like(b)
        st = lib().or_dense_solve(self._h, g, dt, _p(b), _p(x))
        if st != 0:
            raise RuntimeError("grid too large for the dense solve")
        return x

    def _gmask(self, grids):
        if grids is None:
            return None
        m = np.zeros(self.G, dtype=np.uint8)
        m[np.asarray(grids, dtype=np.int64)] = 1
        return m

    def _forcing(self, forcing, nsteps):
        if forcing is None:
            return None
        f = _f64(forcing)
        if f.size != nsteps * self.n_total:
            raise ValueError("forcing must hold nsteps packed states")
        return f

    def _tmul(self, tmul):
        if tmul is None:
            return None
        t = np.ascontiguousarray(tmul, dtype=np.int32)
        if t.size != self.G or np.any(t < 1):
            raise ValueError("tmul must hold one integer >= 1 per grid")
        return t

    def sequential(self, u0, dt, nsteps, rtol=1e-14, maxit=100000, grids=None, forcing=None,
                   tmul=None) -> np.ndarray:
        """Sequential stepping; with `grids`, only those grids are computed
        (the other entries of the result are zero).  forcing: f_n of steps
        n = 1..nsteps (nsteps packed states); tmul: per grid steps per step."""
        u0 = _f64(u0)
        out = np.zeros_like(u0)
        gm = self._gmask(grids)
        F = self._forcing(forcing, nsteps)
        tm = self._tmul(tmul)
        st = lib().or_sequential(self._h, _p(u0), dt, nsteps, rtol, maxit, _p(out), _p(gm), _p(F), _p(tm))
        if st != 0:
            raise RuntimeError(f"oracle sequential: {STATUS.get(st, st)}")
        return out

    def mgrit(self, u0, dt, nsteps, m, levels=2, tol=1e-10, maxit=100, coarse_kind=0,
              theta=None, rtol=1e-14, krylov_maxit=100000, check=True, grids=None, relax="FCF", init=False,
              forcing=None, tmul=None):
        """Returns (uT, cycles per grid, residual history G x maxit, status);
        with `grids`, only those grids are computed.  relax: "FCF" (Sec. 4.1)
        or "F" (F-relaxation on the finest level) or "F_ALL" (F-relaxation on
        every level).  init: start from one sweep
        of the level-1 propagator over the C-points instead of u0 everywhere
        (2: that sweep with the extrapolated backward Euler, coarse kind 4)."""
        if relax not in ("FCF", "F", "F_ALL"):
            raise ValueError("relax must be 'FCF', 'F' or 'F_ALL'")
        u0 = _f64(u0)
        out = np.zeros_like(u0)
        gm = self._gmask(grids)
        its = np.zeros(self.G, dtype=np.int32)
        hist = np.full((self.G, maxit), np.nan)
        th = _f64(theta) if theta is not None else None
        F = self._forcing(forcing, nsteps)
        tm = self._tmul(tmul)
        st = lib().or_mgrit(self._h, _p(u0), dt, nsteps, m, levels, tol, maxit, coarse_kind,
                            _p(th), rtol, krylov_maxit, _p(out), _p(its), _p(hist), _p(gm),
                            {"FCF": 0, "F": 1, "F_ALL": 2}[relax], int(init), _p(F), _p(tm))
        if check and st != 0:
            raise RuntimeError(f"oracle mgrit: {STATUS.get(st, st)}")
        return out, its, hist, st

    def coarse_step(self, u, dt, m, level=1, coarse_kind=0, rtol=1e-14) -> np.ndarray:
        """One step of the MGRIT hierarchy's level-`level` propagator (fine
        step dt, coarsening m) on every grid: coarse_kind 0 backward Euler with
        dt m^level, 3 the two-stage SDIRK step of that size."""
        u = _f64(u)
        out = np.empty_like(u)
        st = lib().or_coarse_step(self._h, dt, m, level, coarse_kind, rtol, _p(u), _p(out))
        if st != 0:
            raise RuntimeError(f"oracle coarse_step: {STATUS.get(st, st)}")
        return out

    def combine(self, u, pts) -> np.ndarray:
        u = _f64(u)
        pts = _f64(pts).reshape(-1, self.d)
        out = np.empty(pts.shape[0])
        lib().or_combine(self._h, _p(u), pts.shape[0], _p(pts), _p(out))
        return out

    def interp(self, g: int, ug, pts) -> np.ndarray:
        ug = _f64(ug)
        pts = _f64(pts).reshape(-1, self.d)
        out = np.empty(pts.shape[0])
        lib().or_interp(self._h, g, _p(ug), pts.shape[0], _p(pts), _p(out))
        return out

    def hierarchize(self, u, inverse=False) -> np.ndarray:
        """Hierarchical surpluses of every grid's nodal values (inverse:
        nodal values from surpluses), Sec. 2.2.2."""
        u = _f64(u)
        out = np.empty_like(u)
        lib().or_hierarchize(self._h, _p(u), _p(out), 1 if inverse else 0)
        return out

    def recombine(self, u) -> np.ndarray:
        """Q u of Eq. "overall_combination_operator": hierarchize, combine
        the surpluses node by node over the grids that share the node, and
        dehierarchize."""
        u = _f64(u)
        out = np.empty_like(u)
        lib().or_recombine(self._h, _p(u), _p(out))
        return out

    def initial(self, kind: int, params) -> np.ndarray:
        params = _f64(params)
        out = np.empty(self.n_total)
        st = lib().or_initial(self._h, kind, _p(params), params.size, _p(out))
        if st != 0:
            raise ValueError("bad initial-value parameters")
        return out

    # learned coarse propagator (FP64 restatement of the network)
    @staticmethod
    def net_param_count() -> int:
        return int(lib().or_net_param_count())

    def net_forward(self, dT, theta, u) -> np.ndarray:
        u = _f64(u)
        nb = u.size // self.n_total
        out = np.empty_like(u)
        lib().or_net_forward(self._h, dT, _p(_f64(theta)), nb, _p(u), _p(out))
        return out

    def net_loss_grad(self, dT, theta, u, y):
        u, y = _f64(u), _f64(y)
        nb = u.size // self.n_total
        grad = np.empty(self.net_param_count())
        loss = lib().or_net_loss_grad(self._h, dT, _p(_f64(theta)), nb, _p(u), _p(y), _p(grad))
        return loss, grad

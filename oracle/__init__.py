"""FP64 CPU oracle for the points-as-tori SDF -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
never calls the CUDA library: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, POSIX threads
over queries); this module is a ctypes wrapper with numpy arrays.  Functions:

  Cloud(points, normals, params, weights=None)
                                        fit every torus (Sec. 4.1, App. C); the
                                        optional per-point weights A_i enter
                                        every blend (the area weights of Eq.
                                        SelfNormalizedConvolutionalDistanceFormula)
  Cloud.phi(x, C=64, ...)               shifted blend, Eqs. BasicFormulaShifted
                                        and RelationshipBetweenLambdaAndRadius
  Cloud.lse(x, C=64, ...)               log-sum-exp distance, Eq.
                                        ConvolutionalDistanceFormula (h = 1)
  Cloud.lse_grad(x, ...)                d~ and grad d~ (forward-mode duals)
  Cloud.sspd(x, ...)                    smoothed signed planar distance, Eq.
                                        SmoothedSignedPlanarDistance
  Cloud.shc(x, ...)                     signed Hopf-Cole distance, Eq.
                                        ScreenedWindingNumber
  Cloud.grad_x(x, ...)                  d phi / d x (forward-mode duals; App. D
                                        plus the x-dependence of lambda_x)
  Cloud.grad_params(x, G, ...)          d (sum_q G_q phi_q) / d a_i
  Cloud.g(i, x)                         g_i(x) = sign(T_i) phi_T(x), Eq. SingleTorusSDF
  Cloud.set_params(i, a)                refit point i's torus from new coefficients
  Cloud.laplacian(x, ...)               phi, grad phi and lap phi by second-order
                                        jets (App. D plus the x-dependence of lambda_x)
  Cloud.phi_radius(x, lam, ...)         radius-limited blend or log-sum-exp distance
                                        (Sec. 4.2, "Acceleration and adaptive lambda")
  Cloud.trace(org, dir, ...)            sphere tracing (Sec. 6)
  knn_mean_distance(points, k)          D of the lambda heuristic (Sec. 4.2)
  knn_mean_distance_sample(points, idx) its mean over sampled points only
  fit_record(p, n, a)                   the fitted torus of one point
  torus_sdf(c, u, R, r, x)              literal Eq. SingleTorusSDF for an explicit torus
  frame(n)                              the (s, t) frame convention

Submodules (numpy on top of the above): oracle.orient (orientation repair,
Sec. 6), oracle.mesh (marching tetrahedra of a phi grid, offset surfaces,
Sec. 6), oracle.morph (level-set sampling with normals, Sec. 6).

Parity status: every function is pinned (tests/test_oracle_*.py).  The blend
on noisy clouds with per-query lambda has no closed form; its pins are the
invariances of tests/test_oracle_invariances.py (rotations and reflections
with re-expressed coefficients, uniform scale, duplicated points, point
order, every normal flipped) beside the limits and exact cases of
tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

GLOBAL, FIXED = 0, 1
SHIFT_SIGMA, SHIFT_DMIN = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (-O2, IEEE double; no
    fast-math so the oracle keeps correctly rounded libm semantics)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        _lib.or_build.restype = P
        _lib.or_build.argtypes = [P, P, P, i64]
        _lib.or_free.argtypes = [P]
        _lib.or_phi.argtypes = [P, i32, f64, f64, i32, P, i64, P, P, i32]
        _lib.or_grad_x.argtypes = [P, i32, f64, f64, P, i64, P, P, i32]
        _lib.or_grad_params.argtypes = [P, i32, f64, f64, P, i64, P, P, i32]
        _lib.or_g.argtypes = [P, i64, P, i64, P]
        _lib.or_trace.argtypes = [P, i32, f64, f64, P, P, i64, i32, f64, f64, f64, P, P, i32]
        _lib.or_fit_record.argtypes = [P, P, P, P]
        _lib.or_torus_sdf.argtypes = [P, P, f64, f64, P, i64, P]
        _lib.or_frame.argtypes = [P, P, P]
        _lib.or_phi_radius.argtypes = [P, f64, f64, i32, P, i64, P, P, i32, i32]
        _lib.or_set_weights.argtypes = [P, P]
        _lib.or_set_weights.restype = i32
        _lib.or_set_params.argtypes = [P, i64, P]
        _lib.or_baseline.argtypes = [P, i32, i32, f64, f64, P, i64, P, P, i32]
        _lib.or_set_params.restype = i32
        _lib.or_lse.argtypes = [P, i32, f64, f64, P, i64, P, i32]
        _lib.or_lse_grad.argtypes = [P, i32, f64, f64, P, i64, P, P, i32]
        _lib.or_laplacian.argtypes = [P, i32, f64, f64, P, i64, P, P, P, i32]
        _lib.or_knn_mean_distance.argtypes = [P, i64, i32, i32]
        _lib.or_knn_mean_distance.restype = f64
        _lib.or_knn_mean_distance_sample.argtypes = [P, i64, P, i64, i32, i32]
        _lib.or_knn_mean_distance_sample.restype = f64
    return _lib


def _f64(a, cols=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


class Cloud:
    """A fitted cloud held by the oracle."""

    def __init__(self, points, normals, params, weights=None):
        lib = _load()
        self._p = _f64(points, 3)
        self._n = _f64(normals, 3)
        self._a = _f64(params, 6)
        n = self._p.shape[0]
        if self._n.shape[0] != n or self._a.shape[0] != n:
            raise ValueError("points, normals and params must have the same length")
        self._h = lib.or_build(_ptr(self._p), _ptr(self._n), _ptr(self._a), n)
        if not self._h:
            raise ValueError("oracle build rejected the cloud (empty, or a zero / non-finite normal)")
        self.n = n
        self._w = None
        if weights is not None:
            self._w = _f64(weights).ravel()
            if self._w.shape[0] != n or lib.or_set_weights(self._h, _ptr(self._w)) != 0:
                raise ValueError("weights: one finite value > 0 per point")

    def set_params(self, i: int, a):
        """Replaces point i's six coefficients and refits its torus (for finite
        differences of phi in the coefficients)."""
        a = _f64(a).ravel()
        if a.shape[0] != 6 or _load().or_set_params(self._h, int(i), _ptr(a)) != 0:
            raise ValueError("set_params: six coefficients and a point index in range")

    def __del__(self):
        if getattr(self, "_h", None):
            _load().or_free(self._h)
            self._h = None

    def phi(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0,
            shift: int = SHIFT_SIGMA, threads: int | None = None, stats: bool = False):
        x = _f64(x, 3)
        m = x.shape[0]
        out = np.empty(m)
        st = np.empty((m, 5)) if stats else None
        _load().or_phi(self._h, mode, C, lam, shift, _ptr(x), m, _ptr(out),
                       _ptr(st) if stats else None, threads or default_threads())
        return (out, st) if stats else out

    def laplacian(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0, threads: int | None = None):
        """(phi, grad phi, lap phi) by second-order jets through the definition
        (App. D; lambda_x(x) included for GLOBAL)."""
        x = _f64(x, 3)
        m = x.shape[0]
        phi, g, lap = np.empty(m), np.empty((m, 3)), np.empty(m)
        _load().or_laplacian(self._h, mode, C, lam, _ptr(x), m, _ptr(phi), _ptr(g), _ptr(lap),
                             threads or default_threads())
        return phi, g, lap

    def lse(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0, threads: int | None = None):
        """Log-sum-exp distance -(1/lambda) log sum_i A_i exp(-lambda |x - p_i|)
        (Eq. ConvolutionalDistanceFormula with h = 1), lambda as in phi."""
        x = _f64(x, 3)
        out = np.empty(x.shape[0])
        _load().or_lse(self._h, mode, C, lam, _ptr(x), x.shape[0], _ptr(out), threads or default_threads())
        return out

    def sspd(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0, threads: int | None = None):
        """Smoothed signed planar distance (Eq. SmoothedSignedPlanarDistance):
        the self-normalised blend of <x - p_i, n_i>, lambda as in phi."""
        x = _f64(x, 3)
        out = np.empty(x.shape[0])
        _load().or_baseline(self._h, 0, mode, C, lam, _ptr(x), x.shape[0], _ptr(out), None,
                            threads or default_threads())
        return out

    def shc(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0, threads: int | None = None,
            cond: bool = False):
        """Signed Hopf-Cole distance (Eq. ScreenedWindingNumber): sign(w)
        (-(1/lambda) log|w| + sigma_x) of the screened double-layer sum w,
        lambda as in phi.  cond: also sum |terms| / |w| per query."""
        x = _f64(x, 3)
        out = np.empty(x.shape[0])
        c = np.empty(x.shape[0]) if cond else None
        _load().or_baseline(self._h, 1, mode, C, lam, _ptr(x), x.shape[0], _ptr(out), _ptr(c) if cond else None,
                            threads or default_threads())
        return (out, c) if cond else out

    def lse_grad(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0, threads: int | None = None):
        """(d~, grad d~) by forward-mode duals through the definition, the
        x-dependence of lambda_x included (GLOBAL)."""
        x = _f64(x, 3)
        out, g = np.empty(x.shape[0]), np.empty((x.shape[0], 3))
        _load().or_lse_grad(self._h, mode, C, lam, _ptr(x), x.shape[0], _ptr(out), _ptr(g),
                            threads or default_threads())
        return out, g

    def phi_radius(self, x, lam: float, reval: float | None = None, C: float = 64.0, kfb: int = 32,
                   threads: int | None = None, used: bool = False, lse: bool = False):
        """Radius-limited blend (Sec. 4.2, "Acceleration and adaptive lambda"):
        constant lambda, the points within R_eval (default 2 C / lambda), else
        the kfb nearest.  used: also return, per query, the number of points
        inside R_eval (or minus the number of fallback neighbours).  lse: the
        log-sum-exp distance of the same set instead of the blend."""
        x = _f64(x, 3)
        m = x.shape[0]
        if reval is None:
            reval = 2.0 * C / lam
        out = np.empty(m)
        u = np.empty(m) if used else None
        _load().or_phi_radius(self._h, float(lam), float(reval), int(kfb), _ptr(x), m, _ptr(out),
                              _ptr(u) if used else None, threads or default_threads(), int(lse))
        return (out, u) if used else out

    def grad_x(self, x, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0,
               threads: int | None = None):
        x = _f64(x, 3)
        m = x.shape[0]
        phi = np.empty(m)
        g = np.empty((m, 3))
        _load().or_grad_x(self._h, mode, C, lam, _ptr(x), m, _ptr(phi), _ptr(g), threads or default_threads())
        return phi, g

    def grad_params(self, x, G, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0,
                    threads: int | None = None):
        x = _f64(x, 3)
        G = _f64(G).ravel()
        out = np.empty((self.n, 6))
        _load().or_grad_params(self._h, mode, C, lam, _ptr(x), x.shape[0], _ptr(G), _ptr(out),
                               threads or default_threads())
        return out

    def g(self, i: int, x):
        x = _f64(x, 3)
        out = np.empty(x.shape[0])
        _load().or_g(self._h, int(i), _ptr(x), x.shape[0], _ptr(out))
        return out

    def trace(self, org, dirs, max_steps: int = 48, eps: float = 1e-4, t_max: float = 6.0,
              offset: float = 0.0, C: float = 64.0, mode: int = GLOBAL, lam: float = 0.0,
              threads: int | None = None):
        org, dirs = _f64(org, 3), _f64(dirs, 3)
        m = org.shape[0]
        th = np.empty(m)
        steps = np.empty(m, dtype=np.int32)
        _load().or_trace(self._h, mode, C, lam, _ptr(org), _ptr(dirs), m, max_steps, eps, t_max, offset,
                         _ptr(th), _ptr(steps), threads or default_threads())
        return th, steps


FIT_FIELDS = {"q": slice(0, 3), "nstar": slice(3, 6), "vmin": slice(6, 9), "u": slice(9, 12),
              "c": slice(12, 15), "R": 15, "r": 16, "kmin": 17, "kmax": 18, "kplus": 19,
              "kminus": 20, "H": 21, "K": 22, "sign": 23, "flat": 24, "plane": 25}


def knn_mean_distance(points, k: int = 64, threads: int | None = None) -> float:
    """D of the paper's lambda heuristic (lambda = 10^3 / D): the mean distance
    between a point and its k nearest other points, averaged over the cloud
    (Sec. 4.2, "Acceleration and adaptive lambda").  Brute force, FP64."""
    p = _f64(points, 3)
    return float(_load().or_knn_mean_distance(_ptr(p), p.shape[0], int(k), threads or default_threads()))


def knn_mean_distance_sample(points, idx, k: int = 64, threads: int | None = None) -> float:
    """The same mean over the points idx only (each against all points): an
    estimate of D for clouds too large for the all-points brute force."""
    p = _f64(points, 3)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
    if ix.size == 0 or ix.min() < 0 or ix.max() >= p.shape[0]:
        raise ValueError("idx: indices of points")
    return float(_load().or_knn_mean_distance_sample(_ptr(p), p.shape[0], _ptr(ix), ix.size, int(k),
                                                     threads or default_threads()))


def fit_record(p, n, a) -> dict:
    p, n, a = _f64(p).ravel(), _f64(n).ravel(), _f64(a).ravel()
    out = np.zeros(32)
    _load().or_fit_record(_ptr(p), _ptr(n), _ptr(a), _ptr(out))
    return {k: (out[v].copy() if isinstance(v, slice) else float(out[v])) for k, v in FIT_FIELDS.items()}


def torus_sdf(c, u, R: float, r: float, x):
    c, u, x = _f64(c).ravel(), _f64(u).ravel(), _f64(x, 3)
    out = np.empty(x.shape[0])
    _load().or_torus_sdf(_ptr(c), _ptr(u), float(R), float(r), _ptr(x), x.shape[0], _ptr(out))
    return out


def frame(n):
    n = _f64(n).ravel()
    s, t = np.empty(3), np.empty(3)
    _load().or_frame(_ptr(n), _ptr(s), _ptr(t))
    return s, t

"""Python access to the FP64 CPU oracle (oracle/gpss_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA library ``paper_0902_4424_gb300`` and never
imports it.

Pins (what checks the oracle against something other than itself) live in
``tests/test_oracle_pins.py``:
  * ``project``      - brute force over supports and signs (tiny p), identity
                       inside the ball, exact l1 norm on the boundary,
                       variational inequality;
  * ``gpss``         - closed form for orthonormal K, brute force over supports
                       and signs for tiny p, FISTA on eq. 1 at the lambda that
                       corresponds to rho (relation of Sec. 1), KKT sign
                       conditions on every configuration, Armijo/feasibility
                       invariants, a hand-derived trace on a diagonal problem;
  * ``certificates`` - closed-form values on the orthonormal problem.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_SRC = [os.path.join(_HERE, "gpss_oracle.c")]

STOP_NAMES = {0: "rel_gap", 1: "stationary", 2: "fw", 3: "max_iter", 4: "linesearch",
              5: "nonfinite", 6: "stagnation"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C, OpenMP; no target-specific flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    srcs = list(_SRC)
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "gpss_oracle.h")])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("theta", ctypes.c_double), ("M", ctypes.c_int),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("tau1", ctypes.c_double), ("M_alpha", ctypes.c_int), ("tol", ctypes.c_double),
                ("f_star", ctypes.c_double), ("stop_fw", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_backtracks", ctypes.c_int), ("stagnation", ctypes.c_int),
                ("alpha0_rule", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("stop", ctypes.c_int), ("iters", ctypes.c_int), ("backtracks", ctypes.c_int),
                ("f", ctypes.c_double), ("lambda_reg", ctypes.c_double), ("l1", ctypes.c_double),
                ("fw_gap", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.ora_project_l1.restype = ctypes.c_double
        _lib.ora_residual.restype = ctypes.c_double
        _lib.ora_gpss.restype = ctypes.c_int
        _lib.ora_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_params(**kw) -> Params:
    prm = Params()
    lib().ora_params_default(ctypes.byref(prm))
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


def num_threads() -> int:
    return int(lib().ora_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (for a single-threaded timing)."""
    lib().ora_set_threads(ctypes.c_int(int(n)))


def project(v, rho: float):
    """Euclidean projection onto the l1 ball of radius rho; returns (w, tau)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty_like(v)
    tau = lib().ora_project_l1(_p(v), _p(out), ctypes.c_long(v.size), ctypes.c_double(rho))
    return out, float(tau)


def _kargs(prob):
    K = np.ascontiguousarray(prob.K)
    return K, (_p(K), ctypes.c_int(prob.dtype), ctypes.c_long(prob.n), ctypes.c_long(prob.p),
               ctypes.c_long(prob.ldk))


def objective(prob, x) -> float:
    """f(x) = ||K x - y||^2 in FP64 on the stored K."""
    K, ka = _kargs(prob)
    y = np.ascontiguousarray(prob.y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty(prob.n)
    return float(lib().ora_residual(*ka, _p(y), _p(x), _p(r)))


def certificates(prob, x):
    """(f, lambda, fw_gap, g) at x: lambda = max|K^T(y-Kx)|, fw = g^T x + rho ||g||_inf."""
    K, ka = _kargs(prob)
    y = np.ascontiguousarray(prob.y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    f, lam, fw = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    g = np.empty(prob.p)
    lib().ora_certificates(*ka, _p(y), ctypes.c_double(prob.rho), _p(x), ctypes.byref(f),
                           ctypes.byref(lam), ctypes.byref(fw), _p(g))
    return f.value, lam.value, fw.value, g


def gpss(prob, x0=None, trace: bool = False, **params):
    """Run Algorithm GP + SS on a workloads.Problem; returns (x, Result, trace or None)."""
    K, ka = _kargs(prob)
    y = np.ascontiguousarray(prob.y, dtype=np.float64)
    x = np.zeros(prob.p) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    prm = default_params(**params)
    res = Result()
    tr = np.zeros((max(prm.max_iter, 1), 4)) if trace else None
    lib().ora_gpss(*ka, _p(y), ctypes.c_double(prob.rho), _p(x), ctypes.byref(prm),
                   ctypes.byref(res), _p(tr) if trace else None)
    if trace:
        tr = tr[: res.iters + (1 if res.stop == 4 else 0)]
    return x, res, tr


def reference_solve(prob, tol: float = 1e-13, max_iter: int = 200000):
    """Solve eq. 2 to the oracle's precision floor: FW certificate <= tol, or stagnation."""
    return gpss(prob, stop_fw=1, tol=tol, max_iter=max_iter, stagnation=30)


def floor_solve(prob, max_iter: int = 20000):
    """Faster reference: iterate until the line search can no longer decrease f in
    FP64 (20 reductions of the step fail), i.e. until f sits at the FP64 floor."""
    return gpss(prob, stop_fw=1, tol=1e-12, stagnation=5, max_backtracks=20, max_iter=max_iter)

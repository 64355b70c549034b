"""Python binding of libgpl1 (include/gpl1.h): GPSS on one GB300 GPU.

Argument marshalling only.  Tensors supply device pointers and PyTorch's
current stream supplies the CUDA stream; every step of the method runs in the
library's CUDA kernels.  There is no CPU path: if the compiled library is
missing, every call raises.

Names follow the C ABI: ``Context.project`` -> ``gpl1_project``,
``Context.solve`` -> ``gpl1_solve``, ``Context.solve_batched`` ->
``gpl1_solve_batched``, ``params_default`` -> ``gpl1_params_default``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libgpl1.so")

F64, F32, BF16 = 0, 1, 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NOT_CONVERGED", 4: "LINESEARCH", 5: "NONFINITE",
          6: "TIMEOUT", 7: "UNSUPPORTED"}
STOP = {0: "rel_gap", 1: "stationary", 2: "fw", 3: "max_iter", 4: "error", 5: "stagnation"}
STOP_ON_REL_GAP, STOP_ON_FW = 1, 2
DEBUG_UNREACHABLE_BARRIER = 1
ENGINE_AUTO, ENGINE_ONE_READ, ENGINE_TWO_PASS, ENGINE_ONE_READ_NCH2, ENGINE_ONE_READ_NCH4 = 0, 1, 2, 3, 4
METHOD_GPSS, METHOD_ISTA, METHOD_FISTA, METHOD_PSD = 0, 1, 2, 3
TILE_AUTO, TILE_SMALL, TILE_MEDIUM, TILE_LARGE = 0, 1, 2, 3
TRACE_COLS = 28
# statuses that describe how a solve ended (reported in Result.status, not raised)
ALGORITHMIC = (0, 3, 4, 5, 6)

EXPORTS = ["gpl1_create", "gpl1_destroy", "gpl1_set_stream", "gpl1_last_error", "gpl1_params_default",
           "gpl1_project", "gpl1_solve", "gpl1_solve_batched", "gpl1_solve_noalloc", "gpl1_gemm_bf16",
           "gpl1_gemm_bf16_ex", "gpl1_gemm_tuned", "gpl1_gemm_tuned_set", "gpl1_solve_shared_k", "gpl1_lista_forward",
           "gpl1_lista_grad", "gpl1_lista_train", "gpl1_plan_create", "gpl1_plan_run", "gpl1_plan_destroy",
           "gpl1_solve_async", "gpl1_solve_batched_async", "gpl1_spectral_norm_sq", "gpl1_lista_init",
           "gpl1_solve_warm", "gpl1_solve_tuned", "gpl1_batched_tuned"]


class Gpl1Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"gpl1 {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("theta", ctypes.c_double), ("M", ctypes.c_int),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double), ("tau1", ctypes.c_double),
                ("M_alpha", ctypes.c_int), ("tol", ctypes.c_double), ("f_star", ctypes.c_double),
                ("stop_rule", ctypes.c_int), ("max_iter", ctypes.c_int), ("max_backtracks", ctypes.c_int),
                ("alpha0_rule", ctypes.c_int), ("x0_is_zero", ctypes.c_int), ("debug", ctypes.c_int),
                ("timeout_ns", ctypes.c_longlong), ("engine", ctypes.c_int), ("method", ctypes.c_int),
                ("lambda_pen", ctypes.c_double), ("step", ctypes.c_double), ("tile", ctypes.c_int),
                ("tile_pad", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("stop", ctypes.c_int), ("iters", ctypes.c_int),
                ("backtracks", ctypes.c_int), ("f", ctypes.c_double), ("rel_gap", ctypes.c_double),
                ("fw_gap", ctypes.c_double), ("lambda_", ctypes.c_double), ("alpha", ctypes.c_double),
                ("tau", ctypes.c_double), ("kernel_ms", ctypes.c_double), ("fail_site", ctypes.c_int),
                ("fail_iter", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Problem(ctypes.Structure):
    _fields_ = [("K", ctypes.c_void_p), ("n", ctypes.c_longlong), ("p", ctypes.c_longlong),
                ("ldk", ctypes.c_longlong), ("y", ctypes.c_void_p), ("rho", ctypes.c_double),
                ("x", ctypes.c_void_p), ("f_star", ctypes.c_double), ("trace", ctypes.c_void_p),
                ("trace_cap", ctypes.c_longlong)]


_lib = None


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
        L = ctypes.CDLL(LIB_PATH)
        L.gpl1_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
        L.gpl1_destroy.argtypes = [ctypes.c_void_p]
        L.gpl1_destroy.restype = None
        L.gpl1_set_stream.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.gpl1_last_error.argtypes = [ctypes.c_void_p]
        L.gpl1_last_error.restype = ctypes.c_char_p
        L.gpl1_params_default.argtypes = [ctypes.POINTER(Params)]
        L.gpl1_params_default.restype = None
        L.gpl1_project.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong,
                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
        L.gpl1_solve.argtypes = [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.c_int,
                                 ctypes.POINTER(Params), ctypes.POINTER(Result)]
        L.gpl1_solve_batched.argtypes = [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(Params), ctypes.POINTER(Result)]
        L.gpl1_gemm_bf16.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong,
                                     ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong,
                                     ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_float]
        L.gpl1_solve_async.argtypes = [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.c_int,
                                       ctypes.POINTER(Params), ctypes.c_void_p]
        L.gpl1_solve_batched_async.argtypes = [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(Params), ctypes.c_void_p]
        L.gpl1_plan_create.argtypes = [ctypes.c_void_p, ctypes.POINTER(Problem), ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]
        L.gpl1_plan_run.argtypes = [ctypes.c_void_p, ctypes.POINTER(Result)]
        L.gpl1_plan_destroy.argtypes = [ctypes.c_void_p]
        L.gpl1_plan_destroy.restype = None
        L.gpl1_gemm_bf16_ex.argtypes = L.gpl1_gemm_bf16.argtypes + [ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
        L.gpl1_gemm_tuned.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_float)]
        L.gpl1_gemm_tuned.restype = ctypes.c_int
        L.gpl1_solve_tuned.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        L.gpl1_solve_tuned.restype = ctypes.c_int
        L.gpl1_batched_tuned.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        L.gpl1_batched_tuned.restype = ctypes.c_int
        L.gpl1_gemm_tuned_set.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                          ctypes.c_int]
        L.gpl1_solve_shared_k.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong,
                                          ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                          ctypes.POINTER(Params), ctypes.POINTER(Result)]
        vp, ll, ci, cf = ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_float
        L.gpl1_lista_forward.argtypes = [vp, vp, ll, ll, ll, ci, vp, vp, vp, ll, ll, vp, ll]
        L.gpl1_lista_grad.argtypes = [vp, vp, ll, ll, ll, ci, vp, vp, vp, ll, ll, vp, ll, vp, vp,
                                      ctypes.POINTER(ctypes.c_double)]
        L.gpl1_lista_train.argtypes = [vp, vp, ll, ll, ll, ci, vp, vp, vp, vp, vp, ll, vp, ll, ll, ll, ci, ci, cf, cf,
                                       vp]
        L.gpl1_spectral_norm_sq.argtypes = [vp, vp, ci, ll, ll, ll, ci, ctypes.POINTER(ctypes.c_double)]
        L.gpl1_lista_init.argtypes = [vp, vp, ll, ll, ll, ci, vp, ll, ci, vp, vp, ctypes.POINTER(ctypes.c_double)]
        L.gpl1_solve_warm.argtypes = [vp, vp, ll, ll, ll, ci, vp, vp, vp, ll, vp, vp, vp, ll, ci,
                                      ctypes.POINTER(Params), ci, ctypes.POINTER(Result), vp,
                                      ctypes.POINTER(ctypes.c_int)]
        L.gpl1_solve_noalloc.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(Params),
                                         ctypes.POINTER(Result), ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
        _lib = L
    return _lib


def params_default(**overrides) -> Params:
    prm = Params()
    lib().gpl1_params_default(ctypes.byref(prm))
    for k, v in overrides.items():
        if not hasattr(prm, k):
            raise KeyError(k)
        setattr(prm, k, v)
    return prm


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    if t.dtype in (torch.bfloat16, torch.int16, torch.uint16):
        return BF16
    raise TypeError(f"unsupported K dtype {t.dtype}")


def _stream_handle(device=None):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _same_device(device, *tensors):
    """Raise unless every tensor lives on CUDA device index `device`."""
    for t in tensors:
        if t is None:
            continue
        if not t.is_cuda or t.device.index != device:
            raise ValueError(f"tensor on {t.device}, expected cuda:{device}")


class Context:
    """A gpl1 context on one CUDA device (``gpl1_create``)."""

    def __init__(self, device: int | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gpl1 needs a CUDA GPU")
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        st = lib().gpl1_create(ctypes.byref(h), self.device, _stream_handle(self.device))
        if st != 0:
            raise Gpl1Error(st, "gpl1_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().gpl1_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise Gpl1Error(st, lib().gpl1_last_error(self._h).decode())

    def _bind_stream(self):
        """Bind the context to PyTorch's current stream of the context's device."""
        lib().gpl1_set_stream(self._h, _stream_handle(self.device))

    # ------------------------------------------------------------ project
    def project(self, v, rho, out=None, tau=None):
        """Project each row of v (p,) or (batch, p) onto {||w||_1 <= rho_b}; returns out."""
        import torch
        v2 = v if v.dim() == 2 else v.view(1, -1)
        batch, p = v2.shape
        if v2.stride(1) != 1:
            raise ValueError("rows of v must be contiguous")
        out = torch.empty_like(v2) if out is None else out.view(batch, p)
        code = _dtype_code(v2)
        if isinstance(rho, torch.Tensor) and rho.is_cuda:
            rho_ptr, on_dev = ctypes.c_void_p(rho.data_ptr()), 1
            keep = rho
        else:
            vals = [float(rho)] * batch if not isinstance(rho, (list, tuple, torch.Tensor)) else \
                [float(r) for r in (rho.tolist() if isinstance(rho, torch.Tensor) else rho)]
            keep = (ctypes.c_double * batch)(*vals)
            rho_ptr, on_dev = ctypes.cast(keep, ctypes.c_void_p), 0
        self._bind_stream()
        st = lib().gpl1_project(self._h, ctypes.c_void_p(v2.data_ptr()), ctypes.c_void_p(out.data_ptr()), code,
                                p, batch, v2.stride(0), rho_ptr, on_dev,
                                ctypes.c_void_p(tau.data_ptr()) if tau is not None else None)
        del keep
        self._check(st)
        return out.view_as(v)

    # --------------------------------------------------------------- gemm
    def gemm_bf16(self, A, B, Kd=None, out=None, scale=1.0):
        """gpl1_gemm_bf16: out (N, M) FP32 with out[n, m] = scale * sum_k A[m, k % Ka] B[n, k].
        A (M, Ka) and B (N, Kd) are bfloat16 (or int16 bit patterns), K contiguous."""
        import torch
        M, Ka = A.shape
        N, Kb = B.shape
        Kd = Kb if Kd is None else int(Kd)
        out = torch.empty(N, M, dtype=torch.float32, device=A.device) if out is None else out
        self._bind_stream()
        st = lib().gpl1_gemm_bf16(self._h, ctypes.c_void_p(A.data_ptr()), M, Ka, A.stride(0),
                                  ctypes.c_void_p(B.data_ptr()), N, Kd, B.stride(0),
                                  ctypes.c_void_p(out.data_ptr()), out.stride(0), float(scale))
        self._check(st)
        return out

    def gemm_bf16_ex(self, A, B, config, splits, Kd=None, scale=1.0):
        """gpl1_gemm_bf16_ex: the same product with kernel configuration `config` and the
        contraction split into `splits` parts; returns the parts, (splits, N, M) FP32."""
        import torch
        M, Ka = A.shape
        N, Kb = B.shape
        Kd = Kb if Kd is None else int(Kd)
        out = torch.empty(splits, N, M, dtype=torch.float32, device=A.device)
        self._bind_stream()
        st = lib().gpl1_gemm_bf16_ex(self._h, ctypes.c_void_p(A.data_ptr()), M, Ka, A.stride(0),
                                     ctypes.c_void_p(B.data_ptr()), N, Kd, B.stride(0),
                                     ctypes.c_void_p(out.data_ptr()), out.stride(1), float(scale),
                                     int(config), int(splits), out.stride(0))
        self._check(st)
        return out

    def gemm_tuned(self):
        """The autotuner's choices: [{shape: (M, N, Kd, Ka, max_splits), config, splits, ms}]."""
        L = lib()
        count = L.gpl1_gemm_tuned(self._h, 0, None, None, None, None)
        out = []
        for i in range(max(count, 0)):
            shp = (ctypes.c_longlong * 5)()
            cfg, spl, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
            L.gpl1_gemm_tuned(self._h, i, shp, ctypes.byref(cfg), ctypes.byref(spl), ctypes.byref(ms))
            out.append({"shape": tuple(shp), "config": cfg.value, "splits": spl.value, "ms": ms.value})
        return out

    def solve_tuned(self):
        """The single-solve autotuner's choices: [{shape: (dtype, n, p, class), engine, ms}]."""
        L = lib()
        count = L.gpl1_solve_tuned(self._h, 0, None, None, None)
        out = []
        for i in range(max(count, 0)):
            shp = (ctypes.c_longlong * 4)()
            eng, ms = ctypes.c_int(), ctypes.c_float()
            L.gpl1_solve_tuned(self._h, i, shp, ctypes.byref(eng), ctypes.byref(ms))
            out.append({"shape": tuple(shp), "engine": eng.value, "ms": ms.value})
        return out

    def batched_tuned(self):
        """The batched autotuner's choices: [{key: (dtype, count, sum n p, max n p), tile, ms: (S, M, L)}]."""
        L = lib()
        count = L.gpl1_batched_tuned(self._h, 0, None, None, None)
        out = []
        for i in range(max(count, 0)):
            key = (ctypes.c_longlong * 4)()
            tile, ms = ctypes.c_int(), (ctypes.c_float * 3)()
            L.gpl1_batched_tuned(self._h, i, key, ctypes.byref(tile), ms)
            out.append({"key": tuple(key), "tile": tile.value, "ms": tuple(ms)})
        return out

    def gemm_tuned_set(self, shape, config, splits):
        """gpl1_gemm_tuned_set: pin (config, splits) for shape (M, N, Kd, Ka, max_splits)."""
        shp = (ctypes.c_longlong * 5)(*[int(v) for v in shape])
        self._check(lib().gpl1_gemm_tuned_set(self._h, shp, int(config), int(splits)))

    # ------------------------------------------------ learned warm start
    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    def spectral_norm_sq(self, K, dtype, p=None, iters=100):
        """gpl1_spectral_norm_sq: ||K||_2^2 of the n x p matrix K (n x ldk storage)."""
        n, ldk = K.shape
        out = ctypes.c_double()
        self._bind_stream()
        self._check(lib().gpl1_spectral_norm_sq(self._h, self._ptr(K), int(dtype), n, ldk if p is None else int(p),
                                                ldk, int(iters), ctypes.byref(out)))
        return out.value

    def lista_init(self, K, layers, lambdas, p=None, power_iters=100, W=None, theta=None):
        """gpl1_lista_init: (W (layers, p, n), theta (layers), L) with W_l = K^T / L and
        theta_l = median(lambdas) / L, L = ||K||_2^2."""
        import torch
        n, ldk = K.shape
        p = ldk if p is None else int(p)
        W = torch.empty(layers, p, n, dtype=torch.float32, device=K.device) if W is None else W
        theta = torch.empty(layers, dtype=torch.float32, device=K.device) if theta is None else theta
        lam = (ctypes.c_double * len(lambdas))(*[float(v) for v in lambdas])
        L = ctypes.c_double()
        self._bind_stream()
        self._check(lib().gpl1_lista_init(self._h, self._ptr(K), n, p, ldk, int(layers), ctypes.cast(lam, ctypes.c_void_p),
                                          len(lambdas), int(power_iters), self._ptr(W), self._ptr(theta),
                                          ctypes.byref(L)))
        return W, theta, L.value

    def solve_warm(self, K, W, theta, Y, rho, f_star=None, params: Params | None = None, warm_max_iter=0, X=None):
        """gpl1_solve_warm: the network's output as x0 for Alg. GP on every row of Y (nrhs, n),
        the cold solve as the fallback; returns (X, [Result], fell_back list, fallbacks)."""
        import torch
        n, ldk = K.shape
        layers, p, _ = W.shape
        nrhs = Y.shape[0]
        X = torch.empty(nrhs, p, dtype=torch.float32, device=K.device) if X is None else X
        _same_device(self.device, K, W, theta, Y, X)
        prm = params_default() if params is None else params
        rho_h = (ctypes.c_double * nrhs)(*[float(r) for r in rho])
        fs_h = None if f_star is None else (ctypes.c_double * nrhs)(*[float(f) for f in f_star])
        res = (Result * nrhs)()
        fb = (ctypes.c_int * nrhs)()
        nfb = ctypes.c_int()
        self._bind_stream()
        self._check(lib().gpl1_solve_warm(self._h, self._ptr(K), n, p, ldk, layers, self._ptr(W), self._ptr(theta),
                                          self._ptr(Y), Y.stride(0), ctypes.cast(rho_h, ctypes.c_void_p),
                                          None if fs_h is None else ctypes.cast(fs_h, ctypes.c_void_p), self._ptr(X),
                                          X.stride(0), nrhs, ctypes.byref(prm), int(warm_max_iter), res,
                                          ctypes.cast(fb, ctypes.c_void_p), ctypes.byref(nfb)))
        return X, list(res), list(fb), nfb.value

    def lista_forward(self, K, W, theta, Y, p=None, X=None):
        """gpl1_lista_forward: x^L (B, p) float32 for right-hand sides Y (B, n)."""
        import torch
        n, ldk = K.shape
        layers, pp, nn = W.shape
        p = pp if p is None else int(p)
        B = Y.shape[0]
        X = torch.empty(B, p, dtype=torch.float32, device=Y.device) if X is None else X
        self._bind_stream()
        self._check(lib().gpl1_lista_forward(self._h, self._ptr(K), n, p, ldk, layers, self._ptr(W), self._ptr(theta),
                                             self._ptr(Y), Y.stride(0), B, self._ptr(X), X.stride(0)))
        return X

    def lista_grad(self, K, W, theta, Y, Xt):
        """gpl1_lista_grad: (loss, dW, dtheta) of mean ||x^L - Xt||^2 over the batch."""
        import torch
        n, ldk = K.shape
        layers, p, _ = W.shape
        dW = torch.empty_like(W)
        dth = torch.empty_like(theta)
        loss = ctypes.c_double()
        self._bind_stream()
        self._check(lib().gpl1_lista_grad(self._h, self._ptr(K), n, p, ldk, layers, self._ptr(W), self._ptr(theta),
                                          self._ptr(Y), Y.stride(0), Y.shape[0], self._ptr(Xt), Xt.stride(0),
                                          self._ptr(dW), self._ptr(dth), ctypes.byref(loss)))
        return loss.value, dW, dth

    def lista_train(self, K, W, theta, m, v, Y, Xt, batch, steps, t0=0, lr=1e-3, lr_theta=1e-3):
        """gpl1_lista_train: `steps` Adam updates of W, theta in place; returns the losses."""
        n, ldk = K.shape
        layers, p, _ = W.shape
        losses = (ctypes.c_double * steps)()
        self._bind_stream()
        self._check(lib().gpl1_lista_train(self._h, self._ptr(K), n, p, ldk, layers, self._ptr(W), self._ptr(theta),
                                           self._ptr(m), self._ptr(v), self._ptr(Y), Y.stride(0), self._ptr(Xt),
                                           Xt.stride(0), Y.shape[0], batch, steps, t0, float(lr), float(lr_theta),
                                           ctypes.cast(losses, ctypes.c_void_p)))
        return list(losses)

    # -------------------------------------------------------------- solve
    @staticmethod
    def make_problem(K, y, rho, x, p=None, f_star=-1.0, trace=None) -> Problem:
        n, ldk = K.shape
        return Problem(ctypes.c_void_p(K.data_ptr()), n, ldk if p is None else int(p), ldk,
                       ctypes.c_void_p(y.data_ptr()), float(rho), ctypes.c_void_p(x.data_ptr()), float(f_star),
                       ctypes.c_void_p(trace.data_ptr()) if trace is not None else None,
                       trace.shape[0] if trace is not None else 0)

    def solve(self, K, y, rho, x=None, p=None, params: Params | None = None, f_star: float = -1.0, trace=None):
        """Solve min ||Kx - y||^2 s.t. ||x||_1 <= rho (gpl1_solve); x (device) is x0 in, solution out.

        K: (n, ldk) tensor (float64, float32, or bfloat16 / int16 bit patterns); p <= ldk columns are used.
        trace: optional float64 device tensor (cap, TRACE_COLS) receiving one row per iteration.
        Returns (x, Result).
        """
        import torch
        code = _dtype_code(K)
        n, ldk = K.shape
        p = ldk if p is None else int(p)
        vdt = torch.float64 if code == F64 else torch.float32
        prm = params_default() if params is None else params
        if x is None:
            x = torch.zeros(p, dtype=vdt, device=K.device)
            prm = Params.from_buffer_copy(prm)
            prm.x0_is_zero = 1
        _same_device(self.device, K, y, x, trace)
        pr = self.make_problem(K, y, rho, x, p, f_star, trace)
        res = Result()
        self._bind_stream()
        st = lib().gpl1_solve(self._h, ctypes.byref(pr), code, ctypes.byref(prm), ctypes.byref(res))
        if st not in ALGORITHMIC:   # argument / CUDA errors raise; solver outcomes are in res.status
            self._check(st)
        return x, res

    def solve_shared_k(self, K, Y, rho, p=None, f_star=None, params: Params | None = None, X=None):
        """gpl1_solve_shared_k: instances sharing the BF16 K (n, ldk) with right-hand sides
        Y (nrhs, n) float32 and radii rho (nrhs); X (nrhs, p) float32 holds x0 when given
        (else x0 = 0); returns (X, [Result])."""
        import torch
        n, ldk = K.shape
        nrhs = Y.shape[0]
        p = ldk if p is None else int(p)
        prm = Params.from_buffer_copy(params_default() if params is None else params)
        if X is None:
            X = torch.empty(nrhs, p, dtype=torch.float32, device=K.device)
            prm.x0_is_zero = 1
        else:
            prm.x0_is_zero = 0
        rho_h = (ctypes.c_double * nrhs)(*[float(r) for r in rho])
        fs_h = None if f_star is None else (ctypes.c_double * nrhs)(*[float(f) for f in f_star])
        res = (Result * nrhs)()
        self._bind_stream()
        st = lib().gpl1_solve_shared_k(self._h, ctypes.c_void_p(K.data_ptr()), n, p, ldk,
                                       ctypes.c_void_p(Y.data_ptr()), Y.stride(0), ctypes.cast(rho_h, ctypes.c_void_p),
                                       ctypes.cast(fs_h, ctypes.c_void_p) if fs_h is not None else None,
                                       ctypes.c_void_p(X.data_ptr()), X.stride(0), nrhs, ctypes.byref(prm), res)
        if st not in ALGORITHMIC:
            self._check(st)
        return X, list(res)

    def plan_batched(self, problems: Sequence[Problem], dtype: int, params: Params | None = None):
        """gpl1_plan_create: the batched solve of these instances recorded once as a CUDA
        graph; BatchedPlan.run() replays it.  The tensors behind the descriptors must outlive
        the plan (their contents may change between runs)."""
        count = len(problems)
        arr = (Problem * count)(*problems)
        prm = params_default() if params is None else params
        h = ctypes.c_void_p()
        self._bind_stream()
        self._check(lib().gpl1_plan_create(self._h, arr, count, dtype, ctypes.byref(prm), ctypes.byref(h)))
        return BatchedPlan(self, h, count)

    def solve_batched_async(self, problems: Sequence[Problem], dtype: int, params: Params | None = None, res=None):
        """gpl1_solve_batched_async: enqueue on PyTorch's current stream without waiting.
        res: a uint8 device tensor of count * sizeof(Result) bytes (allocated when None);
        returns it.  Result.from_buffer_copy on res.cpu().numpy() reads the results."""
        import torch
        count = len(problems)
        arr = (Problem * count)(*problems)
        prm = params_default() if params is None else params
        if res is None:
            res = torch.empty(count * ctypes.sizeof(Result), dtype=torch.uint8, device="cuda")
        self._bind_stream()
        self._check(lib().gpl1_solve_batched_async(self._h, arr, count, dtype, ctypes.byref(prm),
                                                   ctypes.c_void_p(res.data_ptr())))
        return res

    @staticmethod
    def results_from_device(res, count: int):
        """Results written by an asynchronous solve (a uint8 device tensor) as Result objects."""
        raw = bytes(res.cpu().numpy().tobytes())
        size = ctypes.sizeof(Result)
        return [Result.from_buffer_copy(raw[i * size:(i + 1) * size]) for i in range(count)]

    def solve_batched(self, problems: Sequence[Problem], dtype: int, params: Params | None = None):
        """Solve independent instances in one persistent launch (gpl1_solve_batched); returns results."""
        count = len(problems)
        arr = (Problem * count)(*problems)
        res = (Result * count)()
        prm = params_default() if params is None else params
        self._bind_stream()
        st = lib().gpl1_solve_batched(self._h, arr, count, dtype, ctypes.byref(prm), res)
        if st not in ALGORITHMIC:
            self._check(st)
        return list(res)


class BatchedPlan:
    """A batched solve recorded as a CUDA graph (gpl1_plan_*); run() replays it."""

    def __init__(self, ctx: "Context", handle, count: int):
        self._ctx, self._h, self.count = ctx, handle, count

    def run(self):
        """Replay on the context's stream (bound to PyTorch's current stream); returns the results."""
        res = (Result * self.count)()
        self._ctx._bind_stream()
        st = lib().gpl1_plan_run(self._h, res)
        if st not in ALGORITHMIC:
            self._ctx._check(st)
        return list(res)

    def close(self):
        if self._h:
            lib().gpl1_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_SCRATCH_BYTES = 4 << 20


def solve_noalloc(K, y, rho, x=None, p=None, params: Params | None = None, f_star: float = -1.0):
    """gpl1_solve_noalloc: one solve with the library's static scratch instead of
    a context's workspace (no allocation inside the C call).  Same arguments as
    Context.solve; runs with K's device current and enqueues on PyTorch's
    current stream of that device.  Pass a preallocated x (x0 in, solution out)
    to keep this wrapper from allocating too; with x None it allocates a zero
    x through PyTorch before the call.
    Returns (x, Result); raises Gpl1Error on argument, size or CUDA errors."""
    import torch
    code = _dtype_code(K)
    n, ldk = K.shape
    p = ldk if p is None else int(p)
    prm = params_default() if params is None else params
    if x is None:
        x = torch.zeros(p, dtype=torch.float64 if code == F64 else torch.float32, device=K.device)
        prm = Params.from_buffer_copy(prm)
        prm.x0_is_zero = 1
    _same_device(K.device.index, K, y, x)
    pr = Context.make_problem(K, y, rho, x, p, f_star)
    res = Result()
    err = ctypes.create_string_buffer(256)
    with torch.cuda.device(K.device):
        st = lib().gpl1_solve_noalloc(ctypes.byref(pr), code, ctypes.byref(prm), ctypes.byref(res),
                                      _stream_handle(K.device), err, len(err))
    if st not in ALGORITHMIC:   # argument, size and CUDA errors raise; solver outcomes are in res.status
        raise Gpl1Error(st, err.value.decode())
    return x, res

"""Thin ctypes binding of ``libsmsm.so`` (include/smsm.h), same names as the C ABI.

Argument marshalling only: every step of the reconstruction runs in the
library's CUDA kernels.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: if the library is missing this module
raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmsm.so")

SMSM_OK, SMSM_ERR_ARG, SMSM_ERR_CUDA, SMSM_ERR_NOMEM = 0, 1, 2, 3
SMSM_ERR_DIVERGED, SMSM_ERR_NOT_PD, SMSM_ERR_TIMEOUT, SMSM_ERR_STATE = 4, 5, 6, 7
SMSM_ERR_EIG_UNCONVERGED = 8
SMSM_MODE_IRLS, SMSM_MODE_NULLSPACE = 0, 1
SMSM_FLAG_GENERIC_KERNELS = 1
SMSM_FLAG_PER_COIL_NORMAL = 2
SMSM_FLAG_CLUSTER_EIG = 4
SMSM_BOUNDARY_VALID = 0
SMSM_BOUNDARY_PERIODIC = 1
SMSM_PRECISION_FP32, SMSM_PRECISION_BF16_SPLIT = 0, 1
SMSM_MAX_OUTER = 128
STAGES = ["adjoint", "gram", "eig", "vapply", "weights", "filters", "rowfft_inv", "column", "rowfft_fwd",
          "band", "cg"]
STAGE = {name: k for k, name in enumerate(STAGES)}


class Opts(ctypes.Structure):
    _fields_ = [("caipi_div", ctypes.c_int), ("batch", ctypes.c_int), ("flags", ctypes.c_int),
                ("precision", ctypes.c_int), ("boundary", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("eps0_rel", ctypes.c_double), ("eta", ctypes.c_double),
                ("eps_min_rel", ctypes.c_double), ("outer_iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("mode", ctypes.c_int), ("rank", ctypes.c_int), ("warm", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("timing", ctypes.c_int), ("eig_cold", ctypes.c_int),
                ("lanes", ctypes.c_int), ("eig_tol", ctypes.c_float), ("reserved", ctypes.c_int * 2)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_done", ctypes.c_int),
                ("eps", ctypes.c_double * SMSM_MAX_OUTER), ("rr_start", ctypes.c_double * SMSM_MAX_OUTER),
                ("rr_end", ctypes.c_double * SMSM_MAX_OUTER), ("sweeps", ctypes.c_int * SMSM_MAX_OUTER),
                ("elapsed_ms", ctypes.c_float), ("graph_kernels", ctypes.c_int),
                ("stage_ms", ctypes.c_float * 16), ("stage_launches", ctypes.c_int * 16),
                ("lanes", ctypes.c_int), ("lane0_batch", ctypes.c_int)]


class TuneReport(ctypes.Structure):
    _fields_ = [("gram_nG", ctypes.c_int), ("n_gram", ctypes.c_int), ("gram_candidates", ctypes.c_int * 8),
                ("gram_ms", ctypes.c_float * 8), ("lanes", ctypes.c_int), ("lane_ms", ctypes.c_float * 4)]


class SmsmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"smsm status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsmsm.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, st = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    L.smsm_plan.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, ctypes.POINTER(Opts)]
    L.smsm_plan.restype = st
    L.smsm_plan_destroy.argtypes = [vp]
    L.smsm_plan_destroy.restype = st
    L.smsm_plan_workspace_bytes.argtypes = [vp]
    L.smsm_plan_workspace_bytes.restype = ctypes.c_size_t
    L.smsm_plan_set_sens.argtypes = [vp, vp, vp]
    L.smsm_plan_set_sens.restype = st
    for fn in ("smsm_forward", "smsm_adjoint"):
        getattr(L, fn).argtypes = [vp, vp, vp, vp, vp]
        getattr(L, fn).restype = st
    L.smsm_hankel_gram.argtypes = [vp, vp, vp, vp]
    L.smsm_hankel_gram.restype = st
    L.smsm_apply_filters.argtypes = [vp, vp, vp, vp, vp]
    L.smsm_apply_filters.restype = st
    L.smsm_reconstruct.argtypes = [vp, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(Report), vp]
    L.smsm_reconstruct.restype = st
    L.smsm_fft2c.argtypes = [vp, vp, vp, i, i, vp]
    L.smsm_fft2c.restype = st
    L.smsm_sense.argtypes = [vp, vp, vp, vp, i, ctypes.POINTER(Report), vp]
    L.smsm_sense.restype = st
    L.smsm_reconstruct_groups.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                          ctypes.POINTER(Params), ctypes.POINTER(Report), vp]
    L.smsm_reconstruct_groups.restype = st
    L.smsm_hankel_gram_noalloc.argtypes = [vp, vp, i, i, i, i, vp]
    L.smsm_hankel_gram_noalloc.restype = st
    L.smsm_plan_device_status.argtypes = [vp, vp]
    L.smsm_plan_device_status.restype = st
    L.smsm_last_error.argtypes = []
    L.smsm_last_error.restype = ctypes.c_char_p
    L.smsm_default_params.argtypes = [ctypes.POINTER(Params)]
    L.smsm_default_params.restype = None
    L.smsm_autotune.argtypes = [vp, vp, ctypes.POINTER(Params), ctypes.POINTER(TuneReport), vp]
    L.smsm_autotune.restype = st
    L.smsm_cnn_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i]
    L.smsm_cnn_create.restype = st
    L.smsm_cnn_destroy.argtypes = [vp]
    L.smsm_cnn_destroy.restype = st
    L.smsm_cnn_param_count.argtypes = [vp]
    L.smsm_cnn_param_count.restype = ctypes.c_size_t
    for fn in ("smsm_cnn_set_params", "smsm_cnn_get_params"):
        getattr(L, fn).argtypes = [vp, vp, vp]
        getattr(L, fn).restype = st
    L.smsm_cnn_forward.argtypes = [vp, vp, vp, i, vp]
    L.smsm_cnn_forward.restype = st
    dp = ctypes.POINTER(ctypes.c_double)
    L.smsm_cnn_gradients.argtypes = [vp, vp, vp, i, vp, dp, vp]
    L.smsm_cnn_gradients.restype = st
    L.smsm_cnn_train_step.argtypes = [vp, vp, vp, i, ctypes.c_float, dp, vp]
    L.smsm_cnn_train_step.restype = st
    L.smsm_learned_start.argtypes = [vp, vp, vp, vp, vp]
    L.smsm_learned_start.restype = st
    _lib = L
    return L


def _check(status: int) -> None:
    if status != SMSM_OK:
        raise SmsmError(status, lib().smsm_last_error().decode())


def reconstruct_groups(plans, ys, params: Params | None = None, report: bool = True, xs=None):
    """Solve independent groups of possibly different geometry together (one plan each, one
    graph launch): returns ([x_k], [Report_k] or None).  xs: output tensors to reuse (they
    also hold the warm starts when params.warm is set)."""
    n = len(plans)
    if params is None:
        params = default_params()
    if xs is None:
        xs = [torch.empty(p.x_shape, dtype=torch.complex64, device=y.device) for p, y in zip(plans, ys)]
    hp = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    hy = (ctypes.c_void_p * n)(*[_dev(y, p.y_shape, "y") for p, y in zip(plans, ys)])
    hx = (ctypes.c_void_p * n)(*[_dev(x, p.x_shape, "x") for p, x in zip(plans, xs)])
    reps = (Report * n)() if report else None
    _check(lib().smsm_reconstruct_groups(n, hp, hy, hx, ctypes.byref(params), reps, _stream()))
    return xs, (list(reps) if report else None)


def default_params(**kw) -> Params:
    p = Params()
    lib().smsm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k in ("lam", "lambda") else k, v)
    return p


def smsm_hankel_gram_noalloc(x: torch.Tensor, filter: int, G: torch.Tensor | None = None) -> torch.Tensor:
    """Hankel Gram of x [mb][shots][n][n] without a plan and without any device
    allocation inside the library (G is allocated here by torch when not given)."""
    mb, shots, n, _ = x.shape
    C = shots * filter * filter
    if G is None:
        G = torch.empty((mb, C, C), dtype=torch.complex128, device=x.device)
    _check(lib().smsm_hankel_gram_noalloc(_dev(x, x.shape, "x"), _dev(G, (mb, C, C), "G", torch.complex128),
                                          mb, shots, n, filter, _stream()))
    return G


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, shape, name: str, dtype=torch.complex64) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


class Plan:
    """One slice-group geometry: smsm_plan(mb, shots, coils, N, N, filter).

    With batch > 1 every per-problem tensor has a leading batch dimension.
    """

    def __init__(self, mb: int, shots: int, coils: int, n: int, filter: int, caipi_div: int = 0,
                 batch: int = 1, flags: int = 0, precision: int = 0, boundary: int = 0):
        self.L, self.Ns, self.Nc, self.N, self.r = mb, shots, coils, n, filter
        self.D = batch
        self.C = shots * filter * filter
        self.M = n // shots if shots else 0
        h = ctypes.c_void_p()
        opts = Opts(caipi_div=caipi_div, batch=batch, flags=flags, precision=precision, boundary=boundary)
        _check(lib().smsm_plan(ctypes.byref(h), mb, shots, coils, n, n, filter, ctypes.byref(opts)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().smsm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self) -> int:
        """Synchronise and return the plan's device error flag (0 = fine)."""
        return lib().smsm_plan_device_status(self._h, _stream())

    @property
    def workspace_bytes(self) -> int:
        return lib().smsm_plan_workspace_bytes(self._h)

    # shapes
    def _b(self, shape):
        return (self.D,) + tuple(shape) if self.D > 1 else tuple(shape)

    @property
    def x_shape(self):
        return self._b((self.L, self.Ns, self.N, self.N))

    @property
    def y_shape(self):
        return self._b((self.Ns, self.Nc, self.M, self.N))

    @property
    def g_shape(self):
        return self._b((self.L, self.C, self.C))

    def smsm_plan_set_sens(self, sens: torch.Tensor) -> None:
        _check(lib().smsm_plan_set_sens(self._h, _dev(sens, (self.L, self.Nc, self.N, self.N), "sens"), _stream()))
        self._sens = sens  # keep alive until the transpose has run

    set_sens = smsm_plan_set_sens

    def smsm_forward(self, x: torch.Tensor, phase: torch.Tensor | None = None, y: torch.Tensor | None = None):
        xs = self._b((self.L, 1 if phase is not None else self.Ns, self.N, self.N))
        if y is None:
            y = torch.empty(self.y_shape, dtype=torch.complex64, device=x.device)
        pp = _dev(phase, self.x_shape, "phase") if phase is not None else None
        _check(lib().smsm_forward(self._h, _dev(x, xs, "x"), pp, _dev(y, self.y_shape, "y"), _stream()))
        return y

    forward = smsm_forward

    def smsm_adjoint(self, y: torch.Tensor, phase: torch.Tensor | None = None, x: torch.Tensor | None = None):
        xs = self._b((self.L, 1 if phase is not None else self.Ns, self.N, self.N))
        if x is None:
            x = torch.empty(xs, dtype=torch.complex64, device=y.device)
        pp = _dev(phase, self.x_shape, "phase") if phase is not None else None
        _check(lib().smsm_adjoint(self._h, _dev(y, self.y_shape, "y"), pp, _dev(x, xs, "x"), _stream()))
        return x

    adjoint = smsm_adjoint

    def smsm_hankel_gram(self, x: torch.Tensor, G: torch.Tensor | None = None):
        if G is None:
            G = torch.empty(self.g_shape, dtype=torch.complex128, device=x.device)
        _check(lib().smsm_hankel_gram(self._h, _dev(x, self.x_shape, "x"),
                                      _dev(G, self.g_shape, "G", torch.complex128), _stream()))
        return G

    hankel_gram = smsm_hankel_gram

    def smsm_apply_filters(self, W: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None):
        if out is None:
            out = torch.empty(self.x_shape, dtype=torch.complex64, device=x.device)
        _check(lib().smsm_apply_filters(self._h, _dev(W, self.g_shape, "W", torch.complex128),
                                        _dev(x, self.x_shape, "x"), _dev(out, self.x_shape, "out"), _stream()))
        return out

    apply_filters = smsm_apply_filters

    def smsm_reconstruct(self, y: torch.Tensor, x: torch.Tensor | None = None, params: Params | None = None,
                         report: bool = True):
        """Returns (x, Report or None).  x is the warm start when params.warm."""
        if params is None:
            params = default_params()
        if x is None:
            x = torch.empty(self.x_shape, dtype=torch.complex64, device=y.device)
        rep = Report() if report else None
        _check(lib().smsm_reconstruct(self._h, _dev(y, self.y_shape, "y"), _dev(x, self.x_shape, "x"),
                                      ctypes.byref(params), ctypes.byref(rep) if rep is not None else None,
                                      _stream()))
        return x, rep

    reconstruct = smsm_reconstruct

    def smsm_autotune(self, y: torch.Tensor, params: Params | None = None) -> TuneReport:
        """Time the Gram's split-K blocks and the lane count on y; keep (and cache per shape)
        the fastest.  Returns what was timed."""
        if params is None:
            params = default_params()
        rep = TuneReport()
        _check(lib().smsm_autotune(self._h, _dev(y, self.y_shape, "y"), ctypes.byref(params), ctypes.byref(rep),
                                   _stream()))
        return rep

    autotune = smsm_autotune

    def smsm_sense(self, y: torch.Tensor, phase: torch.Tensor | None = None, cg_iters: int = 30,
                   x: torch.Tensor | None = None, report: bool = True):
        """SMS-SENSE comparison reconstruction: returns (x [.., L, 1, N, N], Report or None)."""
        xs = self._b((self.L, 1, self.N, self.N))
        if x is None:
            x = torch.empty(xs, dtype=torch.complex64, device=y.device)
        pp = _dev(phase, self.x_shape, "phase") if phase is not None else None
        rep = Report() if report else None
        _check(lib().smsm_sense(self._h, _dev(y, self.y_shape, "y"), pp, _dev(x, xs, "x"), int(cg_iters),
                                ctypes.byref(rep) if rep is not None else None, _stream()))
        return x, rep

    sense = smsm_sense

    def smsm_fft2c(self, t: torch.Tensor, inverse: bool = False, out: torch.Tensor | None = None):
        if out is None:
            out = torch.empty_like(t)
        count = t.numel() // (self.N * self.N)
        _check(lib().smsm_fft2c(self._h, _dev(t, t.shape, "in"), _dev(out, t.shape, "out"), count,
                                1 if inverse else 0, _stream()))
        return out

    fft2c = smsm_fft2c


class CNN:
    """The warm-start network: smsm_cnn_create(channels, width, layers, H, W, max_batch)."""

    def __init__(self, channels: int, height: int, width_px: int, width: int = 64, layers: int = 6,
                 max_batch: int = 1):
        self.B, self.H, self.W, self.width, self.layers, self.maxn = channels, height, width_px, width, layers, max_batch
        h = ctypes.c_void_p()
        _check(lib().smsm_cnn_create(ctypes.byref(h), channels, width, layers, height, width_px, max_batch))
        self._h = h
        self.count = lib().smsm_cnn_param_count(h)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().smsm_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _io(self, t: torch.Tensor, n: int, name: str) -> int:
        return _dev(t, (n, self.B, self.H, self.W), name)

    def set_params(self, p: torch.Tensor) -> None:
        _check(lib().smsm_cnn_set_params(self._h, _dev(p, (self.count,), "params"), _stream()))

    def get_params(self) -> torch.Tensor:
        p = torch.empty(self.count, dtype=torch.complex64, device="cuda")
        _check(lib().smsm_cnn_get_params(self._h, _dev(p, (self.count,), "params"), _stream()))
        return p

    def forward(self, a: torch.Tensor) -> torch.Tensor:
        n = a.shape[0]
        out = torch.empty_like(a)
        _check(lib().smsm_cnn_forward(self._h, self._io(a, n, "a"), self._io(out, n, "x0"), n, _stream()))
        return out

    def gradients(self, a: torch.Tensor, t: torch.Tensor):
        """(mean loss, gradient [count]) of the batch."""
        n = a.shape[0]
        g = torch.empty(self.count, dtype=torch.complex64, device=a.device)
        loss = ctypes.c_double()
        _check(lib().smsm_cnn_gradients(self._h, self._io(a, n, "a"), self._io(t, n, "t"), n,
                                        _dev(g, (self.count,), "grad"), ctypes.byref(loss), _stream()))
        return loss.value, g

    def train_step(self, a: torch.Tensor, t: torch.Tensor, lr: float, want_loss: bool = True):
        n = a.shape[0]
        loss = ctypes.c_double()
        _check(lib().smsm_cnn_train_step(self._h, self._io(a, n, "a"), self._io(t, n, "t"), n, float(lr),
                                         ctypes.byref(loss) if want_loss else None, _stream()))
        return loss.value if want_loss else None


def learned_start(plan: "Plan", cnn: CNN, x_in: torch.Tensor, x_out: torch.Tensor | None = None) -> torch.Tensor:
    """x_out = F(cnn(F^-1(x_in))): the network applied to a k-space estimate of every problem."""
    if x_out is None:
        x_out = torch.empty(plan.x_shape, dtype=torch.complex64, device=x_in.device)
    _check(lib().smsm_learned_start(plan._h, cnn._h, _dev(x_in, plan.x_shape, "x_in"),
                                    _dev(x_out, plan.x_shape, "x_out"), _stream()))
    return x_out

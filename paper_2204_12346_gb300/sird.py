"""Python binding of the C ABI in ``include/sird_pso.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/libsird_pso.so``; this module only
builds the C structs, passes torch device pointers and the current CUDA stream, and turns
status codes into exceptions.  There is no CPU fallback: if the library cannot be loaded,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from collections.abc import Sequence

import numpy as np

from . import build as _build

MAX_PARAMS = 32
OK, ERR_ARG, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, ERR_STATE, ERR_NOMEM, ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_NUMERIC", "ERR_TIMEOUT", "ERR_STATE", "ERR_NOMEM", "ERR_UNSUPPORTED"]
COST_MSE, COST_MXSE, COST_MAE, COST_MAPE = 0, 1, 2, 3
COSTS = {"mse": COST_MSE, "mxse": COST_MXSE, "mae": COST_MAE, "mape": COST_MAPE}
BETA_PWC, BETA_RAMP = 0, 1
FIT_D, FIT_IRD = 0, 1
LAUNCH_AUTO, LAUNCH_PER_ITER, LAUNCH_PERSISTENT, LAUNCH_WINDOW_PER_BLOCK, LAUNCH_FLAT, LAUNCH_CLUSTER = 0, 1, 2, 3, 4, 5

# Symbols the header declares (checked by the ABI test).
EXPORTS = [
    "sird_pso_create", "sird_pso_destroy", "sird_last_error", "sird_pso_clear_error", "sird_pso_set_stream",
    "sird_pso_num_params", "sird_pso_eval", "sird_pso_init", "sird_pso_step", "sird_pso_calibrate",
    "sird_pso_result", "sird_pso_sync", "sird_pso_get_state", "sird_pso_set_state", "sird_loss_grad",
    "sird_forecast", "sird_pso_calibrate_batched", "sird_pso_set_observations", "sird_pso_set_timing", "sird_pso_launch_mode",
    "sird_pso_step_f32_noalloc", "sird_pso_topk", "sird_ensemble_bands", "sird_pso_polish", "sird_batch_create", "sird_batch_calibrate", "sird_batch_set_observations", "sird_batch_launch_mode",
    "sird_batch_block_size", "sird_batch_blocks_per_sm", "sird_batch_destroy", "sird_batch_set_timing",
    "sird_batch_polish", "sird_parameter_bands",
    "sird_pso_topk_indexed", "sird_pso_set_shard", "sird_pso_shard_best", "sird_pso_set_gbest",
]


class SirdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [
        ("n_obs", C.c_int), ("y_D", C.POINTER(C.c_double)), ("y_I", C.POINTER(C.c_double)),
        ("y_R", C.POINTER(C.c_double)), ("N", C.c_double), ("I0", C.c_double), ("R0", C.c_double),
        ("fit_I0", C.c_int), ("beta_form", C.c_int), ("K", C.c_int), ("steps_per_day", C.c_int),
        ("cost", C.c_int), ("objective", C.c_int),
    ]


class Config(C.Structure):
    _fields_ = [
        ("particles", C.c_int), ("iters", C.c_int), ("w", C.c_double), ("c1", C.c_double), ("c2", C.c_double),
        ("lb", C.POINTER(C.c_double)), ("ub", C.POINTER(C.c_double)), ("log_scale", C.POINTER(C.c_int)),
        ("precision", C.c_int), ("seed", C.c_uint64), ("stream_id", C.c_uint32), ("reeval_topk", C.c_int),
        ("block_size", C.c_int), ("launch_mode", C.c_int),
    ]


class Result(C.Structure):
    _fields_ = [
        ("n_params", C.c_int), ("theta", C.c_double * MAX_PARAMS), ("loss", C.c_double),
        ("loss_search", C.c_double), ("r2_D", C.c_double), ("index", C.c_int), ("iters_done", C.c_int),
    ]

    def as_dict(self) -> dict:
        return {"theta": np.array(self.theta[: self.n_params]), "loss": self.loss, "loss_search": self.loss_search,
                "r2_D": self.r2_D, "index": self.index, "iters_done": self.iters_done}


class BatchResults(Sequence):
    """Per-window results of a batched call, in window order: results[i] is window i's result dict
    (as Result.as_dict gives it, built on first access and kept), so a caller that reads a few
    windows of a large batch pays for those only."""

    def __init__(self, raw):
        self._raw = raw  # the ctypes Result array the library filled
        self._dicts = {}

    def __len__(self) -> int:
        return len(self._raw)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        n = len(self._raw)
        if i < 0:
            i += n
        if not 0 <= i < n:
            raise IndexError("window index out of range")
        d = self._dicts.get(i)
        if d is None:
            d = self._dicts[i] = self._raw[i].as_dict()
        return d


_lib = None


def lib():
    """Loads (building first if needed) the CUDA library.  Raises if it cannot."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not found at {path}")
        L = C.CDLL(path)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.sird_pso_create.argtypes = [C.POINTER(Problem), C.POINTER(Config), vp, C.POINTER(vp)]
        L.sird_pso_destroy.argtypes = [vp]
        L.sird_pso_destroy.restype = None
        L.sird_last_error.argtypes = [vp]
        L.sird_last_error.restype = C.c_char_p
        L.sird_pso_clear_error.argtypes = [vp]
        L.sird_pso_set_stream.argtypes = [vp, vp]
        L.sird_pso_num_params.argtypes = [vp]
        L.sird_pso_eval.argtypes = [vp, vp, ip, ip, vp, ip]
        L.sird_pso_init.argtypes = [vp]
        L.sird_pso_step.argtypes = [vp, ip]
        L.sird_pso_calibrate.argtypes = [vp, C.POINTER(Result)]
        L.sird_pso_result.argtypes = [vp, C.POINTER(Result)]
        L.sird_pso_sync.argtypes = [vp]
        L.sird_pso_get_state.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.sird_pso_set_state.argtypes = [vp, vp, C.c_size_t]
        L.sird_loss_grad.argtypes = [vp, vp, ip, ip, vp, vp, ip, vp, ip, ip]
        L.sird_forecast.argtypes = [C.POINTER(Problem), dp, ip, ip, dp, ip, vp]
        L.sird_ensemble_bands.argtypes = [C.POINTER(Problem), dp, ip, ip, dp, ip, dp, vp]
        L.sird_parameter_bands.argtypes = [C.POINTER(Problem), dp, ip, dp, ip, dp, vp]
        L.sird_pso_calibrate_batched.argtypes = [ip, C.POINTER(Problem), C.POINTER(Config), vp, C.POINTER(Result)]
        L.sird_pso_set_observations.argtypes = [vp, dp, ip]
        L.sird_pso_set_timing.argtypes = [vp, vp, vp]
        L.sird_pso_launch_mode.argtypes = [vp]
        L.sird_pso_topk.argtypes = [vp, ip, dp, dp]
        L.sird_pso_topk_indexed.argtypes = [vp, ip, dp, dp, C.POINTER(C.c_int)]
        L.sird_pso_set_shard.argtypes = [vp, ip, ip]
        L.sird_pso_shard_best.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_float)]
        L.sird_pso_set_gbest.argtypes = [vp, C.POINTER(C.c_float), C.c_float, ip]
        L.sird_batch_create.argtypes = [ip, C.POINTER(Problem), C.POINTER(Config), vp, C.POINTER(vp)]
        L.sird_batch_calibrate.argtypes = [vp, C.POINTER(Result)]
        L.sird_batch_polish.argtypes = [vp, ip, ip, C.c_double, C.POINTER(Result)]
        L.sird_batch_block_size.argtypes = [vp]
        L.sird_batch_blocks_per_sm.argtypes = [vp]
        L.sird_batch_launch_mode.argtypes = [vp]
        L.sird_batch_set_timing.argtypes = [vp, vp, vp]
        L.sird_batch_set_observations.argtypes = [vp, C.POINTER(C.c_double), C.c_longlong, C.POINTER(C.c_size_t)]
        L.sird_batch_destroy.argtypes = [vp]
        L.sird_batch_destroy.restype = None
        L.sird_pso_polish.argtypes = [vp, ip, ip, C.c_double, ip, ip, C.POINTER(Result)]
        L.sird_pso_step_f32_noalloc.argtypes = [C.POINTER(Problem), C.POINTER(Config)] + [vp] * 6 + [ip, ip, vp, vp]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def current_stream_handle(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def n_params(K=1, beta_form=BETA_PWC, fit_I0=True) -> int:
    """Entries of theta: beta_1..beta_K (or beta1, beta2, t1, t2 of the ramp), gamma, mu[, I0]."""
    return (6 if int(beta_form) == BETA_RAMP else int(K) + 2) + (1 if fit_I0 else 0)


def _check_box(P, lb, ub, log_scale):
    """The library reads P entries of lb, ub and log_scale: shorter arrays are refused here."""
    for name, a in (("lb", lb), ("ub", ub), ("log_scale", log_scale)):
        if a is not None and np.asarray(a).size < P:
            raise ValueError(f"{name} has {np.asarray(a).size} entries; the model has {P} parameters")
    if lb is None or ub is None:
        raise ValueError("lb and ub are required")


def make_problem(yD, N, K=1, spd=10, R0=0.0, I0=0.0, fit_I0=True, beta_form=BETA_PWC, cost=COST_MSE,
                 objective=FIT_D, yI=None, yR=None):
    """Builds a Problem struct; the returned keep-alive list must outlive the call that uses it."""
    yD = _f64(yD)
    for name, a in (("yI", yI), ("yR", yR)):  # the library reads len(yD) values of each
        if a is not None and np.asarray(a).size < yD.size:
            raise ValueError(f"{name} has {np.asarray(a).size} values; yD has {yD.size}")
    keep = [yD]
    null = C.POINTER(C.c_double)()
    pI = pR = null
    if yI is not None:
        yI = _f64(yI)
        keep.append(yI)
        pI = _dptr(yI)
    if yR is not None:
        yR = _f64(yR)
        keep.append(yR)
        pR = _dptr(yR)
    pb = Problem(len(yD), _dptr(yD), pI, pR, float(N), float(I0), float(R0), int(fit_I0), int(beta_form), int(K),
                 int(spd), int(cost), int(objective))
    return pb, keep


def make_config(particles, iters, lb, ub, log_scale=None, w=0.5, c1=0.5, c2=0.5, precision=32, seed=0,
                stream_id=0, reeval_topk=0, block_size=0, launch_mode=0):
    lb, ub = _f64(lb), _f64(ub)
    keep = [lb, ub]
    lsp = C.POINTER(C.c_int)()
    if log_scale is not None:
        ls = np.ascontiguousarray(np.asarray(log_scale, dtype=np.int32))
        keep.append(ls)
        lsp = ls.ctypes.data_as(C.POINTER(C.c_int))
    cfg = Config(int(particles), int(iters), float(w), float(c1), float(c2), _dptr(lb), _dptr(ub), lsp,
                 int(precision), int(seed) & (2**64 - 1), int(stream_id) & 0xFFFFFFFF, int(reeval_topk),
                 int(block_size), int(launch_mode))
    return cfg, keep


class Calibrator:
    """One calibration window and its swarm on the GPU (wraps a sird_pso_t handle)."""

    def __init__(self, yD, N, *, K=1, spd=10, R0=0.0, I0=0.0, fit_I0=True, beta_form=BETA_PWC, cost=COST_MSE,
                 particles=64, iters=100, lb=None, ub=None, log_scale=None, w=0.5, c1=0.5, c2=0.5, precision=32,
                 seed=0, stream_id=0, reeval_topk=0, block_size=0, launch_mode=0, stream=None, objective=FIT_D,
                 yI=None, yR=None):
        self._lib = lib()
        self.problem, k1 = make_problem(yD, N, K, spd, R0, I0, fit_I0, beta_form, cost, objective, yI, yR)
        _check_box(n_params(K, beta_form, fit_I0), lb, ub, log_scale)
        self.config, k2 = make_config(particles, iters, lb, ub, log_scale, w, c1, c2, precision, seed, stream_id,
                                      reeval_topk, block_size, launch_mode)
        self._keep = k1 + k2
        self.precision = int(precision)
        self.M = int(particles)
        h = C.c_void_p()
        st = self._lib.sird_pso_create(C.byref(self.problem), C.byref(self.config),
                                       C.c_void_p(current_stream_handle(stream)), C.byref(h))
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(None).decode())
        self.h = h
        self.P = self._lib.sird_pso_num_params(h)
        self.launch_mode = self._lib.sird_pso_launch_mode(h)

    def _check(self, st):
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.sird_pso_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream=None):
        self._check(self._lib.sird_pso_set_stream(self.h, C.c_void_p(current_stream_handle(stream))))

    def eval(self, theta, out=None, precision=None):
        """Loss of each column of theta ([P, M] or [P, ld] torch CUDA tensor, float32/float64)."""
        import torch

        precision = precision or (32 if theta.dtype == torch.float32 else 64)
        dt = torch.float32 if precision == 32 else torch.float64
        if theta.dtype != dt or not theta.is_cuda or theta.dim() != 2 or theta.shape[0] != self.P:
            raise ValueError("theta must be a CUDA tensor [P, M] of the requested precision")
        if theta.stride(1) != 1:
            raise ValueError("theta rows must be contiguous")
        M = theta.shape[1]
        if out is None:
            out = torch.empty(M, dtype=dt, device=theta.device)
        self._check(self._lib.sird_pso_eval(self.h, C.c_void_p(theta.data_ptr()), M, theta.stride(0),
                                            C.c_void_p(out.data_ptr()), precision))
        return out

    def eval64(self, thetas) -> np.ndarray:
        """FP64 losses (the paper's arithmetic) of the rows of thetas ([k, P], host)."""
        import torch

        th = torch.from_numpy(np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).T)).cuda()
        torch.cuda.current_stream().synchronize()  # th is on the device before the handle's stream reads it
        out = self.eval(th, precision=64)
        self.sync()
        return out.cpu().numpy()

    def set_observations(self, yD):
        """Uploads new observations (same length, same first value) for the next calibration."""
        y = _f64(yD)
        self._keep_obs = y
        self._check(self._lib.sird_pso_set_observations(self.h, _dptr(y), len(y)))

    def set_timing(self, ev_begin=None, ev_end=None):
        """torch.cuda.Event pair recorded around the iteration launches of every calibrate."""
        b = C.c_void_p(ev_begin.cuda_event) if ev_begin is not None else None
        e = C.c_void_p(ev_end.cuda_event) if ev_end is not None else None
        self._check(self._lib.sird_pso_set_timing(self.h, b, e))

    def loss_grad(self, theta, ckpt_every=16, grad_u0=False):
        """Loss and exact gradient (discrete adjoint) of each column of theta ([P, M] CUDA
        tensor; float64: the paper's FP64 arithmetic, float32: the compensated FP32 path).
        Returns (loss [M], grad [P, M]) or (loss, grad, grad_u0 [4, M]) in theta's dtype."""
        import torch

        if theta.dtype not in (torch.float32, torch.float64) or not theta.is_cuda or theta.dim() != 2 \
                or theta.shape[0] != self.P:
            raise ValueError("theta must be a CUDA float32/float64 tensor [P, M]")
        if theta.stride(1) != 1:
            raise ValueError("theta rows must be contiguous")
        prec = 64 if theta.dtype == torch.float64 else 32
        M = theta.shape[1]
        loss = torch.empty(M, dtype=theta.dtype, device=theta.device)
        grad = torch.empty(self.P, M, dtype=theta.dtype, device=theta.device)
        gu = torch.empty(4, M, dtype=theta.dtype, device=theta.device) if grad_u0 else None
        self._check(self._lib.sird_loss_grad(self.h, C.c_void_p(theta.data_ptr()), M, theta.stride(0),
                                             C.c_void_p(loss.data_ptr()), C.c_void_p(grad.data_ptr()), M,
                                             C.c_void_p(gu.data_ptr()) if gu is not None else None, prec,
                                             int(ckpt_every)))
        return (loss, grad, gu) if grad_u0 else (loss, grad)

    def init(self):
        self._check(self._lib.sird_pso_init(self.h))
        return self

    def step(self, n=1):
        self._check(self._lib.sird_pso_step(self.h, int(n)))
        return self

    def sync(self):
        self._check(self._lib.sird_pso_sync(self.h))

    def calibrate(self) -> dict:
        r = Result()
        self._check(self._lib.sird_pso_calibrate(self.h, C.byref(r)))
        return r.as_dict()

    def result(self) -> dict:
        r = Result()
        self._check(self._lib.sird_pso_result(self.h, C.byref(r)))
        return r.as_dict()

    def polish(self, k=32, iters=50, first_step=1e-2, ckpt_every=16, precision=64) -> dict:
        """L-BFGS polish of the k best personal bests (discrete-adjoint gradient); trials and
        gradients in FP64 (precision=64) or FP32 (32); the reported loss is FP64."""
        r = Result()
        self._check(self._lib.sird_pso_polish(self.h, int(k), int(iters), float(first_step), int(ckpt_every),
                                              int(precision), C.byref(r)))
        return r.as_dict()

    def topk(self, k: int, with_index: bool = False):
        """(theta [k, P], loss [k]) of the k best personal bests, best first; with_index adds
        their particle indices (global for a shard)."""
        th = np.zeros((k, self.P))
        lo = np.zeros(k)
        if not with_index:
            self._check(self._lib.sird_pso_topk(self.h, int(k), _dptr(th), _dptr(lo)))
            return th, lo
        idx = np.zeros(k, dtype=np.int32)
        self._check(self._lib.sird_pso_topk_indexed(self.h, int(k), _dptr(th), _dptr(lo),
                                                    idx.ctypes.data_as(C.POINTER(C.c_int))))
        return th, lo, idx

    def set_shard(self, offset: int, total: int):
        """Declares this handle's particles offset .. offset + M - 1 of a swarm of `total`."""
        self._check(self._lib.sird_pso_set_shard(self.h, int(offset), int(total)))
        return self

    def shard_best(self):
        """(FP32 loss, global index, z [P] float32) of the best personal best among this
        handle's particles."""
        f = C.c_float()
        i = C.c_int()
        z = np.zeros(self.P, dtype=np.float32)
        self._check(self._lib.sird_pso_shard_best(self.h, C.byref(f), C.byref(i),
                                                  z.ctypes.data_as(C.POINTER(C.c_float))))
        return float(f.value), int(i.value), z

    def set_gbest(self, z, loss: float, index: int):
        """The swarm's global best (position z in the search coordinates) for the next step."""
        z = np.ascontiguousarray(np.asarray(z, dtype=np.float32))
        if z.size != self.P:
            raise ValueError(f"z has {z.size} entries; the model has {self.P} parameters")
        self._check(self._lib.sird_pso_set_gbest(self.h, z.ctypes.data_as(C.POINTER(C.c_float)), float(loss),
                                                 int(index)))

    def get_state(self) -> dict:
        n = C.c_size_t(0)
        self._check(self._lib.sird_pso_get_state(self.h, None, C.byref(n)))
        buf = (C.c_ubyte * n.value)()
        self._check(self._lib.sird_pso_get_state(self.h, buf, C.byref(n)))
        raw = bytes(buf)
        hdr = np.frombuffer(raw[:48], dtype=np.uint32)  # 48-byte header, see include/sird_pso.h
        M, P, prec, it, gidx = [int(np.int32(v)) for v in hdr[2:7]]
        dt = np.float32 if prec == 32 else np.float64
        body = np.frombuffer(raw[48:], dtype=dt)
        plane = M * P
        return {"raw": raw, "M": M, "P": P, "precision": prec, "iter": it, "gbest_idx": gidx,
                "x": body[:plane].reshape(P, M).copy(), "v": body[plane:2 * plane].reshape(P, M).copy(),
                "pbest": body[2 * plane:3 * plane].reshape(P, M).copy(),
                "pbest_f": body[3 * plane:3 * plane + M].copy()}

    def set_state(self, x, v, pbest, pbest_f, gbest_idx, iteration, seed=None, stream_id=None):
        """Loads a swarm state (arrays [P, M] and [M] in the swarm precision)."""
        dt = np.float32 if self.precision == 32 else np.float64
        hdr = np.zeros(10, dtype=np.uint32)
        hdr[0], hdr[1] = 0x44524953, 1
        hdr[2:8] = [self.M, self.P, self.precision, int(iteration), int(gbest_idx), 0]
        seed = int(self.config.seed if seed is None else seed)
        hdr[8] = seed & 0xFFFFFFFF
        hdr[9] = (seed >> 32) & 0xFFFFFFFF
        tail = np.array([int(self.config.stream_id if stream_id is None else stream_id), 0], dtype=np.uint32)
        body = np.concatenate([np.asarray(a, dtype=dt).ravel() for a in (x, v, pbest, pbest_f)])
        raw = hdr.tobytes() + tail.tobytes() + body.tobytes()
        buf = (C.c_ubyte * len(raw)).from_buffer_copy(raw)
        self._check(self._lib.sird_pso_set_state(self.h, buf, len(raw)))


try:
    import torch as _torch

    class SirdLoss(_torch.autograd.Function):
        """FP64 loss of each column of theta ([P, M] CUDA float64) with its exact gradient from
        the discrete-adjoint kernel: SirdLoss.apply(calibrator, theta[, ckpt_every])."""

        @staticmethod
        def forward(ctx, cal, theta, ckpt_every=16):
            loss, grad = cal.loss_grad(theta.detach().contiguous(), ckpt_every=ckpt_every)
            ctx.save_for_backward(grad)
            return loss

        @staticmethod
        def backward(ctx, grad_out):
            (grad,) = ctx.saved_tensors
            return None, grad * grad_out.unsqueeze(0), None
except ImportError:  # the binding still loads for CPU-only tooling
    SirdLoss = None


def _batch_structs(windows, K, spd, cost, beta_form, fit_I0, iters, lb, ub, log_scale, w, c1, c2, particles, seed,
                   block_size, objective=FIT_D, launch_mode=0):
    W = len(windows)
    _check_box(n_params(K, beta_form, fit_I0), lb, ub, log_scale)
    keep = []
    pbs = (Problem * W)()
    cfgs = (Config * W)()
    for i, win in enumerate(windows):
        pb, k1 = make_problem(win["yD"], win["N"], K, spd, win.get("R0", 0.0), win.get("I0", 0.0), fit_I0,
                              beta_form, cost, objective, win.get("yI"), win.get("yR"))
        cfg, k2 = make_config(int(win.get("particles", particles)), iters, lb, ub, log_scale, w, c1, c2, 32,
                              int(win.get("seed", seed)), int(win.get("stream_id", i)), 0,
                              block_size if i == 0 else 0, launch_mode if i == 0 else 0)
        keep += k1 + k2
        pbs[i] = pb
        cfgs[i] = cfg
    keep += [pbs, cfgs]
    return pbs, cfgs, keep


class Batch:
    """Many calibration windows in one persistent launch (wraps a sird_batch_t).

    windows: list of dicts with keys yD, N and optionally R0, I0, particles, seed, stream_id;
    the model and PSO settings (K, spd, cost, beta_form, fit_I0, iters, lb, ub, log_scale, w,
    c1, c2, block_size) are shared."""

    def __init__(self, windows, *, K=1, spd=10, cost=COST_MSE, beta_form=BETA_PWC, fit_I0=True, iters=100,
                 lb=None, ub=None, log_scale=None, w=0.5, c1=0.5, c2=0.5, particles=256, seed=0, block_size=0,
                 stream=None, objective=FIT_D, launch_mode=0):
        self._lib = lib()
        W = len(windows)
        pbs, cfgs, self._keep = _batch_structs(windows, K, spd, cost, beta_form, fit_I0, iters, lb, ub, log_scale,
                                               w, c1, c2, particles, seed, block_size, objective, launch_mode)
        h = C.c_void_p()
        st = self._lib.sird_batch_create(W, pbs, cfgs, C.c_void_p(current_stream_handle(stream)), C.byref(h))
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(None).decode())
        self.h = h
        self.W = W
        self.block_size = self._lib.sird_batch_block_size(h)
        self.blocks_per_sm = self._lib.sird_batch_blocks_per_sm(h)
        self.launch_mode = self._lib.sird_batch_launch_mode(h)

    def set_timing(self, ev_begin=None, ev_end=None):
        """torch.cuda.Event pair recorded around the batch kernel of every calibrate."""
        b = C.c_void_p(ev_begin.cuda_event) if ev_begin is not None else None
        e = C.c_void_p(ev_end.cuda_event) if ev_end is not None else None
        st = self._lib.sird_batch_set_timing(self.h, b, e)
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(None).decode())

    def set_observations(self, y_all) -> int:
        """New observations for every window (concatenated, each window's original length; for an
        F_IRD batch each window's yD, yI, yR in turn); the copy is ordered before the next
        calibrate.  Returns the bytes copied to the device."""
        y = _f64(y_all)
        nb = C.c_size_t(0)
        st = self._lib.sird_batch_set_observations(self.h, _dptr(y), len(y), C.byref(nb))
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(None).decode())
        return int(nb.value)

    def calibrate(self):
        """Calibrates every window (one graph launch); a BatchResults sequence of result dicts."""
        res = (Result * self.W)()
        st = self._lib.sird_batch_calibrate(self.h, res)
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(None).decode())
        return BatchResults(res)

    def polish(self, k=32, iters=40, first_step=1e-2):
        """L-BFGS polish of every window's k best personal bests (FP32 trials and adjoint, FP64
        algebra and re-scoring), all windows together; a BatchResults sequence, one result dict
        per window."""
        res = (Result * self.W)()
        st = self._lib.sird_batch_polish(self.h, int(k), int(iters), float(first_step), res)
        if st != OK:
            raise SirdError(st, self._lib.sird_last_error(None).decode())
        return BatchResults(res)

    def close(self):
        if getattr(self, "h", None):
            self._lib.sird_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def calibrate_batched(windows, *, K=1, spd=10, cost=COST_MSE, beta_form=BETA_PWC, fit_I0=True, iters=100, lb=None,
                      ub=None, log_scale=None, w=0.5, c1=0.5, c2=0.5, particles=256, seed=0, block_size=0,
                      stream=None, objective=FIT_D):
    """One-shot batched calibration (sird_pso_calibrate_batched): host inputs in, results out."""
    L = lib()
    W = len(windows)
    pbs, cfgs, keep = _batch_structs(windows, K, spd, cost, beta_form, fit_I0, iters, lb, ub, log_scale, w, c1, c2,
                                     particles, seed, block_size, objective)
    res = (Result * W)()
    st = L.sird_pso_calibrate_batched(W, pbs, cfgs, C.c_void_p(current_stream_handle(stream)), res)
    if st != OK:
        raise SirdError(st, L.sird_last_error(None).decode())
    return [r.as_dict() for r in res]


def forecast(yD, N, theta, horizon, *, K=1, spd=10, R0=0.0, I0=0.0, fit_I0=True, beta_form=BETA_PWC,
             precision=64, stream=None) -> np.ndarray:
    """D on the `horizon` days after the window for each row of theta ([k, P]); returns [k, horizon]."""
    L = lib()
    pb, keep = make_problem(yD, N, K, spd, R0, I0, fit_I0, beta_form)
    th = _f64(np.atleast_2d(theta))
    if th.ndim != 2 or th.shape[1] != n_params(K, beta_form, fit_I0):
        raise ValueError(f"theta must be [k, {n_params(K, beta_form, fit_I0)}]")
    out = np.zeros((th.shape[0], int(horizon)))
    st = L.sird_forecast(C.byref(pb), _dptr(th), th.shape[0], int(horizon), _dptr(out), int(precision),
                         C.c_void_p(current_stream_handle(stream)))
    if st != OK:
        raise SirdError(st, L.sird_last_error(None).decode())
    return out


BAND_QUANTITIES = ("beta", "R0", "S", "I", "R", "D")


def ensemble_bands(yD, N, theta, horizon, fractions=(0.95, 0.9, 0.5), *, K=1, spd=10, R0=0.0, I0=0.0, fit_I0=True,
                   beta_form=BETA_PWC, stream=None) -> dict:
    """Median and central bands over an ensemble of parameter vectors ([k, P]) per day of the
    window and `horizon` more days: {quantity: [n_days, 1 + 2 len(fractions)]} with columns
    median, low_0, high_0, low_1, high_1, ..."""
    L = lib()
    pb, keep = make_problem(yD, N, K, spd, R0, I0, fit_I0, beta_form)
    th = _f64(np.atleast_2d(theta))
    if th.ndim != 2 or th.shape[1] != n_params(K, beta_form, fit_I0):
        raise ValueError(f"theta must be [k, {n_params(K, beta_form, fit_I0)}]")
    fr = _f64(fractions)
    n_days = len(_f64(yD)) + int(horizon)
    nq = 1 + 2 * len(fr)
    out = np.zeros((len(BAND_QUANTITIES), n_days, nq))
    st = L.sird_ensemble_bands(C.byref(pb), _dptr(th), th.shape[0], int(horizon), _dptr(fr), len(fr), _dptr(out),
                               C.c_void_p(current_stream_handle(stream)))
    if st != OK:
        raise SirdError(st, L.sird_last_error(None).decode())
    return {q: out[i] for i, q in enumerate(BAND_QUANTITIES)}


def parameter_bands(yD, N, theta, fractions=(0.95, 0.9, 0.5), *, K=1, spd=10, R0=0.0, I0=0.0, fit_I0=True,
                    beta_form=BETA_PWC, stream=None) -> np.ndarray:
    """Median and central bands of each parameter over an ensemble of parameter vectors ([k, P];
    the ramp's change times as t1 <= t2): [P, 1 + 2 len(fractions)] with columns median, low_0,
    high_0, low_1, high_1, ..."""
    L = lib()
    pb, keep = make_problem(yD, N, K, spd, R0, I0, fit_I0, beta_form)
    P = n_params(K, beta_form, fit_I0)
    th = _f64(np.atleast_2d(theta))
    if th.ndim != 2 or th.shape[1] != P:
        raise ValueError(f"theta must be [k, {P}]")
    fr = _f64(fractions)
    out = np.zeros((P, 1 + 2 * len(fr)))
    st = L.sird_parameter_bands(C.byref(pb), _dptr(th), th.shape[0], _dptr(fr), len(fr), _dptr(out),
                                C.c_void_p(current_stream_handle(stream)))
    if st != OK:
        raise SirdError(st, L.sird_last_error(None).decode())
    return out


def check_noalloc_buffers(P, M, n_obs, obs, x, v, pbest, pbest_f, gbest, gbest_index=None, require_cuda=True):
    """Refuses, before any library call, buffers that the no-allocation step would read or write
    past their ends: x, v and pbest float32 [P, ld] with one leading dimension ld >= M and unit
    stride along particles; pbest_f float32 with at least ld entries; gbest float32 with at
    least P; obs float32 with at least n_obs; gbest_index int32 with at least one; every tensor
    contiguous where it is read as a flat array and on the current CUDA device."""
    import torch

    def flat(t, name, dtype, n):
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} entries, needs at least {n}")

    tensors = {"obs": obs, "x": x, "v": v, "pbest": pbest, "pbest_f": pbest_f, "gbest": gbest}
    if gbest_index is not None:
        tensors["gbest_index"] = gbest_index
    if require_cuda:
        if not torch.cuda.is_available():
            raise ValueError("the buffers must be tensors on the current CUDA device (no CUDA device is available)")
        dev = torch.cuda.current_device()
        for name, t in tensors.items():
            if not t.is_cuda or t.device.index != dev:
                raise ValueError(f"{name} must be a tensor on the current CUDA device (cuda:{dev})")
    ld = None
    for name, t in (("x", x), ("v", v), ("pbest", pbest)):
        if t.dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
        if t.dim() != 2 or t.shape[0] < P:
            raise ValueError(f"{name} must be [P={P}, ld]")
        if t.stride(1) != 1:
            raise ValueError(f"{name} must have unit stride along particles")
        if ld is None:
            ld = t.stride(0)
        elif t.stride(0) != ld:
            raise ValueError("x, v and pbest must share one leading dimension")
        if t.shape[1] < M or ld < M:
            raise ValueError(f"{name} holds fewer than {M} particles per row")
        if t.storage_offset() + (P - 1) * ld + M > t.untyped_storage().nbytes() // 4:
            raise ValueError(f"{name} is too short for [P={P}, ld={ld}]")
    flat(pbest_f, "pbest_f", torch.float32, ld)
    flat(gbest, "gbest", torch.float32, P)
    flat(obs, "obs", torch.float32, n_obs)
    if gbest_index is not None:
        flat(gbest_index, "gbest_index", torch.int32, 1)
    return ld


def step_f32_noalloc(yD, N, obs, x, v, pbest, pbest_f, gbest, iteration, *, gbest_index=None, stream=None,
                     K=1, spd=10, R0=0.0, I0=0.0, fit_I0=True, beta_form=BETA_PWC, cost=COST_MSE, particles=None,
                     lb=None, ub=None, log_scale=None, w=0.5, c1=0.5, c2=0.5, seed=0, stream_id=0, block_size=0):
    """One FP32 PSO iteration on caller-owned torch CUDA buffers, through the entry point that
    allocates nothing (sird_pso_step_f32_noalloc).  x, v, pbest: [P, ld] float32; pbest_f: [ld];
    gbest: [P]; obs: [n_obs] float32 observations of D as yD - yD[0], the handle's own copy (the
    float values of yD give the same results when yD[0] = 0 or yD holds integers below 2^24);
    gbest_index: optional int32 CUDA tensor [1]."""
    L = lib()
    pb, k1 = make_problem(yD, N, K, spd, R0, I0, fit_I0, beta_form, cost)
    P = n_params(K, beta_form, fit_I0)
    _check_box(P, lb, ub, log_scale)
    M = int(particles if particles is not None else x.shape[1])
    check_noalloc_buffers(P, M, len(_f64(yD)), obs, x, v, pbest, pbest_f, gbest, gbest_index)
    cfg, k2 = make_config(M, 1, lb, ub, log_scale, w, c1, c2, 32, seed, stream_id, 0, block_size, 0)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    st = L.sird_pso_step_f32_noalloc(C.byref(pb), C.byref(cfg), ptr(obs), ptr(x), ptr(v), ptr(pbest), ptr(pbest_f),
                                     ptr(gbest), int(x.stride(0)), int(iteration), ptr(gbest_index),
                                     C.c_void_p(current_stream_handle(stream)))
    if st != OK:
        raise SirdError(st, L.sird_last_error(None).decode())


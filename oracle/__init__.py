"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does, and
nothing here is shared with it.

Every function follows the paper (arXiv 2204.12346) as cited in
``sird_oracle.c``: eq. (SIRD) and eq. (beta) of Sec. 2.2, the Euler scheme and
costs of Sec. 3.1, the PSO of Sec. 3.3 and the extension of Sec. 4.2.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sird_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsird_oracle.so")

BETA_PWC, BETA_RAMP = 0, 1
MSE, MXSE, MAE, MAPE = 0, 1, 2, 3
FIT_D, FIT_IRD = 0, 1
OBJ_SIRD, OBJ_SPHERE, OBJ_ROSENBROCK = 0, 1, 2
COSTS = {"mse": MSE, "mxse": MXSE, "mae": MAE, "mape": MAPE}


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (ISO C11, FMA contraction off, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sird_oracle.h"))
    ):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
             "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("n_obs", C.c_int),
        ("yD", C.POINTER(C.c_double)),
        ("yI", C.POINTER(C.c_double)),
        ("yR", C.POINTER(C.c_double)),
        ("N", C.c_double),
        ("I0", C.c_double),
        ("R0", C.c_double),
        ("fit_I0", C.c_int),
        ("beta_form", C.c_int),
        ("K", C.c_int),
        ("spd", C.c_int),
        ("cost", C.c_int),
        ("objective", C.c_int),
    ]


class _PsoCfg(C.Structure):
    _fields_ = [
        ("M", C.c_int),
        ("P", C.c_int),
        ("w", C.c_double),
        ("c1", C.c_double),
        ("c2", C.c_double),
        ("zlb", C.POINTER(C.c_double)),
        ("zub", C.POINTER(C.c_double)),
        ("logdim", C.POINTER(C.c_int)),
        ("seed", C.c_uint64),
        ("stream", C.c_uint32),
        ("store_f32", C.c_int),
        ("objective_kind", C.c_int),
        ("p_offset", C.c_uint32),
    ]


class _PsoState(C.Structure):
    _fields_ = [
        ("x", C.POINTER(C.c_double)),
        ("v", C.POINTER(C.c_double)),
        ("pbest", C.POINTER(C.c_double)),
        ("pbest_f", C.POINTER(C.c_double)),
        ("gbest", C.POINTER(C.c_double)),
        ("gbest_idx", C.c_int),
        ("gbest_f", C.c_double),
        ("iter", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        P = C.POINTER(_Problem)
        _lib.orc_nparams.argtypes = [P]
        _lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        _lib.orc_u01.argtypes = [C.c_uint32]
        _lib.orc_u01.restype = C.c_double
        _lib.orc_beta.argtypes = [P, dp, C.c_long, C.c_long]
        _lib.orc_beta.restype = C.c_double
        _lib.orc_simulate.argtypes = [P, dp, C.c_int, dp, dp, dp, dp]
        _lib.orc_simulate_schedule.argtypes = [C.c_double] * 5 + [dp, C.c_double, C.c_double, C.c_int, C.c_int,
                                                                   dp, dp, dp, dp]
        _lib.orc_loss.argtypes = [P, dp]
        _lib.orc_loss.restype = C.c_double
        _lib.orc_r2_D.argtypes = [P, dp]
        _lib.orc_r2_D.restype = C.c_double
        _lib.orc_loss_grad.argtypes = [P, dp, dp, dp]
        _lib.orc_loss_grad.restype = C.c_double
        _lib.orc_forecast.argtypes = [P, dp, C.c_int, dp]
        Cfg, St = C.POINTER(_PsoCfg), C.POINTER(_PsoState)
        _lib.orc_objective.argtypes = [Cfg, P, dp]
        _lib.orc_objective.restype = C.c_double
        _lib.orc_pso_init.argtypes = [Cfg, P, St]
        _lib.orc_pso_step.argtypes = [Cfg, P, St]
        _lib.orc_argmin.argtypes = [dp, C.c_int]
        _lib.orc_reeval_topk.argtypes = [Cfg, P, St, C.c_int, dp]
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Problem:
    """One calibration window (Sec. 3.1): n_obs daily observations of D on days 0..n_obs-1."""
    yD: np.ndarray
    N: float
    R0: float = 0.0
    I0: float = 0.0
    fit_I0: bool = True
    beta_form: int = BETA_PWC
    K: int = 1
    spd: int = 10
    cost: int = MSE
    objective: int = FIT_D
    yI: np.ndarray | None = None
    yR: np.ndarray | None = None
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Problem:
        yD = _f64(self.yD)
        yI = _f64(self.yI) if self.yI is not None else None
        yR = _f64(self.yR) if self.yR is not None else None
        self._keep = [yD, yI, yR]
        null = C.POINTER(C.c_double)()
        return _Problem(len(yD), _dptr(yD), _dptr(yI) if yI is not None else null,
                        _dptr(yR) if yR is not None else null, float(self.N), float(self.I0),
                        float(self.R0), int(self.fit_I0), int(self.beta_form), int(self.K),
                        int(self.spd), int(self.cost), int(self.objective))

    @property
    def n_params(self) -> int:
        base = 6 if self.beta_form == BETA_RAMP else self.K + 2
        return base + (1 if self.fit_I0 else 0)

    @property
    def days(self) -> int:
        return len(self.yD) - 1


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return np.array(list(out), dtype=np.uint32)


def u01(r: int) -> float:
    return lib().orc_u01(int(r) & 0xFFFFFFFF)


def beta_at(pb: Problem, theta, k: int) -> float:
    th = _f64(theta)
    return lib().orc_beta(C.byref(pb.c()), _dptr(th), int(k), int(pb.days * pb.spd))


def simulate(pb: Problem, theta, n_days: int | None = None) -> dict:
    """Daily S, I, R, D on days 0..n_days (explicit Euler on eq. (SIRD))."""
    n_days = pb.days if n_days is None else int(n_days)
    th = _f64(theta)
    out = {k: np.zeros(n_days + 1) for k in "SIRD"}
    rc = lib().orc_simulate(C.byref(pb.c()), _dptr(th), n_days, *[_dptr(out[k]) for k in "SIRD"])
    if rc != 0:
        raise ValueError("orc_simulate: bad arguments")
    return out


def simulate_schedule(N, u0, beta_steps, gamma, mu, spd, n_days) -> dict:
    """Euler with a per-step transmission rate; used to build synthetic series."""
    b = _f64(beta_steps)
    if b.size < n_days * spd:
        raise ValueError("beta_steps too short")
    out = {k: np.zeros(n_days + 1) for k in "SIRD"}
    rc = lib().orc_simulate_schedule(float(N), *[float(v) for v in u0], _dptr(b), float(gamma), float(mu),
                                     int(spd), int(n_days), *[_dptr(out[k]) for k in "SIRD"])
    if rc != 0:
        raise ValueError("orc_simulate_schedule: bad arguments")
    return out


def loss(pb: Problem, theta) -> float:
    th = _f64(theta)
    return lib().orc_loss(C.byref(pb.c()), _dptr(th))


def losses(pb: Problem, thetas) -> np.ndarray:
    """Loss of every row of thetas [M, P]."""
    thetas = _f64(thetas)
    cp = pb.c()
    return np.array([lib().orc_loss(C.byref(cp), _dptr(np.ascontiguousarray(t))) for t in thetas])


def r2_D(pb: Problem, theta) -> float:
    th = _f64(theta)
    return lib().orc_r2_D(C.byref(pb.c()), _dptr(th))


def loss_grad(pb: Problem, theta):
    """(L, dL/dtheta, dL/d(S0,I0,R0,D0)) by the discrete adjoint of the Euler map."""
    th = _f64(theta)
    g = np.zeros(pb.n_params)
    gu = np.zeros(4)
    L = lib().orc_loss_grad(C.byref(pb.c()), _dptr(th), _dptr(g), _dptr(gu))
    return L, g, gu


def forecast(pb: Problem, theta, horizon: int) -> np.ndarray:
    th = _f64(theta)
    out = np.zeros(horizon)
    if lib().orc_forecast(C.byref(pb.c()), _dptr(th), int(horizon), _dptr(out)) != 0:
        raise ValueError("orc_forecast: bad arguments")
    return out


def _band_drops(k: int, fractions) -> list:
    """Sorted values the central band holding the fraction f of k values leaves out at either end:
    floor(k (1 - f) / 2) (the small offset keeps e.g. k = 1000, f = 0.9 at exactly 50)."""
    return [int(np.floor(k * (1.0 - f) / 2.0 + 1e-9)) for f in fractions]


def ensemble_bands(pb: Problem, thetas, horizon: int, fractions=(0.95, 0.9, 0.5)) -> dict:
    """Per-day summaries of an ensemble of parameter vectors (Sec. 4.2): each member simulated
    over the window and `horizon` more days; per day the values of beta(t) (at the day's first
    step), R0(t) = beta(t) / (gamma + mu), S, I, R, D sorted over the members, the median (mean
    of the two middle values for an even count) and, for each fraction f, the central band that
    leaves floor(k (1 - f) / 2) sorted values out at either end.  Returns {quantity: [n_days,
    1 + 2 len(fractions)]} with columns median, low_0, high_0, ..."""
    th = np.atleast_2d(_f64(thetas))
    k = th.shape[0]
    n_days = pb.days + 1 + int(horizon)
    gi = 4 if pb.beta_form == BETA_RAMP else pb.K
    vals = {q: np.zeros((n_days, k)) for q in ("beta", "R0", "S", "I", "R", "D")}
    for j in range(k):
        tr = simulate(pb, th[j], n_days - 1)
        beta = np.array([beta_at(pb, th[j], d * pb.spd) for d in range(n_days)])
        vals["beta"][:, j] = beta
        vals["R0"][:, j] = beta / (th[j, gi] + th[j, gi + 1])
        for q in "SIRD":
            vals[q][:, j] = tr[q]
    drops = _band_drops(k, fractions)
    out = {}
    for q, v in vals.items():
        v = np.sort(v, axis=1)
        med = v[:, k // 2] if k % 2 else (v[:, k // 2 - 1] + v[:, k // 2]) * 0.5
        cols = [med]
        for dr in drops:
            cols += [v[:, dr], v[:, k - 1 - dr]]
        out[q] = np.stack(cols, axis=1)
    return out


def parameter_bands(pb: Problem, thetas, fractions=(0.95, 0.9, 0.5)) -> np.ndarray:
    """Stability of the fitted parameters over repeated calibrations (Sec. 4.2): for each
    parameter, its values over the k members sorted, the median (mean of the two middle values for
    an even count) and, for each fraction f, the central band that leaves floor(k (1 - f) / 2)
    sorted values out at either end -- the summary ensemble_bands gives per day.  The ramp's change
    times enter as t1 = min and t2 = max of the pair, the order the model uses them in (eq. (beta)).
    Returns [P, 1 + 2 len(fractions)] with columns median, low_0, high_0, ..."""
    th = np.array(np.atleast_2d(_f64(thetas)), dtype=np.float64)
    k, P = th.shape
    if P != pb.n_params:
        raise ValueError(f"thetas must be [k, {pb.n_params}]")
    if pb.beta_form == BETA_RAMP:
        ta, tb = th[:, 2].copy(), th[:, 3].copy()
        th[:, 2] = np.minimum(ta, tb)
        th[:, 3] = np.maximum(ta, tb)
    drops = _band_drops(k, fractions)
    out = np.zeros((P, 1 + 2 * len(drops)))
    for d in range(P):
        v = np.sort(th[:, d])
        out[d, 0] = v[k // 2] if k % 2 else (v[k // 2 - 1] + v[k // 2]) * 0.5
        for b, dr in enumerate(drops):
            out[d, 1 + 2 * b] = v[dr]
            out[d, 2 + 2 * b] = v[k - 1 - dr]
    return out


class PSO:
    """Synchronous PSO of Sec. 3.3 with particle-major FP64 state arrays.  p_offset: the swarm
    is particles p_offset .. p_offset + M - 1 of a larger one, numbered so in the random-number
    counter (its gbest is then the caller's to set between steps)."""

    def __init__(self, pb: Problem | None, M: int, zlb, zub, logdim=None, w=0.5, c1=0.5, c2=0.5,
                 seed: int = 0, stream: int = 0, store_f32: bool = False, objective_kind: int = OBJ_SIRD,
                 p_offset: int = 0):
        self.pb = pb
        self.zlb = _f64(zlb)
        self.zub = _f64(zub)
        P = self.zlb.size
        self.logdim = np.ascontiguousarray(np.zeros(P, np.int32) if logdim is None else np.asarray(logdim, np.int32))
        self.cfg = _PsoCfg(int(M), P, float(w), float(c1), float(c2), _dptr(self.zlb), _dptr(self.zub),
                           self.logdim.ctypes.data_as(C.POINTER(C.c_int)), int(seed) & (2**64 - 1),
                           int(stream) & 0xFFFFFFFF, int(store_f32), int(objective_kind), int(p_offset))
        self.M, self.P = int(M), P
        self.x = np.zeros((M, P))
        self.v = np.zeros((M, P))
        self.pbest = np.zeros((M, P))
        self.pbest_f = np.zeros(M)
        self.gbest = np.zeros(P)
        self.st = _PsoState(_dptr(self.x), _dptr(self.v), _dptr(self.pbest), _dptr(self.pbest_f),
                            _dptr(self.gbest), 0, 0.0, 0)
        self._cpb = pb.c() if pb is not None else _Problem()
        self._cpb_p = C.byref(self._cpb)

    @property
    def gbest_idx(self) -> int:
        return self.st.gbest_idx

    @property
    def gbest_f(self) -> float:
        return self.st.gbest_f

    @property
    def iter(self) -> int:
        return self.st.iter

    def init(self):
        lib().orc_pso_init(C.byref(self.cfg), self._cpb_p, C.byref(self.st))
        return self

    def step(self, n: int = 1):
        for _ in range(n):
            lib().orc_pso_step(C.byref(self.cfg), self._cpb_p, C.byref(self.st))
        return self

    def set_state(self, x, v, pbest, pbest_f, gbest_idx: int, iteration: int):
        """Loads a swarm state (particle-major); gbest is taken from pbest[gbest_idx]."""
        self.x[...] = x
        self.v[...] = v
        self.pbest[...] = pbest
        self.pbest_f[...] = pbest_f
        self.st.gbest_idx = int(gbest_idx)
        self.st.gbest_f = float(self.pbest_f[gbest_idx])
        self.gbest[...] = self.pbest[gbest_idx]
        self.st.iter = int(iteration)
        return self

    def objective(self, z) -> float:
        z = _f64(z)
        return lib().orc_objective(C.byref(self.cfg), self._cpb_p, _dptr(z))

    def reeval_topk(self, k: int):
        f = C.c_double()
        idx = lib().orc_reeval_topk(C.byref(self.cfg), self._cpb_p, C.byref(self.st), int(k), C.byref(f))
        return idx, f.value

    def decode(self, z) -> np.ndarray:
        z = np.asarray(z, dtype=np.float64)
        return np.where(self.logdim.astype(bool), np.exp(z), z)


def argmin(f) -> int:
    f = _f64(f)
    return lib().orc_argmin(_dptr(f), f.size)

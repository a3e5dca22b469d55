"""Thin ctypes binding of libnrs (include/nrs.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``csrc/``.  Tensors are torch CUDA tensors (device memory); the context's
work is enqueued on the torch stream that is current when it is created.
If libnrs.so has not been built, importing this module raises: there is no
CPU or library fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnrs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2001_06468_gb300.build`")

_lib = ctypes.CDLL(LIB_PATH)

NRS_OK, NRS_EINVAL, NRS_ENOMEM, NRS_ECUDA = 0, -1, -2, -3
NRS_ESINGULAR, NRS_ENOCONV, NRS_ENONFINITE, NRS_ETIMEOUT = -4, -5, -6, -7
STATUS_NAMES = {0: "NRS_OK", -1: "NRS_EINVAL", -2: "NRS_ENOMEM", -3: "NRS_ECUDA",
                -4: "NRS_ESINGULAR", -5: "NRS_ENOCONV", -6: "NRS_ENONFINITE", -7: "NRS_ETIMEOUT"}
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
# largest sizes nrs_nearest_build_static accepts (NRS_STATIC_MAX_* in include/nrs.h)
NRS_STATIC_LIMITS = {"N": 65536, "Q": 1048576, "bodies": 1024}
FREE, PRESCRIBED, STATIC = 0, 1, 2

EXPORTS = ["nrs_create", "nrs_destroy", "nrs_last_error", "nrs_sizes", "nrs_set_state",
           "nrs_get_state", "nrs_set_external", "nrs_kinematics", "nrs_nearest_build",
           "nrs_assemble", "nrs_factor", "nrs_solve", "nrs_residual", "nrs_step", "nrs_sync", "nrs_counters",
           "nrs_residual_counters",
           "nrs_velocity", "nrs_set_tracers", "nrs_get_tracers", "nrs_dp_start",
           "nrs_dp_next_time", "nrs_dp_stage", "nrs_dp_info_get",
           "nrs_set_timing",
           "nrs_get_timing", "nrs_get_trace", "nrs_rank64_update", "nrs_nearest_build_static",
           "nrs_mlp_set_params", "nrs_mlp_get_params", "nrs_mlp_config", "nrs_mlp_eval",
           "nrs_mlp_adam", "nrs_mlp_features", "nrs_mlp_start",
           "nrs_batch_create", "nrs_batch_destroy", "nrs_batch_last_error", "nrs_batch_context",
           "nrs_batch_step", "nrs_batch_config", "nrs_batch_tune", "nrs_batch_info",
           "nrs_batch_plan"]
# the learned starting guess (NRS_MLP_* in include/nrs.h)
MLP_IN, MLP_HID, MLP_OUT = 17, 64, 3
MLP_PARAMS = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT
START_KINDS = {0: "cold", 1: "previous", 2: "learned"}
PHASES = ["kinematics", "nearest", "segments", "assemble", "border", "convert", "lu_panel",
          "lu_update", "trsv", "gemv", "krylov", "update", "lu_diag", "assemble32"]


class ProblemDesc(ctypes.Structure):
    _fields_ = [("nbodies", ctypes.c_int32),
                ("n_off", ctypes.POINTER(ctypes.c_int64)),
                ("q_off", ctypes.POINTER(ctypes.c_int64)),
                ("kind", ctypes.POINTER(ctypes.c_int32)),
                ("rigid", ctypes.POINTER(ctypes.c_int32)),
                ("U", ctypes.POINTER(ctypes.c_double)),
                ("Omega", ctypes.POINTER(ctypes.c_double)),
                ("eps", ctypes.c_double),
                ("mu", ctypes.c_double),
                ("nn_global", ctypes.c_int32),
                ("factor_prec", ctypes.c_int32),
                ("nb", ctypes.c_int32),
                ("tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32),
                ("max_inner", ctypes.c_int32),
                ("reuse_factor", ctypes.c_int32),
                ("reuse_max_inner", ctypes.c_int32),
                ("reuse_max_stages", ctypes.c_int32),
                ("warm_start", ctypes.c_int32),
                ("solve_mode", ctypes.c_int32),
                ("inner_tol", ctypes.c_double),
                ("factor_input", ctypes.c_int32),
                ("graph", ctypes.c_int32),
                ("factor_schedule", ctypes.c_int32),
                ("residual", ctypes.c_int32),
                ("arnoldi", ctypes.c_int32)]


class SolveReport(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("inner", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("backward_err", ctypes.c_double), ("last_update", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepReport(ctypes.Structure):
    _fields_ = [("stage", SolveReport * 2), ("ms_total", ctypes.c_double),
                ("factorizations", ctypes.c_int32), ("start", ctypes.c_int32 * 2),
                ("mlp_rel_err", ctypes.c_double), ("retried", ctypes.c_int32 * 2)]


class DpInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("h", ctypes.c_double), ("err", ctypes.c_double),
                ("stage", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("rejected", ctypes.c_int32), ("last_accepted", ctypes.c_int32),
                ("done", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Shapes(ctypes.Structure):
    _fields_ = [("xi", ctypes.c_void_p), ("Xiw", ctypes.c_void_p), ("xidot", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_sig = {
    "nrs_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ProblemDesc), _P]),
    "nrs_destroy": (ctypes.c_int, [_P]),
    "nrs_last_error": (ctypes.c_char_p, [_P]),
    "nrs_sizes": (ctypes.c_int, [_P, _I64P, _I64P, _I64P, _I64P]),
    "nrs_set_state": (ctypes.c_int, [_P, _P, _P]),
    "nrs_get_state": (ctypes.c_int, [_P, _P, _P]),
    "nrs_set_external": (ctypes.c_int, [_P, _P]),
    "nrs_kinematics": (ctypes.c_int, [_P, ctypes.POINTER(Shapes), _P, _P, _P]),
    "nrs_nearest_build": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "nrs_assemble": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64]),
    "nrs_factor": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "nrs_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(SolveReport)]),
    "nrs_residual": (ctypes.c_int, [_P, _P, _P, _P]),
    "nrs_step": (ctypes.c_int, [_P, ctypes.POINTER(Shapes), ctypes.POINTER(Shapes), ctypes.c_double,
                                _P, ctypes.POINTER(StepReport)]),
    "nrs_sync": (ctypes.c_int, [_P]),
    "nrs_counters": (ctypes.c_int, [_P, _I64P, _I64P, _I64P, _I64P, _I64P]),
    "nrs_residual_counters": (ctypes.c_int, [_P, _I64P, _I64P]),
    "nrs_velocity": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "nrs_set_tracers": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "nrs_get_tracers": (ctypes.c_int, [_P, _P]),
    "nrs_dp_start": (ctypes.c_int, [_P] + [ctypes.c_double] * 7),
    "nrs_dp_next_time": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "nrs_dp_stage": (ctypes.c_int, [_P, ctypes.POINTER(Shapes), _P, ctypes.POINTER(DpInfo)]),
    "nrs_dp_info_get": (ctypes.c_int, [_P, ctypes.POINTER(DpInfo)]),
    "nrs_set_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
    "nrs_rank64_update": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                         ctypes.c_int32]),
    "nrs_nearest_build_static": (ctypes.c_int, [_P, _P, ctypes.c_int32, _I64P, _I64P, ctypes.c_int32,
                                                _P, _P, _P, _P, _P]),
    "nrs_get_timing": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), _I64P, _I64P]),
    "nrs_get_trace": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int64, _I64P]),
    "nrs_mlp_set_params": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32]),
    "nrs_mlp_get_params": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int32), _P]),
    "nrs_mlp_config": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _P]),
    "nrs_mlp_eval": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P,
                                    ctypes.POINTER(ctypes.c_double)]),
    "nrs_mlp_adam": (ctypes.c_int, [_P, _P, ctypes.c_float]),
    "nrs_mlp_features": (ctypes.c_int, [_P, ctypes.POINTER(Shapes), _P, _P, _P, _P]),
    "nrs_mlp_start": (ctypes.c_int, [_P, _P, _P, _P]),
    "nrs_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ProblemDesc),
                                        ctypes.c_int32, _P]),
    "nrs_batch_destroy": (ctypes.c_int, [_P]),
    "nrs_batch_last_error": (ctypes.c_char_p, [_P]),
    "nrs_batch_context": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    "nrs_batch_step": (ctypes.c_int, [_P, ctypes.POINTER(Shapes), ctypes.POINTER(Shapes),
                                      ctypes.c_double, ctypes.POINTER(_P), ctypes.POINTER(StepReport)]),
    "nrs_batch_config": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]),
    "nrs_batch_tune": (ctypes.c_int, [_P, ctypes.POINTER(Shapes), ctypes.POINTER(Shapes),
                                      ctypes.c_double, ctypes.c_char_p,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_double)]),
    "nrs_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), _I64P]),
    "nrs_batch_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                      ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class NrsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t: Optional[torch.Tensor], dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _np_ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Context:
    """One NEAREST problem on the current CUDA device (see include/nrs.h)."""

    def __init__(self, n_off: Sequence[int], q_off: Sequence[int], kind: Sequence[int],
                 eps: float, mu: float = 1.0, rigid: Optional[Sequence[int]] = None,
                 U=None, Omega=None, nn_global: bool = False, factor_prec: str = "fp32",
                 tol: float = 0.0, max_outer: int = 0, max_inner: int = 0,
                 reuse_factor: bool = False, reuse_max_inner: int = 0, reuse_max_stages: int = 0,
                 warm_start: bool = False, solve_mode: str = "device", graph: bool = False,
                 inner_tol: float = 0.0, factor_input: str = "fp32",
                 factor_schedule: str = "auto", residual: str = "extended",
                 arnoldi: str = "fp64",
                 stream: Optional[torch.cuda.Stream] = None, _handle=None):
        d, self._keep = _make_desc(n_off, q_off, kind, eps, mu, rigid, U, Omega, nn_global,
                                   factor_prec, tol, max_outer, max_inner, reuse_factor,
                                   reuse_max_inner, reuse_max_stages, warm_start, solve_mode,
                                   graph, inner_tol, factor_input, factor_schedule, residual,
                                   arnoldi)
        self.stream = stream or torch.cuda.current_stream()
        self._owner = _handle is None
        if _handle is None:
            self._h = ctypes.c_void_p()
            st = _lib.nrs_create(ctypes.byref(self._h), ctypes.byref(d),
                                 ctypes.c_void_p(self.stream.cuda_stream))
            if st != NRS_OK:
                raise NrsError(st, "nrs_create failed")
        else:
            self._h = _handle
        N, Q, F, n = (ctypes.c_int64() for _ in range(4))
        _lib.nrs_sizes(self._h, ctypes.byref(N), ctypes.byref(Q), ctypes.byref(F), ctypes.byref(n))
        self.N, self.Q, self.F, self.n = N.value, Q.value, F.value, n.value
        self.nbodies = d.nbodies

    @classmethod
    def from_problem(cls, problem, factor_prec: str = "fp32", **kw) -> "Context":
        """Context for a ``synth.geometry.Problem`` (its body table and eps, mu)."""
        return cls(*_problem_args(problem), factor_prec=factor_prec, **kw)

    def close(self):
        if getattr(self, "_h", None) and self._h.value and getattr(self, "_owner", True):
            _lib.nrs_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != NRS_OK:
            raise NrsError(st, (_lib.nrs_last_error(self._h) or b"").decode())
        return st

    def last_error(self) -> str:
        return (_lib.nrs_last_error(self._h) or b"").decode()

    # -- state -------------------------------------------------------------
    def set_state(self, x0, B):
        x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(self.nbodies * 3)
        B = np.ascontiguousarray(B, dtype=np.float64).reshape(self.nbodies * 9)
        self._check(_lib.nrs_set_state(self._h, x0.ctypes.data, B.ctypes.data))

    def get_state(self):
        x0 = np.empty(self.nbodies * 3)
        B = np.empty(self.nbodies * 9)
        self._check(_lib.nrs_get_state(self._h, x0.ctypes.data, B.ctypes.data))
        return {"x0": x0.reshape(-1, 3), "B": B.reshape(-1, 3, 3)}

    def set_external(self, ext=None):
        if ext is None:
            self._check(_lib.nrs_set_external(self._h, None))
        else:
            e = np.ascontiguousarray(ext, dtype=np.float64).reshape(self.F * 6)
            self._check(_lib.nrs_set_external(self._h, e.ctypes.data))

    # -- the steps of the method --------------------------------------------
    @staticmethod
    def shapes(xi: torch.Tensor, Xiw: torch.Tensor, xidot: torch.Tensor) -> Shapes:
        s = Shapes()
        s.xi = _ptr(xi, torch.float64).value
        s.Xiw = _ptr(Xiw, torch.float64).value
        s.xidot = _ptr(xidot, torch.float64).value
        s._keep = (xi, Xiw, xidot)
        return s

    def kinematics(self, xi, Xiw, xidot):
        dev = xi.device
        x = torch.empty((self.N, 4), dtype=torch.float64, device=dev)
        Xw = torch.empty((self.Q, 4), dtype=torch.float64, device=dev)
        b = torch.empty(self.n, dtype=torch.float64, device=dev)
        s = self.shapes(xi, Xiw, xidot)
        self._check(_lib.nrs_kinematics(self._h, ctypes.byref(s), _ptr(x), _ptr(Xw), _ptr(b)))
        return x, Xw, b

    def nearest_build(self, x, Xw):
        dev = x.device
        nn = torch.empty(self.Q, dtype=torch.int32, device=dev)
        seg_ptr = torch.empty(self.N + 1, dtype=torch.int32, device=dev)
        perm = torch.empty(self.Q, dtype=torch.int32, device=dev)
        self._check(_lib.nrs_nearest_build(self._h, _ptr(x, torch.float64), _ptr(Xw, torch.float64),
                                           _ptr(nn), _ptr(seg_ptr), _ptr(perm)))
        return nn, seg_ptr, perm

    def assemble(self, x, Xw, want_matrix: bool = True):
        """Assemble A (kept in the context); returns the n x n FP64 matrix as a
        tensor At with At[j, i] = A[i, j] (column-major storage) if asked."""
        At = torch.empty((self.n, self.n), dtype=torch.float64, device=x.device) if want_matrix else None
        self._check(_lib.nrs_assemble(self._h, _ptr(x, torch.float64), _ptr(Xw, torch.float64),
                                      _ptr(At), self.n))
        return At

    def factor(self, prec: str = "fp32") -> int:
        info = ctypes.c_int32(0)
        st = _lib.nrs_factor(self._h, PREC[prec], ctypes.byref(info))
        if st not in (NRS_OK, NRS_ESINGULAR):
            self._check(st)
        return info.value

    def solve(self, b: torch.Tensor, x0: Optional[torch.Tensor] = None, check: bool = True):
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        x = torch.empty_like(b)
        reps = (SolveReport * nrhs)()
        st = _lib.nrs_solve(self._h, _ptr(b, torch.float64), _ptr(x), nrhs, _ptr(x0), reps)
        if check:
            self._check(st)
        return x, [r.as_dict() for r in reps]

    def residual(self, b: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        """r = b - A x (device float64, length n) with the last assembled FP64
        matrix, in the context's residual precision."""
        if b.shape != (self.n,) or x.shape != (self.n,):
            raise ValueError(f"residual: b and x must have shape ({self.n},)")
        r = torch.empty_like(b)
        self._check(_lib.nrs_residual(self._h, _ptr(b, torch.float64), _ptr(x, torch.float64),
                                      _ptr(r)))
        return r

    def step(self, s0: Shapes, s_half: Shapes, dt: float, sol: Optional[torch.Tensor] = None,
             report: bool = True, check: bool = True):
        rep = StepReport() if report else None
        st = _lib.nrs_step(self._h, ctypes.byref(s0), ctypes.byref(s_half), float(dt), _ptr(sol),
                           ctypes.byref(rep) if rep is not None else None)
        if check:
            self._check(st)
        if rep is None:
            return None
        return {"stages": [rep.stage[0].as_dict(), rep.stage[1].as_dict()], "ms": rep.ms_total,
                "status": st, "factorizations": rep.factorizations,
                "start": [START_KINDS.get(rep.start[0], rep.start[0]),
                          START_KINDS.get(rep.start[1], rep.start[1])],
                "mlp_rel_err": rep.mlp_rel_err, "retried": [rep.retried[0], rep.retried[1]]}

    def sync(self):
        return self._check(_lib.nrs_sync(self._h))

    def velocity(self, xp: torch.Tensor, f: torch.Tensor, Xw: Optional[torch.Tensor] = None):
        """Fluid velocity (P, 4) at device field points xp (P, 4) from the force
        density f (device, 3 per force point); Xw: lab-frame quadrature points
        (None = those of the last step stage)."""
        P = xp.shape[0]
        u = torch.empty((P, 4), dtype=torch.float64, device=xp.device)
        self._check(_lib.nrs_velocity(self._h, _ptr(Xw, torch.float64), _ptr(xp, torch.float64), P,
                                      _ptr(f, torch.float64), _ptr(u)))
        return u

    def set_tracers(self, xp):
        """Tracers (host array (P, 4)) advanced by nrs_step; None or empty removes them."""
        a = np.zeros((0, 4)) if xp is None else np.ascontiguousarray(xp, dtype=np.float64).reshape(-1, 4)
        self._check(_lib.nrs_set_tracers(self._h, a.ctypes.data if len(a) else None, len(a)))
        self.n_tracers = len(a)

    def get_tracers(self):
        out = np.empty((getattr(self, "n_tracers", 0), 4), dtype=np.float64)
        self._check(_lib.nrs_get_tracers(self._h, out.ctypes.data if len(out) else None))
        return out

    # -- adaptive Dormand-Prince stepping ----------------------------------
    def dp_start(self, t0, t_end, h0, rtol, atol, h_min=1e-8, h_max=None):
        self._check(_lib.nrs_dp_start(self._h, float(t0), float(t_end), float(h0), float(rtol),
                                      float(atol), float(h_min),
                                      float(h_max if h_max is not None else t_end - t0)))

    def dp_next_time(self) -> float:
        t = ctypes.c_double()
        self._check(_lib.nrs_dp_next_time(self._h, ctypes.byref(t)))
        return t.value

    def dp_stage(self, s: "Shapes", sol: Optional[torch.Tensor] = None):
        info = DpInfo()
        self._check(_lib.nrs_dp_stage(self._h, ctypes.byref(s), _ptr(sol), ctypes.byref(info)))
        return info.as_dict()

    def dp_info(self):
        info = DpInfo()
        self._check(_lib.nrs_dp_info_get(self._h, ctypes.byref(info)))
        return info.as_dict()

    def dp_integrate(self, shapes_at, t0, t_end, h0, rtol, atol, h_min=1e-8, h_max=None,
                     max_stages=100000):
        """Integrate from the current state to t_end: ``shapes_at(t)`` returns the
        device shapes (an nrs.Shapes) at time t.  Returns the final dp_info."""
        self.dp_start(t0, t_end, h0, rtol, atol, h_min, h_max)
        info = self.dp_info()
        for _ in range(max_stages):
            if info["done"]:
                break
            info = self.dp_stage(shapes_at(self.dp_next_time()))
        return info

    def counters(self):
        """{'factorizations', 'solves', 'outer', 'inner', 'retries'} since creation."""
        v = [ctypes.c_int64() for _ in range(5)]
        self._check(_lib.nrs_counters(self._h, *(ctypes.byref(x) for x in v)))
        return dict(zip(("factorizations", "solves", "outer", "inner", "retries"),
                        (x.value for x in v)))

    def residual_counters(self):
        """{'exact', 'working'}: residuals the refinement formed since creation."""
        v = [ctypes.c_int64() for _ in range(2)]
        self._check(_lib.nrs_residual_counters(self._h, *(ctypes.byref(x) for x in v)))
        return {"exact": v[0].value, "working": v[1].value}

    def rank64_update(self, Mt: torch.Tensor, C: torch.Tensor, Rt: torch.Tensor, prec: str = "tf32"):
        """M -= C Rt^T in place; Mt is the (n_cols, lda) storage of the
        column-major M (Mt[j, i] = M[i, j]); C and Rt are (n, 64) float32."""
        n = C.shape[0]
        self._check(_lib.nrs_rank64_update(self._h, _ptr(Mt, torch.float32), Mt.shape[1], n,
                                           _ptr(C, torch.float32), _ptr(Rt, torch.float32),
                                           PREC[prec]))

    # -- learned starting guess ---------------------------------------------
    def mlp_set_params(self, params, adam_m=None, adam_v=None, t: int = 0):
        """Load the MLP parameters (and Adam state) from host arrays."""
        def f32(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float32).reshape(MLP_PARAMS)
            return a
        p, m, v = f32(params), f32(adam_m), f32(adam_v)
        self._check(_lib.nrs_mlp_set_params(self._h, p.ctypes.data,
                                            None if m is None else m.ctypes.data,
                                            None if v is None else v.ctypes.data, int(t)))

    def mlp_get_params(self):
        """{'params', 'adam_m', 'adam_v', 't', 'scales'} (host copies)."""
        p = np.empty(MLP_PARAMS, np.float32)
        m = np.empty(MLP_PARAMS, np.float32)
        v = np.empty(MLP_PARAMS, np.float32)
        sc = np.empty(3, np.float64)
        t = ctypes.c_int32()
        self._check(_lib.nrs_mlp_get_params(self._h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                            ctypes.byref(t), sc.ctypes.data))
        return {"params": p, "adam_m": m, "adam_v": v, "t": t.value, "scales": sc}

    def mlp_config(self, train_iters: int = 0, predict: bool = False, lr: float = 1e-3,
                   scales=None):
        sc = None if scales is None else np.ascontiguousarray(scales, dtype=np.float64).reshape(3)
        self._check(_lib.nrs_mlp_config(self._h, int(train_iters), int(bool(predict)), float(lr),
                                        None if sc is None else sc.ctypes.data))

    def mlp_eval(self, X: torch.Tensor, T: Optional[torch.Tensor] = None, grad: bool = False,
                 loss: bool = False):
        """Forward (and, with T, loss and gradient) on device features X (npts, 17)."""
        npts = X.shape[0]
        Y = torch.empty((npts, MLP_OUT), dtype=torch.float32, device=X.device)
        G = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device) if grad else None
        lo = ctypes.c_double(0.0)
        self._check(_lib.nrs_mlp_eval(self._h, _ptr(X, torch.float32), _ptr(T, torch.float32),
                                      npts, _ptr(Y), _ptr(G),
                                      ctypes.byref(lo) if loss else None))
        return Y, G, (lo.value if loss else None)

    def mlp_adam(self, G: torch.Tensor, lr: float):
        self._check(_lib.nrs_mlp_adam(self._h, _ptr(G, torch.float32), float(lr)))

    def mlp_features(self, s: Shapes, vprev: Optional[torch.Tensor] = None,
                     sol: Optional[torch.Tensor] = None, device="cuda"):
        """Features (N, 17) of the shapes s and, with sol, the targets (N, 3)."""
        X = torch.empty((self.N, MLP_IN), dtype=torch.float32, device=device)
        T = torch.empty((self.N, MLP_OUT), dtype=torch.float32, device=device) if sol is not None else None
        self._check(_lib.nrs_mlp_features(self._h, ctypes.byref(s), _ptr(vprev, torch.float64),
                                          _ptr(sol, torch.float64), _ptr(X), _ptr(T)))
        return X, T

    def mlp_start(self, Y: torch.Tensor, vprev: Optional[torch.Tensor] = None):
        x0 = torch.empty(self.n, dtype=torch.float64, device=Y.device)
        self._check(_lib.nrs_mlp_start(self._h, _ptr(Y, torch.float32), _ptr(vprev, torch.float64),
                                       _ptr(x0)))
        return x0

    def set_timing(self, enable: bool = True):
        self._check(_lib.nrs_set_timing(self._h, int(bool(enable))))

    def get_trace(self):
        """[(phase, begin_ms, end_ms)] of the spans timed since timing was
        enabled, in recording order; call before get_timing (which clears)."""
        cnt = ctypes.c_int64()
        self._check(_lib.nrs_get_trace(self._h, None, None, None, 0, ctypes.byref(cnt)))
        m = cnt.value
        ph = (ctypes.c_int32 * max(m, 1))()
        t0 = (ctypes.c_double * max(m, 1))()
        t1 = (ctypes.c_double * max(m, 1))()
        self._check(_lib.nrs_get_trace(self._h, ph, t0, t1, m, ctypes.byref(cnt)))
        return [(PHASES[ph[i]], t0[i], t1[i]) for i in range(min(m, cnt.value))]

    def get_timing(self):
        """{phase: (ms, spans)} since timing was enabled, and the kernel count."""
        ms = (ctypes.c_double * len(PHASES))()
        spans = (ctypes.c_int64 * len(PHASES))()
        launches = ctypes.c_int64()
        self._check(_lib.nrs_get_timing(self._h, ms, spans, ctypes.byref(launches)))
        return {p: (ms[i], spans[i]) for i, p in enumerate(PHASES)}, launches.value


def _problem_args(problem):
    n_off = np.cumsum([0] + [b.N for b in problem.bodies])
    q_off = np.cumsum([0] + [b.Q for b in problem.bodies])
    return (n_off, q_off, [b.kind for b in problem.bodies], problem.eps, problem.mu,
            [int(b.rigid) for b in problem.bodies], np.array([b.U for b in problem.bodies]),
            np.array([b.Omega for b in problem.bodies]), problem.nn_global)


def _make_desc(n_off, q_off, kind, eps, mu=1.0, rigid=None, U=None, Omega=None, nn_global=False,
               factor_prec="fp32", tol=0.0, max_outer=0, max_inner=0, reuse_factor=False,
               reuse_max_inner=0, reuse_max_stages=0, warm_start=False, solve_mode="device",
               graph=False, inner_tol=0.0, factor_input="fp32", factor_schedule="auto",
               residual="extended", arnoldi="fp64"):
    """An nrs_problem_desc and the host arrays it points to (keep them alive)."""
    n_off = np.ascontiguousarray(n_off, dtype=np.int64)
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    nb = len(kind)
    rigid = None if rigid is None else np.ascontiguousarray(rigid, dtype=np.int32)
    U = None if U is None else np.ascontiguousarray(U, dtype=np.float64).reshape(nb * 3)
    Om = None if Omega is None else np.ascontiguousarray(Omega, dtype=np.float64).reshape(nb * 3)
    d = ProblemDesc()
    d.nbodies = nb
    d.n_off = _np_ptr(n_off, ctypes.c_int64)
    d.q_off = _np_ptr(q_off, ctypes.c_int64)
    d.kind = _np_ptr(kind, ctypes.c_int32)
    d.rigid = None if rigid is None else _np_ptr(rigid, ctypes.c_int32)
    d.U = None if U is None else _np_ptr(U, ctypes.c_double)
    d.Omega = None if Om is None else _np_ptr(Om, ctypes.c_double)
    d.eps, d.mu = float(eps), float(mu)
    d.nn_global = int(bool(nn_global))
    d.factor_prec = PREC[factor_prec]
    d.nb = 0
    d.tol = float(tol)
    d.max_outer, d.max_inner = int(max_outer), int(max_inner)
    d.reuse_factor, d.warm_start = int(bool(reuse_factor)), int(bool(warm_start))
    d.reuse_max_inner, d.reuse_max_stages = int(reuse_max_inner), int(reuse_max_stages)
    d.solve_mode = {"device": 0, "host": 1}[solve_mode]
    d.graph = int(bool(graph))
    d.inner_tol = float(inner_tol)
    d.factor_input = {"fp32": 0, "rounded": 1}[factor_input]
    # two-level updates from split-TF32 operands (3) or scaled FP16 pairs (4)
    d.factor_schedule = {"auto": 0, "fused": 1, "streams": 2, "two_level_tf32": 3,
                         "two_level": 4}[factor_schedule]
    # "extended": to about u^2 (exact products, see nrs_residual); "fp64": plain
    d.residual = {"extended": 0, "fp64": 1}[residual]
    # GMRES products with the FP64 matrix, or with its float-pair copy ("df")
    d.arnoldi = {"fp64": 0, "df": 1}[arnoldi]
    return d, (n_off, q_off, kind, rigid, U, Om)


class Batch:
    """Many independent problems stepped together through one CUDA graph
    (nrs_batch_* in include/nrs.h)."""

    def __init__(self, problems, factor_prec: str = "tf32", stream=None, **kw):
        descs = (ProblemDesc * len(problems))()
        self._keep = []
        for i, pr in enumerate(problems):
            d, keep = _make_desc(*_problem_args(pr), factor_prec=factor_prec, **kw)
            descs[i] = d
            self._keep.append(keep)
        self.stream = stream or torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        st = _lib.nrs_batch_create(ctypes.byref(self._h), descs, len(problems),
                                   ctypes.c_void_p(self.stream.cuda_stream))
        if st != NRS_OK:
            raise NrsError(st, "nrs_batch_create failed")
        self.count = len(problems)
        self.contexts = []
        for i, pr in enumerate(problems):
            h = ctypes.c_void_p()
            self._check(_lib.nrs_batch_context(self._h, i, ctypes.byref(h)))
            self.contexts.append(Context(*_problem_args(pr), factor_prec=factor_prec,
                                         stream=self.stream, _handle=h, **kw))

    def _check(self, st):
        if st != NRS_OK:
            raise NrsError(st, (_lib.nrs_batch_last_error(self._h) or b"").decode())
        return st

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            for c in self.contexts:
                c._h = ctypes.c_void_p()
            _lib.nrs_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _shapes(pairs):
        s0 = (Shapes * len(pairs))()
        sh = (Shapes * len(pairs))()
        for i, (a, b) in enumerate(pairs):
            s0[i] = Context.shapes(*a)
            sh[i] = Context.shapes(*b)
        return s0, sh

    def step(self, pairs, dt: float, sols=None, report: bool = False, check: bool = True):
        """pairs[i] = ((xi, Xiw, xidot) at t, (xi, Xiw, xidot) at t + dt/2) device tensors."""
        s0, sh = self._shapes(pairs)
        sp = None
        if sols is not None:
            sp = (_P * self.count)(*[None if x is None else _ptr(x, torch.float64).value
                                     for x in sols])
        reps = (StepReport * self.count)() if report else None
        st = _lib.nrs_batch_step(self._h, s0, sh, float(dt), sp, reps)
        if check:
            self._check(st)
        if not report:
            return None
        return [{"stages": [r.stage[0].as_dict(), r.stage[1].as_dict()], "ms": r.ms_total,
                 "factorizations": r.factorizations} for r in reps]

    def config(self, chains: int, grid: int):
        ch = (ctypes.c_int32 * self.count)()
        self._check(_lib.nrs_batch_config(self._h, int(chains), int(grid), ch))
        return list(ch)

    def tune(self, pairs, dt: float, cache_path: Optional[str] = None):
        s0, sh = self._shapes(pairs)
        k, g, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        self._check(_lib.nrs_batch_tune(self._h, s0, sh, float(dt),
                                        None if cache_path is None else cache_path.encode(),
                                        ctypes.byref(k), ctypes.byref(g), ctypes.byref(ms)))
        return {"chains": k.value, "grid": g.value, "ms": ms.value}

    def info(self):
        k, g, nk = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        self._check(_lib.nrs_batch_info(self._h, ctypes.byref(k), ctypes.byref(g), ctypes.byref(nk)))
        return {"chains": k.value, "grid": g.value, "graph_kernels": nk.value}


def batch_plan(cost, chains: int):
    """nrs_batch_plan: (chain of each problem, order) of the LPT plan (host only)."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    ch = np.zeros(len(c), np.int32)
    order = np.zeros(len(c), np.int32)
    st = _lib.nrs_batch_plan(_np_ptr(c, ctypes.c_double), len(c), int(chains),
                             _np_ptr(ch, ctypes.c_int32), _np_ptr(order, ctypes.c_int32))
    if st != NRS_OK:
        raise NrsError(st, "nrs_batch_plan failed")
    return ch, order


def nearest_build_static(x: torch.Tensor, Xw: torch.Tensor, n_off, q_off, global_: bool = False,
                         nn: Optional[torch.Tensor] = None, seg_ptr: Optional[torch.Tensor] = None,
                         perm: Optional[torch.Tensor] = None, status: Optional[torch.Tensor] = None,
                         stream: Optional[torch.cuda.Stream] = None, check: bool = True):
    """nrs_nearest_build_static: the nearest-neighbour map and segments with
    no device allocation inside the library (the outputs are the caller's;
    pass preallocated tensors, status included, to allocate nothing at all).
    The tensors are checked against the offsets and must live on the current
    device (the one the library uses) before anything is launched.  With
    ``check``, the stream is synchronised and a non-finite input raises
    NRS_ENONFINITE.  Returns (nn, seg_ptr, perm)."""
    n_off = np.ascontiguousarray(n_off, dtype=np.int64)
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    N, Q = int(n_off[-1]), int(q_off[-1])
    dev = torch.device("cuda", torch.cuda.current_device())
    nn = nn if nn is not None else torch.empty(Q, dtype=torch.int32, device=dev)
    seg_ptr = seg_ptr if seg_ptr is not None else torch.empty(N + 1, dtype=torch.int32, device=dev)
    perm = perm if perm is not None else torch.empty(Q, dtype=torch.int32, device=dev)
    status = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    if tuple(x.shape) != (N, 4) or tuple(Xw.shape) != (Q, 4):
        raise ValueError(f"x must be ({N}, 4) and Xw ({Q}, 4), got {tuple(x.shape)}, {tuple(Xw.shape)}")
    if nn.numel() < Q or perm.numel() < Q or seg_ptr.numel() < N + 1 or status.numel() < 1:
        raise ValueError("nn and perm need Q entries, seg_ptr N + 1, status 1")
    for t in (x, Xw, nn, seg_ptr, perm, status):
        if t.device != dev:
            raise ValueError(f"every tensor must be on the current device {dev}, got {t.device}")
    st = stream or torch.cuda.current_stream()
    rc = _lib.nrs_nearest_build_static(_ptr(x, torch.float64), _ptr(Xw, torch.float64),
                                       len(n_off) - 1, _np_ptr(n_off, ctypes.c_int64),
                                       _np_ptr(q_off, ctypes.c_int64), int(bool(global_)),
                                       _ptr(nn, torch.int32), _ptr(seg_ptr, torch.int32),
                                       _ptr(perm, torch.int32), _ptr(status, torch.int32),
                                       ctypes.c_void_p(st.cuda_stream))
    if rc != NRS_OK:
        raise NrsError(rc, "nrs_nearest_build_static failed")
    if check:
        st.synchronize()
        if int(status[0].item()) & 4:
            raise NrsError(NRS_ENONFINITE, "nrs_nearest_build_static: non-finite coordinates")
    return nn, seg_ptr, perm


def shapes_to_device(shapes: dict, device="cuda"):
    """Copy packed body-frame arrays (synth.geometry.pack_shapes) to the device."""
    return tuple(torch.from_numpy(np.ascontiguousarray(shapes[k])).to(device)
                 for k in ("x", "Xw", "xidot"))

"""FP64 CPU oracle of the NEAREST regularized-stokeslet method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The product
library never calls it, and it shares no code with the CUDA sources: the two
meet only in the seeded inputs of ``synth``.

The arithmetic lives in ``nrs_oracle.c`` (plain C, double precision, no
fused multiply-add); this module compiles it on first use with gcc and wraps
it with numpy.  Orchestration of one right-hand-side evaluation of the
swimming IVP (Sec. 4 of the paper: build A_s, build A, solve) and of the
explicit-midpoint step is written here in Python.

Every function below cites the passage of Gallagher & Smith, "Passively
parallel regularized stokeslets" that it follows.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FREE, PRESCRIBED, STATIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile nrs_oracle.c into liboracle.so (gcc, -O2, no FP contraction,
    OpenMP).  Rebuilds when the source is newer than the library."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            I32 = ctypes.POINTER(ctypes.c_int32)
            I64 = ctypes.POINTER(ctypes.c_int64)
            i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "or_threads": (c_int, []),
                "or_stokeslet": (None, [D, c_double, D]),
                "or_oseen": (None, [D, D]),
                "or_blob": (c_double, [D, c_double]),
                "or_pressure": (None, [D, c_double, D]),
                "or_nearest": (c_int, [c_int, I64, I64, D, D, c_int, I32]),
                "or_segments": (None, [i64, i64, I32, I32, I32]),
                "or_rigid_map": (None, [i64, D, D, D, D]),
                "or_assemble_stokeslet": (None, [i64, D, i64, D, I32, c_double, c_double, D, i64]),
                "or_assemble_rows": (None, [i64, I64, i64, D, i64, D, I32, c_double, c_double, D,
                                            i64]),
                "or_velocity": (None, [i64, D, i64, D, I32, D, c_double, c_double, D]),
                "or_border": (None, [c_int, I64, I64, I32, D, D, I32, D, D, i64]),
                "or_rhs": (None, [c_int, I64, I32, D, D, D, D, D, D, D, D]),
                "or_lu": (c_int, [i64, D, i64, I32]),
                "or_lu_solve": (None, [i64, D, i64, I32, D, c_int]),
                "or_residual_dd": (None, [i64, D, i64, D, D, D]),
                "or_refine": (c_int, [i64, D, i64, D, I32, D, D, c_int, c_double]),
                "or_cond1": (c_double, [i64, D, i64, D, I32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and (a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"])
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i32(a: np.ndarray):
    assert a.dtype == np.int32
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i64(a: np.ndarray):
    assert a.dtype == np.int64
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().or_threads())


# --------------------------------------------------------------------------
# Sec. 2 / Sec. 3 kernels
# --------------------------------------------------------------------------

def stokeslet(r, eps: float) -> np.ndarray:
    """Regularized stokeslet S^eps_jk(r) (Sec. 3), 3x3."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    S = np.empty(9)
    _load().or_stokeslet(_d(r), float(eps), _d(S))
    return S.reshape(3, 3)


def oseen(r) -> np.ndarray:
    """Singular stokeslet (Oseen tensor) S_jk(r) (Sec. 2), 3x3."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    S = np.empty(9)
    _load().or_oseen(_d(r), _d(S))
    return S.reshape(3, 3)


def blob(r, eps: float) -> float:
    """Blob phi_eps(r) = 15 eps^4 / (8 pi (r^2+eps^2)^{7/2}) (Sec. 3)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    return float(_load().or_blob(_d(r), float(eps)))


def pressure(r, eps: float) -> np.ndarray:
    """Regularized pressure numerator P^eps_k(r) (Sec. 3)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    P = np.empty(3)
    _load().or_pressure(_d(r), float(eps), _d(P))
    return P


# --------------------------------------------------------------------------
# nearest neighbours and segments (Sec. 3)
# --------------------------------------------------------------------------

def nearest(x: np.ndarray, Xw: np.ndarray, n_off: np.ndarray, q_off: np.ndarray,
            global_: bool = False) -> np.ndarray:
    """n-hat(q) = argmin_n |x[n] - X[q]| (Sec. 3), per body unless global_,
    lowest index on exact ties.  x (N,4), Xw (Q,4) float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    Xw = np.ascontiguousarray(Xw, dtype=np.float64)
    n_off = np.ascontiguousarray(n_off, dtype=np.int64)
    q_off = np.ascontiguousarray(q_off, dtype=np.int64)
    nn = np.empty(len(Xw), dtype=np.int32)
    rc = _load().or_nearest(len(n_off) - 1, _i64(n_off), _i64(q_off), _d(x), _d(Xw),
                            int(bool(global_)), _i32(nn))
    if rc != 0:
        raise ValueError("a body has quadrature points but no force points")
    return nn


def segments(nn: np.ndarray, N: int) -> Tuple[np.ndarray, np.ndarray]:
    """Columns of nu as CSR: (seg_ptr (N+1), perm (Q)), q ascending per segment."""
    nn = np.ascontiguousarray(nn, dtype=np.int32)
    seg_ptr = np.empty(N + 1, dtype=np.int32)
    perm = np.empty(len(nn), dtype=np.int32)
    _load().or_segments(N, len(nn), _i32(nn), _i32(seg_ptr), _i32(perm))
    return seg_ptr, perm


# --------------------------------------------------------------------------
# kinematics, assembly, right-hand side (Sec. 3 eq. nnrsbie; Sec. 4)
# --------------------------------------------------------------------------

def rigid_map(p: np.ndarray, x0: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Lab-frame rows x0 + B p (column 3 copied): the state Y = [X0; B] of
    Sec. 4 placing a body-frame cloud."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.empty_like(p)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    _load().or_rigid_map(len(p), _d(p), _d(x0), _d(B), _d(out))
    return out


def lab_frame(shapes: Dict[str, np.ndarray], Y: Dict[str, np.ndarray]):
    """Map every body's packed body-frame clouds to the lab frame."""
    x = np.empty_like(shapes["x"])
    Xw = np.empty_like(shapes["Xw"])
    n_off, q_off = shapes["n_off"], shapes["q_off"]
    for b in range(len(n_off) - 1):
        x[n_off[b]:n_off[b + 1]] = rigid_map(shapes["x"][n_off[b]:n_off[b + 1]], Y["x0"][b], Y["B"][b])
        Xw[q_off[b]:q_off[b + 1]] = rigid_map(shapes["Xw"][q_off[b]:q_off[b + 1]], Y["x0"][b], Y["B"][b])
    return x, Xw


def assemble_stokeslet(x: np.ndarray, Xw: np.ndarray, nn: np.ndarray, eps: float, mu: float,
                       n: Optional[int] = None) -> np.ndarray:
    """A_s of eq. nnrsbie (Sec. 3) in the top-left 3N x 3N corner of an
    n x n column-major (Fortran-order) array."""
    N = len(x)
    n = 3 * N if n is None else n
    A = np.zeros((n, n), order="F")
    _load().or_assemble_stokeslet(N, _d(np.ascontiguousarray(x)), len(Xw),
                                  _d(np.ascontiguousarray(Xw)), _i32(np.ascontiguousarray(nn, dtype=np.int32)),
                                  float(eps), float(mu), _d(A), n)
    return A


def assemble_rows(rows, x: np.ndarray, Xw: np.ndarray, nn: np.ndarray, eps: float,
                  mu: float) -> np.ndarray:
    """Rows 3m..3m+2 of A_s (Sec. 3, eq. nnrsbie) for the force points m in
    ``rows``, as a (3 len(rows), 3N) array: out[3r+j, 3n+k] = A[3m+j, 3n+k]
    with m = rows[r], the same sums as assemble_stokeslet."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    N = len(x)
    out = np.zeros((3 * len(rows), 3 * N), order="F")
    _load().or_assemble_rows(len(rows), _i64(rows), N, _d(np.ascontiguousarray(x)), len(Xw),
                             _d(np.ascontiguousarray(Xw)),
                             _i32(np.ascontiguousarray(nn, dtype=np.int32)), float(eps), float(mu),
                             _d(out), 3 * len(rows))
    return out


def velocity(xp: np.ndarray, Xw: np.ndarray, nn: np.ndarray, f: np.ndarray, eps: float,
             mu: float) -> np.ndarray:
    """Fluid velocity at field points xp (P x 4) induced by the force density
    f (N x 3 or 3N) through the NEAREST boundary integral (Sec. 3):
    u(x_p) = (1/8 pi mu) sum_q S^eps(x_p - X_q) w_q f_{n(q)}, summed in
    ascending q.  Returns P x 4 (u, 0)."""
    xp = np.ascontiguousarray(xp, dtype=np.float64).reshape(-1, 4)
    u = np.empty_like(xp)
    _load().or_velocity(len(xp), _d(xp), len(Xw), _d(np.ascontiguousarray(Xw)),
                        _i32(np.ascontiguousarray(nn, dtype=np.int32)),
                        _d(np.ascontiguousarray(f, dtype=np.float64).reshape(-1)),
                        float(eps), float(mu), _d(u))
    return u


def border(A: np.ndarray, x: np.ndarray, Xw: np.ndarray, nn: np.ndarray, n_off, q_off, kind,
           x0: np.ndarray) -> None:
    """Fill the rigid-body rows/columns of the swimming problem in place
    (Sec. 2 last paragraph and Sec. 4: unknown U, Omega; force and moment
    balance)."""
    _load().or_border(len(n_off) - 1, _i64(np.ascontiguousarray(n_off, dtype=np.int64)),
                      _i64(np.ascontiguousarray(q_off, dtype=np.int64)),
                      _i32(np.ascontiguousarray(kind, dtype=np.int32)),
                      _d(np.ascontiguousarray(x)), _d(np.ascontiguousarray(Xw)),
                      _i32(np.ascontiguousarray(nn, dtype=np.int32)),
                      _d(np.ascontiguousarray(x0, dtype=np.float64)), _d(A), A.shape[0])


def rhs(x: np.ndarray, shapes, table, Y, ext: Optional[np.ndarray] = None) -> np.ndarray:
    """Right-hand side: prescribed boundary velocity per force point, then
    the external force/moment on each free body (zero by default)."""
    kind = np.ascontiguousarray(table["kind"], dtype=np.int32)
    n_off = np.ascontiguousarray(shapes["n_off"], dtype=np.int64)
    N = int(n_off[-1])
    n = 3 * N + 6 * int((kind == FREE).sum())
    b = np.zeros(n)
    Bs = np.ascontiguousarray(Y["B"], dtype=np.float64)
    e = None if ext is None else _d(np.ascontiguousarray(ext, dtype=np.float64))
    _load().or_rhs(len(n_off) - 1, _i64(n_off), _i32(kind), _d(np.ascontiguousarray(x)),
                   _d(np.ascontiguousarray(Y["x0"], dtype=np.float64)), _d(Bs),
                   _d(np.ascontiguousarray(shapes["xidot"])),
                   _d(np.ascontiguousarray(table["U"], dtype=np.float64)),
                   _d(np.ascontiguousarray(table["Omega"], dtype=np.float64)), e, _d(b))
    return b


# --------------------------------------------------------------------------
# dense solve (Sec. 4 step 3)
# --------------------------------------------------------------------------

def lu(A: np.ndarray):
    """Partial-pivoting LU of a copy of A (Fortran order). Returns (LU, ipiv, info)."""
    LU = np.array(A, order="F", dtype=np.float64, copy=True)
    n = LU.shape[0]
    ipiv = np.empty(n, dtype=np.int32)
    info = _load().or_lu(n, _d(LU), n, _i32(ipiv))
    return LU, ipiv, int(info)


def lu_solve(LU: np.ndarray, ipiv: np.ndarray, b: np.ndarray, trans: bool = False) -> np.ndarray:
    x = np.array(b, dtype=np.float64, copy=True)
    _load().or_lu_solve(LU.shape[0], _d(LU), LU.shape[0], _i32(ipiv), _d(x), int(trans))
    return x


def residual_dd(A: np.ndarray, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """b - A x accumulated in double-double (TwoSum/TwoProduct)."""
    A = np.asfortranarray(A, dtype=np.float64)
    r = np.empty(A.shape[0])
    _load().or_residual_dd(A.shape[0], _d(A), A.shape[0], _d(np.ascontiguousarray(x)),
                           _d(np.ascontiguousarray(b)), _d(r))
    return r


def solve(A: np.ndarray, b: np.ndarray, maxit: int = 10, tol: float = 1e-16,
          return_info: bool = False):
    """x = A^{-1} b: partial-pivoting LU, then iterative refinement with a
    double-double residual until the correction is below tol * ||x||_inf."""
    A = np.asfortranarray(A, dtype=np.float64)
    LU, ipiv, info = lu(A)
    if info:
        raise np.linalg.LinAlgError(f"zero pivot at column {info}")
    b = np.asarray(b, dtype=np.float64)
    cols = b.reshape(len(b), -1)
    X = np.empty_like(cols)
    its = []
    for c in range(cols.shape[1]):
        bc = np.ascontiguousarray(cols[:, c])
        x = lu_solve(LU, ipiv, bc)
        its.append(int(_load().or_refine(A.shape[0], _d(A), A.shape[0], _d(LU), _i32(ipiv),
                                         _d(bc), _d(x), int(maxit), float(tol))))
        X[:, c] = x
    X = X.reshape(b.shape)
    if return_info:
        return X, {"refine_steps": its, "LU": LU, "ipiv": ipiv}
    return X


def solve_lapack(A: np.ndarray, b: np.ndarray, maxit: int = 30, tol: float = 1e-16,
                 return_info: bool = False):
    """x = A^{-1} b for systems too large for the unblocked LU above (the
    full-size swimming problems, n ~ 2.5e4): LAPACK's partial-pivoting LU
    (scipy getrf/getrs, a library step) gives the first solution and the
    corrections; the residual b - A x of every refinement step is the
    double-double one of nrs_oracle.c.  Stops when the correction is below
    tol * ||x||_inf, or when it no longer halves (the limit of the
    refinement: the corrections are then rounding noise of x).  This is the
    Sec. 4 step 3 solve carried to working accuracy; the refinement converges
    for kappa(A) u < 1."""
    import scipy.linalg as sla
    A = np.asfortranarray(A, dtype=np.float64)
    lu_piv = sla.lu_factor(A, overwrite_a=False, check_finite=False)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = sla.lu_solve(lu_piv, b, check_finite=False)
    steps, dprev = 0, np.inf
    for steps in range(1, maxit + 1):
        r = residual_dd(A, x, b)
        d = sla.lu_solve(lu_piv, r, check_finite=False)
        x = x + d
        dn, xn = np.max(np.abs(d)), np.max(np.abs(x))
        if dn <= tol * xn or dn >= 0.5 * dprev:
            break
        dprev = dn
    if return_info:
        return x, {"refine_steps": steps, "last_update": float(dn / xn)}
    return x


def cond1(A: np.ndarray, LU: Optional[np.ndarray] = None, ipiv: Optional[np.ndarray] = None) -> float:
    """Hager-Higham estimate of kappa_1(A)."""
    A = np.asfortranarray(A, dtype=np.float64)
    if LU is None:
        LU, ipiv, _ = lu(A)
    return float(_load().or_cond1(A.shape[0], _d(A), A.shape[0], _d(LU), _i32(ipiv)))


# --------------------------------------------------------------------------
# one evaluation of the swimming IVP right-hand side (Sec. 4)
# --------------------------------------------------------------------------

def system(problem, shapes, table, Y, nn: Optional[np.ndarray] = None,
           ext: Optional[np.ndarray] = None):
    """Build (A, b, nn, x_lab, Xw_lab) at one instant (Sec. 4 steps 1-2):
    lab-frame clouds from Y, nearest neighbours (in the body frame per body,
    or in the lab frame when problem.nn_global), A_s, rigid border, RHS."""
    x, Xw = lab_frame(shapes, Y)
    if nn is None:
        if problem.nn_global:
            nn = nearest(x, Xw, shapes["n_off"], shapes["q_off"], True)
        else:
            nn = nearest(shapes["x"], shapes["Xw"], shapes["n_off"], shapes["q_off"], False)
    N = len(x)
    n = 3 * N + 6 * int((table["kind"] == FREE).sum())
    A = assemble_stokeslet(x, Xw, nn, problem.eps, problem.mu, n)
    border(A, x, Xw, nn, shapes["n_off"], shapes["q_off"], table["kind"], Y["x0"])
    b = rhs(x, shapes, table, Y, ext)
    return A, b, nn, x, Xw


def split_solution(sol: np.ndarray, N: int):
    """(f (N,3), V (F,6) = [U, Omega] per free body)."""
    return sol[:3 * N].reshape(N, 3), sol[3 * N:].reshape(-1, 6)


def _cross_matrix(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def rates(problem, table, Y, V: np.ndarray):
    """dY/dt (Sec. 4): dX0/dt = U, dB/dt = [Omega]x B for free bodies (V from
    the solve) and for prescribed bodies (their given U, Omega); zero for
    static bodies."""
    dx0 = np.zeros_like(Y["x0"])
    dB = np.zeros_like(Y["B"])
    f = 0
    for b, kind in enumerate(table["kind"]):
        if kind == FREE:
            U, Om = V[f, :3], V[f, 3:]
            f += 1
        elif kind == PRESCRIBED:
            U, Om = table["U"][b], table["Omega"][b]
        else:
            continue
        dx0[b] = U
        dB[b] = _cross_matrix(Om) @ Y["B"][b]
    return dx0, dB


def mgs(B: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt on the columns 1, 2, 3 of a 3x3 matrix."""
    Q = np.array(B, dtype=np.float64, copy=True)
    for j in range(3):
        for i in range(j):
            Q[:, j] -= (Q[:, i] @ Q[:, j]) * Q[:, i]
        Q[:, j] /= math.sqrt(Q[:, j] @ Q[:, j])
    return Q


# Dormand & Prince (1980), the RK5(4)7M pair behind ode45 (Sec. 4 integrates
# the IVP with ode45): nodes, stage coefficients, fifth- and fourth-order weights
DP_C = [0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0]
DP_A = [[],
        [1 / 5],
        [3 / 40, 9 / 40],
        [44 / 45, -56 / 15, 32 / 9],
        [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
        [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
        [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84]]
DP_B5 = [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0]
DP_B4 = [5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40]


def _dp_state(Y, table):
    """The integrated components per non-static body: x0 (3) and B (9)."""
    return np.concatenate([Y["x0"], Y["B"].reshape(-1, 9)], axis=1)


def dp_step(problem, Y, t: float, h: float, rtol: float, atol: float, K0=None, solver=None):
    """One trial step of the Dormand-Prince pair for dY/dt = F(Y, t): the
    stage states Y_i = Y + h sum_j a_ij K_j (B re-orthonormalised by modified
    Gram-Schmidt, as the RK2 step does), K_i = dY/dt from each stage's solve;
    Y_new = the seventh stage's state; the error norm
    max_c |h sum_j (b5_j - b4_j) K_j,c| / (atol + rtol max(|Y_c|, |Y_new,c|))
    over the components of the non-static bodies.
    Returns (Y_new, K (7 rates per body as (dx0, dB)), err)."""
    from synth.geometry import pack_shapes, body_table
    solver = solver or solve
    table = body_table(problem)
    N = problem.N
    K = []
    Ys = []
    for i in range(7):
        if i == 0:
            Yi = Y
        else:
            x0 = Y["x0"] + h * sum(DP_A[i][j] * K[j][0] for j in range(i))
            B = Y["B"] + h * sum(DP_A[i][j] * K[j][1] for j in range(i))
            Yi = {"x0": x0, "B": np.array([mgs(b) for b in B])}
            for b, kind in enumerate(table["kind"]):
                if kind == STATIC:
                    Yi["x0"][b] = Y["x0"][b]
                    Yi["B"][b] = Y["B"][b]
        Ys.append(Yi)
        if i == 0 and K0 is not None:
            K.append(K0)
            continue
        sh = pack_shapes(problem, t + DP_C[i] * h)
        A, b, *_ = system(problem, sh, table, Yi)
        sol = solver(A, b)
        _, V = split_solution(sol, N)
        K.append(rates(problem, table, Yi, V))
    Yn = Ys[6]
    e = [DP_B5[j] - DP_B4[j] for j in range(7)]
    E0 = h * sum(e[j] * K[j][0] for j in range(7))
    E1 = h * sum(e[j] * K[j][1] for j in range(7))
    E = np.concatenate([E0, E1.reshape(-1, 9)], axis=1)
    y0, y1 = _dp_state(Y, table), _dp_state(Yn, table)
    live = np.array([k != STATIC for k in table["kind"]])
    sc = atol + rtol * np.maximum(np.abs(y0), np.abs(y1))
    err = float(np.max(np.abs(E[live]) / sc[live])) if live.any() else 0.0
    return Yn, K, err


def dp_integrate(problem, Y, t0: float, t_end: float, h0: float, rtol: float, atol: float,
                 h_min: float = 1e-8, h_max: float = None, solver=None):
    """Adaptive integration with dp_step: a trial with err <= 1 is accepted
    (its last stage's rates start the next step), and every trial sets the
    next step to h min(5 (accepted) or 1 (rejected), max(0.2, 0.9 err^(-1/5))),
    within [h_min, h_max] and the interval.  Returns (Y, t, accepted, rejected)."""
    h_max = t_end - t0 if h_max is None else h_max
    t, h = t0, min(h0, h_max, t_end - t0)
    K0 = None
    acc = rej = 0
    while t < t_end * (1 - 1e-14):
        Yn, K, err = dp_step(problem, Y, t, h, rtol, atol, K0=K0, solver=solver)
        ok = np.isfinite(err) and err <= 1.0
        f = 0.9 * err ** -0.2 if err > 0 else 5.0
        f = min(5.0 if ok else 1.0, max(0.2, f))
        if ok:
            t, Y, K0 = t + h, Yn, K[6]
            acc += 1
        else:
            rej += 1
            if h <= h_min:
                raise RuntimeError("step rejected at the smallest step size")
        h = min(h_max, max(h_min, h * f), t_end - t)
    return Y, t, acc, rej


def rk2_step_tracers(problem, Y, tracers, t: float, dt: float, solver=None):
    """One explicit-midpoint step of the bodies (rk2_step) and of passive
    tracers carried by the flow, dx_p/dt = u(x_p) (the particle tracking of
    the paper's mouse-node and sperm examples): the tracers' stage velocities
    come from each stage's force density and geometry,
      x_half = x + dt/2 u(x; stage 1),  x_new = x + dt u(x_half; stage 2).
    Returns (Y_new, tracers_new (P x 4), stages)."""
    from synth.geometry import pack_shapes, body_table
    solver = solver or solve
    table = body_table(problem)
    st = pack_shapes(problem, t)
    sh = pack_shapes(problem, t + 0.5 * dt)
    N = problem.N
    xt = np.ascontiguousarray(tracers, dtype=np.float64).reshape(-1, 4)
    A, b, nn1, _, Xw1 = system(problem, st, table, Y)
    sol1 = solver(A, b)
    u1 = velocity(xt, Xw1, nn1, sol1[:3 * N], problem.eps, problem.mu)
    _, V1 = split_solution(sol1, N)
    d1 = rates(problem, table, Y, V1)
    Yh = {"x0": Y["x0"] + 0.5 * dt * d1[0],
          "B": np.array([mgs(B) for B in Y["B"] + 0.5 * dt * d1[1]])}
    xh = xt.copy()
    xh[:, :3] = xt[:, :3] + 0.5 * dt * u1[:, :3]
    A2, b2, nn2, _, Xw2 = system(problem, sh, table, Yh)
    sol2 = solver(A2, b2)
    u2 = velocity(xh, Xw2, nn2, sol2[:3 * N], problem.eps, problem.mu)
    _, V2 = split_solution(sol2, N)
    d2 = rates(problem, table, Yh, V2)
    Yn = {"x0": Y["x0"] + dt * d2[0],
          "B": np.array([mgs(B) for B in Y["B"] + dt * d2[1]])}
    xn = xt.copy()
    xn[:, :3] = xt[:, :3] + dt * u2[:, :3]
    return Yn, xn, {"sol1": sol1, "sol2": sol2, "u1": u1, "u2": u2}


def rk2_step(problem, Y, t: float, dt: float, shapes_t=None, shapes_half=None,
             solver=None, return_stages: bool = False):
    """One explicit-midpoint step of dY/dt = F(Y, t) (the IVP of Sec. 4,
    stepped with RK2 instead of ode45):
      k1 = F(Y, t); Y_half = Y + dt/2 k1 (B re-orthonormalised);
      k2 = F(Y_half, t + dt/2); Y_new = Y + dt k2 (B re-orthonormalised).
    ``solver(A, b)`` defaults to the refined LU solve."""
    from synth.geometry import pack_shapes, body_table
    solver = solver or solve
    table = body_table(problem)
    st = shapes_t if shapes_t is not None else pack_shapes(problem, t)
    sh = shapes_half if shapes_half is not None else pack_shapes(problem, t + 0.5 * dt)
    N = problem.N
    A, b, *_ = system(problem, st, table, Y)
    sol1 = solver(A, b)
    _, V1 = split_solution(sol1, N)
    d1 = rates(problem, table, Y, V1)
    Yh = {"x0": Y["x0"] + 0.5 * dt * d1[0],
          "B": np.array([mgs(B) for B in Y["B"] + 0.5 * dt * d1[1]])}
    A2, b2, *_ = system(problem, sh, table, Yh)
    sol2 = solver(A2, b2)
    _, V2 = split_solution(sol2, N)
    d2 = rates(problem, table, Yh, V2)
    Yn = {"x0": Y["x0"] + dt * d2[0],
          "B": np.array([mgs(B) for B in Y["B"] + dt * d2[1]])}
    if return_stages:
        return Yn, {"sol1": sol1, "sol2": sol2, "Y_half": Yh}
    return Yn


def resistance_matrix(problem, shapes=None):
    """6x6 resistance matrix of a single rigid body (Sec. 3 sphere example):
    column c holds [total force; total moment about x0] exerted on the
    fluid for unit translation (c<3) or rotation (c>=3) along axis c%3."""
    from synth.geometry import pack_shapes, body_table, initial_state
    shapes = shapes if shapes is not None else pack_shapes(problem, 0.0)
    Y = initial_state(problem)
    table = body_table(problem)
    table["kind"] = np.array([PRESCRIBED], dtype=np.int32)
    x, Xw = lab_frame(shapes, Y)
    nn = nearest(shapes["x"], shapes["Xw"], shapes["n_off"], shapes["q_off"])
    A = assemble_stokeslet(x, Xw, nn, problem.eps, problem.mu)
    N = len(x)
    B6 = np.zeros((3 * N, 6))
    for c in range(6):
        tb = dict(table)
        tb["U"] = np.zeros((1, 3))
        tb["Omega"] = np.zeros((1, 3))
        if c < 3:
            tb["U"][0, c] = 1.0
        else:
            tb["Omega"][0, c - 3] = 1.0
        B6[:, c] = rhs(x, shapes, tb, Y)
    F = solve(A, B6)
    W = np.zeros(N)
    R = np.zeros((N, 3))
    np.add.at(W, nn, Xw[:, 3])
    np.add.at(R, nn, Xw[:, 3:4] * (Xw[:, :3] - Y["x0"][0]))
    Rm = np.zeros((6, 6))
    for c in range(6):
        f = F[:, c].reshape(N, 3)
        Rm[:3, c] = (W[:, None] * f).sum(axis=0)
        Rm[3:, c] = np.cross(R, f).sum(axis=0)
    return Rm

"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, the PDE the regularized stokeslet solves, a special case that reduces
to another method, brute force on tiny inputs, exact rational arithmetic, a
library routine, or a number the paper prints.  A plausible mistake in the
oracle (a dropped term, a wrong sign, a transposed block, a wrong tie rule)
fails at least one of them.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from synth import geometry as g

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# the regularized stokeslet (Sec. 3)
# --------------------------------------------------------------------------

def test_stokeslet_at_origin_is_two_over_eps():
    # S^eps(0) = delta_jk (2 eps^2) / eps^3 = (2/eps) I
    for eps in (0.5, 0.01, 0.005):
        S = O.stokeslet([0.0, 0.0, 0.0], eps)
        assert np.allclose(S, (2.0 / eps) * np.eye(3), rtol=1e-15, atol=0)


def test_oseen_closed_form_on_axis():
    # singular stokeslet at r = (a,0,0): diag(2/a, 1/a, 1/a)
    S = O.oseen([2.0, 0.0, 0.0])
    assert np.allclose(S, np.diag([1.0, 0.5, 0.5]), rtol=1e-15, atol=0)


def test_stokeslet_tends_to_oseen_far_from_the_blob():
    rng = np.random.default_rng(0)
    for _ in range(20):
        r = rng.normal(size=3)
        r *= rng.uniform(0.5, 2.0) / np.linalg.norm(r)
        S_eps = O.stokeslet(r, 1e-6)
        S = O.oseen(r)
        # S^eps - S = O(eps^2 / |r|^3)
        assert np.abs(S_eps - S).max() <= 1e-10 * np.abs(S).max()


def _fd_grad(f, x, h):
    """4th-order central differences of a vector/tensor field f at x."""
    out = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        out.append((-f(x + 2 * e) + 8 * f(x + e) - 8 * f(x - e) + f(x - 2 * e)) / (12 * h))
    return np.array(out)


def test_stokeslet_is_divergence_free():
    # each column S_{.k} is an incompressible velocity field: sum_j d_j S_jk = 0
    eps, h = 0.3, 1e-3
    for x in ([0.2, -0.1, 0.4], [0.05, 0.0, 0.02], [1.0, 0.7, -0.3]):
        x = np.array(x)
        grad = _fd_grad(lambda y: O.stokeslet(y, eps), x, h)  # grad[d, j, k] = d_d S_jk
        div = np.einsum("jjk->k", grad)
        assert np.abs(div).max() <= 1e-8 * np.abs(O.stokeslet(x, eps)).max() / eps


def test_stokeslet_solves_the_blob_forced_stokes_equations():
    # mu lap(u) - grad(p) + phi_eps e_k = 0 with u_j = S_jk / (8 pi mu) and
    # p = P_k / (8 pi)  (Sec. 3, regularized Stokes equations with the blob)
    eps, mu, h = 0.4, 1.7, 2e-3
    for x in ([0.15, -0.2, 0.3], [0.0, 0.1, -0.05], [0.6, 0.2, 0.1]):
        x = np.array(x)
        for k in range(3):
            def u(y):
                return O.stokeslet(y, eps)[:, k] / (8 * math.pi * mu)

            def p(y):
                return O.pressure(y, eps)[k] / (8 * math.pi)
            lap = np.zeros(3)
            for d in range(3):
                e = np.zeros(3)
                e[d] = h
                lap += (-u(x + 2 * e) + 16 * u(x + e) - 30 * u(x) + 16 * u(x - e) - u(x - 2 * e)) / (12 * h * h)
            gp = _fd_grad(lambda y: np.array([p(y)]), x, h)[:, 0]
            force = np.zeros(3)
            force[k] = O.blob(x, eps)
            res = mu * lap - gp + force
            scale = max(abs(mu * lap).max(), abs(gp).max(), force.max())
            assert np.abs(res).max() <= 1e-7 * scale, (x, k, res)


def test_blob_integrates_to_one():
    from scipy.integrate import quad
    for eps in (0.02, 0.01):
        val, _ = quad(lambda r: 4 * math.pi * r * r * O.blob([r, 0.0, 0.0], eps), 0, np.inf,
                      limit=400, epsabs=1e-13, epsrel=1e-12)
        assert abs(val - 1.0) < 1e-9


# --------------------------------------------------------------------------
# nearest neighbours, segments, assembly (Sec. 3)
# --------------------------------------------------------------------------

def _brute_nn(x, X, n_off, q_off):
    nn = np.empty(len(X), dtype=np.int32)
    for b in range(len(n_off) - 1):
        for q in range(q_off[b], q_off[b + 1]):
            best, arg = math.inf, -1
            for n in range(n_off[b], n_off[b + 1]):
                d = [x[n][i] - X[q][i] for i in range(3)]
                d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
                if d2 < best:
                    best, arg = d2, n
            nn[q] = arg
    return nn


def test_nearest_matches_brute_force_and_respects_bodies():
    rng = np.random.default_rng(1)
    n_off = np.array([0, 5, 12], dtype=np.int64)
    q_off = np.array([0, 40, 100], dtype=np.int64)
    x = np.zeros((12, 4))
    X = np.zeros((100, 4))
    x[:, :3] = rng.normal(size=(12, 3))
    X[:, :3] = rng.normal(size=(100, 3))
    X[:, 3] = 1.0
    nn = O.nearest(x, X, n_off, q_off)
    assert np.array_equal(nn, _brute_nn(x, X, n_off, q_off))
    assert np.all(nn[:40] < 5) and np.all(nn[40:] >= 5)
    # global search may cross bodies
    nng = O.nearest(x, X, n_off, q_off, global_=True)
    d = ((X[:, None, :3] - x[None, :, :3]) ** 2).sum(-1)
    assert np.array_equal(nng, np.argmin(d, axis=1))


def test_nearest_exact_ties_go_to_lowest_index():
    # quadrature point equidistant (bit-exactly, by mirror symmetry) from 3 force points
    x = np.array([[0.0, 1.0, 0.0, 0], [1.0, 0.0, 0.0, 0], [0.0, -1.0, 0.0, 0],
                  [-1.0, 0.0, 0.0, 0]], dtype=np.float64)
    X = np.array([[0.0, 0.0, 0.0, 1.0], [0.5, 0.5, 0.0, 1.0], [-0.25, 0.0, 0.0, 1.0]])
    nn = O.nearest(x, X, np.array([0, 4]), np.array([0, 3]))
    assert list(nn) == [0, 0, 3]
    # reversing the order of the force points moves the winner with the index
    nn = O.nearest(x[::-1].copy(), X, np.array([0, 4]), np.array([0, 3]))
    assert list(nn) == [0, 2, 0]


def test_nearest_on_nested_cube_sphere_is_exact_on_coincident_points():
    xi, _ = g.cube_sphere_vertices(4)
    Xi, w = g.cube_sphere_vertices(16)
    x = np.concatenate([xi, np.zeros((len(xi), 1))], axis=1)
    X = np.concatenate([Xi, w[:, None]], axis=1)
    nn = O.nearest(x, X, np.array([0, len(x)]), np.array([0, len(X)]))
    # every force point is also a quadrature point, at distance exactly 0
    for m in range(len(xi)):
        hits = np.nonzero(np.all(Xi == xi[m], axis=1))[0]
        assert len(hits) == 1 and nn[hits[0]] == m
    assert np.array_equal(nn, _brute_nn(x, X, [0, len(x)], [0, len(X)]))


def test_segments_are_a_stable_counting_sort():
    rng = np.random.default_rng(2)
    nn = rng.integers(0, 17, size=300).astype(np.int32)
    nn[nn == 5] = 6  # an empty segment
    seg_ptr, perm = O.segments(nn, 17)
    assert np.array_equal(perm, np.argsort(nn, kind="stable"))
    assert np.array_equal(np.diff(seg_ptr), np.bincount(nn, minlength=17))
    assert seg_ptr[0] == 0 and seg_ptr[-1] == 300


def test_nystrom_special_case():
    # X = x and w = 1 make nu the identity, and the NEAREST matrix reduces to
    # the Nystrom matrix S^eps(x_m, x_n) / (8 pi mu)  (Sec. 3)
    rng = np.random.default_rng(3)
    N, eps, mu = 7, 0.1, 1.3
    x = np.zeros((N, 4))
    x[:, :3] = rng.normal(size=(N, 3))
    Xw = x.copy()
    Xw[:, 3] = 1.0
    nn = O.nearest(x, Xw, np.array([0, N]), np.array([0, N]))
    assert np.array_equal(nn, np.arange(N))
    A = O.assemble_stokeslet(x, Xw, nn, eps, mu)
    for m in range(N):
        for n in range(N):
            blk = A[3 * m:3 * m + 3, 3 * n:3 * n + 3]
            ref = O.stokeslet(x[m, :3] - x[n, :3], eps) / (8 * math.pi * mu)
            assert np.allclose(blk, ref, rtol=1e-15, atol=0)


def test_assembly_equals_dense_times_sparse_product():
    # Sec. 3: A_s = (3N x 3Q stokeslet matrix with weights) x (3Q x 3N nu)
    rng = np.random.default_rng(4)
    N, Q, eps, mu = 4, 12, 0.2, 0.7
    x = np.zeros((N, 4))
    x[:, :3] = rng.normal(size=(N, 3))
    Xw = np.zeros((Q, 4))
    Xw[:, :3] = rng.normal(size=(Q, 3))
    Xw[:, 3] = rng.uniform(0.1, 1.0, size=Q)
    nn = O.nearest(x, Xw, np.array([0, N]), np.array([0, Q]))
    A = O.assemble_stokeslet(x, Xw, nn, eps, mu)
    Sbig = np.zeros((3 * N, 3 * Q))
    for m in range(N):
        for q in range(Q):
            Sbig[3 * m:3 * m + 3, 3 * q:3 * q + 3] = O.stokeslet(x[m, :3] - Xw[q, :3], eps) * Xw[q, 3]
    nu = np.zeros((Q, N))
    nu[np.arange(Q), nn] = 1.0
    ref = Sbig @ np.kron(nu, np.eye(3)) / (8 * math.pi * mu)
    assert np.allclose(A, ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())
    # not symmetric in general: the NEAREST matrix is not a Nystrom matrix
    assert np.abs(A - A.T).max() > 1e-6 * np.abs(A).max()


# --------------------------------------------------------------------------
# dense solve (Sec. 4 step 3)
# --------------------------------------------------------------------------

def _frac_solve(A, b):
    n = len(b)
    M = [[Fraction(A[i][j]) for j in range(n)] + [Fraction(b[i])] for i in range(n)]
    for k in range(n):
        p = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[p] = M[p], M[k]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k] / M[k][k]
                M[i] = [a - f * c for a, c in zip(M[i], M[k])]
    return [M[i][n] / M[i][i] for i in range(n)]


def test_solve_matches_exact_rationals_on_ill_conditioned_system():
    # Hilbert-like matrix (kappa ~ 1e10): LU alone loses digits; refinement
    # with the double-double residual recovers the correctly rounded answer
    n = 8
    A = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
    b = np.arange(1.0, n + 1)
    x = O.solve(A, b)
    exact = _frac_solve(A.tolist(), b.tolist())
    err = max(abs(Fraction(float(x[i])) - exact[i]) / abs(exact[i]) for i in range(n))
    assert err < 1e-12


def test_lapack_refined_solve_matches_exact_rationals():
    # the large-system solve (LAPACK LU + double-double refinement) on a
    # Hilbert matrix of kappa ~ 1e13, the conditioning of the four-swimmer
    # system: the LU solve alone keeps about 3 digits, the refinement brings
    # every component to working accuracy
    n = 10
    A = np.array([[1.0 / (i + j + 1) for j in range(n)] for i in range(n)])
    b = np.arange(1.0, n + 1)
    x, info = O.solve_lapack(A, b, return_info=True)
    exact = _frac_solve(A.tolist(), b.tolist())
    err = max(abs(Fraction(float(x[i])) - exact[i]) / abs(exact[i]) for i in range(n))
    assert err < 1e-13, err
    assert info["refine_steps"] >= 2


def test_lapack_refined_solve_agrees_with_the_plain_lu_solve_on_a_swimmer():
    # two independently factored solves refined to working accuracy agree to
    # working accuracy (the small swimmer, n = 246)
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    sh = g.pack_shapes(pr, 0.2)
    A, b, *_ = O.system(pr, sh, g.body_table(pr), g.initial_state(pr))
    x1 = O.solve(A, b)
    x2 = O.solve_lapack(A, b)
    assert np.linalg.norm(x1 - x2) <= 1e-14 * np.linalg.norm(x1)


def test_assembled_row_subset_equals_the_whole_matrix_rows():
    # the sampled rows of A_s used at full size are the whole matrix's rows,
    # bit for bit (same sums in the same order)
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    sh = g.pack_shapes(pr, 0.1)
    Y = g.initial_state(pr)
    x, Xw = O.lab_frame(sh, Y)
    nn = O.nearest(sh["x"], sh["Xw"], sh["n_off"], sh["q_off"])
    A = O.assemble_stokeslet(x, Xw, nn, pr.eps, pr.mu)
    rows = np.array([0, 17, 5, pr.N - 1])
    sub = O.assemble_rows(rows, x, Xw, nn, pr.eps, pr.mu)
    for r, m in enumerate(rows):
        assert np.array_equal(sub[3 * r:3 * r + 3], A[3 * m:3 * m + 3])


def test_residual_dd_is_exact_to_rounding():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(6, 6))
    x = rng.normal(size=6)
    b = A @ x + 1e-12 * rng.normal(size=6)
    r = O.residual_dd(A, x, b)
    for i in range(6):
        exact = Fraction(b[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(6))
        assert abs(Fraction(r[i]) - exact) <= abs(exact) * Fraction(1, 2 ** 50) + Fraction(1, 2 ** 1074)


def test_lu_reconstructs_and_matches_lapack():
    import scipy.linalg as sla
    rng = np.random.default_rng(6)
    n = 200
    A = rng.normal(size=(n, n))
    LU, ipiv, info = O.lu(A)
    assert info == 0
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for k in range(n):
        PA[[k, ipiv[k]]] = PA[[ipiv[k], k]]
    assert np.abs(L @ U - PA).max() <= 1e-13 * np.abs(A).max()
    lu_ref, piv_ref = sla.lu_factor(A)
    assert np.array_equal(ipiv, piv_ref)  # same pivot rule as LAPACK on generic data
    b = rng.normal(size=n)
    assert np.allclose(O.solve(A, b), np.linalg.solve(A, b), rtol=1e-11, atol=1e-13)
    assert np.allclose(O.lu_solve(LU, ipiv, b, trans=True), np.linalg.solve(A.T, b), rtol=1e-10)


def test_lu_reports_first_zero_pivot():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 1.0, 1.0]])
    _, _, info = O.lu(A)
    assert info == 3


def test_condition_estimate_matches_exact_one_norm_condition():
    rng = np.random.default_rng(7)
    for n in (5, 30, 80):
        A = rng.normal(size=(n, n)) @ np.diag(np.logspace(0, 4, n))
        est = O.cond1(A)
        exact = np.linalg.cond(A, 1)
        assert 0.3 * exact <= est <= exact * (1 + 1e-10)


# --------------------------------------------------------------------------
# the full method: resistance and swimming problems (Sec. 3, Sec. 4)
# --------------------------------------------------------------------------

def test_sphere_resistance_within_two_percent_at_the_papers_sizes():
    spec = json.load(open(os.path.join(GOLDEN, "sphere_resistance.json")))
    pr = g.sphere_cells_config(12, 24, eps=spec["eps"])
    assert pr.N == spec["N"] and pr.Q == spec["Q"]
    R = O.resistance_matrix(pr)
    a, mu = 1.0, 1.0
    drag, torque = 6 * math.pi * mu * a, 8 * math.pi * mu * a ** 3
    for c in range(3):
        assert abs(R[c, c] / drag - 1) <= spec["max_rel_error"]
        assert abs(R[3 + c, 3 + c] / torque - 1) <= spec["max_rel_error"]
    # no translation-rotation coupling for a sphere; R symmetric
    assert np.abs(R[:3, 3:]).max() <= 1e-9 * drag
    assert np.abs(R - R.T).max() <= 1e-9 * drag


def test_sphere_resistance_at_cube_sphere_vertex_sizes():
    # 98 force / 1538 quadrature points: coarser traction grid, larger error
    pr = g.sphere_config()
    R = O.resistance_matrix(pr)
    assert abs(R[0, 0] / (6 * math.pi) - 1) < 0.10
    assert abs(R[3, 3] / (8 * math.pi) - 1) < 0.15
    assert np.abs(R - R.T).max() <= 1e-9 * R[0, 0]


def _small_swimmer():
    return g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)


def _solve_with(pr, shapes, Y, ext=None):
    table = g.body_table(pr)
    A, b, nn, x, Xw = O.system(pr, shapes, table, Y, ext=ext)
    sol = O.solve(A, b)
    f, V = O.split_solution(sol, pr.N)
    return f, V, A, b, nn, x, Xw


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_rigid_translation_of_the_shape_is_cancelled_by_U():
    # a "deformation" that is a uniform translation V leaves the body at rest
    # in the fluid: f = 0, U = -B V, Omega = 0
    pr = _small_swimmer()
    sh = g.pack_shapes(pr, 0.0)
    V = np.array([0.3, -0.2, 0.5])
    sh["xidot"][:, :3] = V
    Y = {"x0": np.array([[0.1, 0.2, 0.3]]), "B": _rot([1, 2, 3], 0.7)[None]}
    f, Vs, *_ = _solve_with(pr, sh, Y)
    assert np.abs(f).max() < 1e-10
    assert np.allclose(Vs[0, :3], -Y["B"][0] @ V, atol=1e-12)
    assert np.allclose(Vs[0, 3:], 0.0, atol=1e-12)


def test_rigid_rotation_of_the_shape_is_cancelled_by_Omega():
    # deformation xidot = w x xi (about the body origin x0): f = 0, U = 0,
    # Omega = -B w; fixes the sign and orientation of the [r]x border columns
    pr = _small_swimmer()
    sh = g.pack_shapes(pr, 0.0)
    w = np.array([0.4, -1.1, 0.7])
    sh["xidot"][:, :3] = np.cross(w, sh["x"][:, :3])
    Y = {"x0": np.array([[-0.3, 0.2, 1.0]]), "B": _rot([0, 1, 1], -0.4)[None]}
    f, Vs, *_ = _solve_with(pr, sh, Y)
    assert np.abs(f).max() < 1e-9
    assert np.allclose(Vs[0, :3], 0.0, atol=1e-11)
    assert np.allclose(Vs[0, 3:], -Y["B"][0] @ w, atol=1e-11)


def test_mobility_recovers_the_resistance_problem():
    # a rigid body pushed by the force/moment that the resistance problem
    # needs for (U, Omega) moves with exactly (U, Omega)
    pr = _small_swimmer()
    sh = g.pack_shapes(pr, 0.0)
    sh["xidot"][:] = 0.0
    Y = g.initial_state(pr)
    U, Om = np.array([0.2, 0.1, -0.3]), np.array([0.5, -0.2, 0.3])
    table = g.body_table(pr)
    x, Xw = O.lab_frame(sh, Y)
    nn = O.nearest(sh["x"], sh["Xw"], sh["n_off"], sh["q_off"])
    A = O.assemble_stokeslet(x, Xw, nn, pr.eps, pr.mu)
    rhs = (U[None] + np.cross(Om[None], x[:, :3] - Y["x0"][0])).ravel()
    fr = O.solve(A, rhs).reshape(-1, 3)
    W = np.zeros(pr.N)
    R = np.zeros((pr.N, 3))
    np.add.at(W, nn, Xw[:, 3])
    np.add.at(R, nn, Xw[:, 3:4] * (Xw[:, :3] - Y["x0"][0]))
    F = (W[:, None] * fr).sum(0)
    M = np.cross(R, fr).sum(0)
    f, Vs, *_ = _solve_with(pr, sh, Y, ext=np.concatenate([F, M])[None])
    assert np.allclose(Vs[0, :3], U, rtol=1e-9, atol=1e-11)
    assert np.allclose(Vs[0, 3:], Om, rtol=1e-9, atol=1e-11)
    assert np.allclose(f, fr, rtol=1e-8, atol=1e-10 * np.abs(fr).max())


def test_swimming_solution_balances_force_and_moment_and_is_equivariant():
    pr = _small_swimmer()
    sh = g.pack_shapes(pr, 0.13)
    Y = g.initial_state(pr)
    f, V, A, b, nn, x, Xw = _solve_with(pr, sh, Y)
    W = np.zeros(pr.N)
    R = np.zeros((pr.N, 3))
    np.add.at(W, nn, Xw[:, 3])
    np.add.at(R, nn, Xw[:, 3:4] * (Xw[:, :3] - Y["x0"][0]))
    scale = np.abs(W[:, None] * f).sum()
    assert np.abs((W[:, None] * f).sum(0)).max() <= 1e-13 * scale
    assert np.abs(np.cross(R, f).sum(0)).max() <= 1e-13 * scale
    # rotate and translate the whole body: forces and velocities rotate with it
    Rm = _rot([0.3, -1.0, 0.5], 1.1)
    Y2 = {"x0": np.array([[1.0, -2.0, 0.5]]), "B": Rm[None]}
    f2, V2, *_ = _solve_with(pr, sh, Y2)
    assert np.allclose(f2, f @ Rm.T, rtol=1e-9, atol=1e-10 * np.abs(f).max())
    assert np.allclose(V2[0, :3], Rm @ V[0, :3], rtol=1e-9, atol=1e-12)
    assert np.allclose(V2[0, 3:], Rm @ V[0, 3:], rtol=1e-9, atol=1e-12)


def test_undulating_tube_swims_against_its_wave():
    # the wave y = a s sin(2 pi (s - t)) travels towards +x (s = 2x), so the
    # body swims towards -x; by the planar symmetry U_z = Omega_x = Omega_y = 0
    pr = _small_swimmer()
    sh = g.pack_shapes(pr, 0.0)
    _, V, *_ = _solve_with(pr, sh, g.initial_state(pr))
    U, Om = V[0, :3], V[0, 3:]
    assert U[0] < 0
    assert abs(U[2]) < 1e-12 and abs(Om[0]) < 1e-12 and abs(Om[1]) < 1e-12


def test_rk2_is_second_order_for_a_prescribed_rotation():
    # prescribed rigid rotation: exact B(t) = exp(t [Omega]x) B0
    pr = g.sphere_config(n_force=2, n_quad=4, U=(0.0, 0.0, 0.0), Omega=(0.3, -0.5, 0.9))
    Om = pr.bodies[0].Omega
    T = 0.4
    errs = []
    for steps in (4, 8, 16):
        Y = g.initial_state(pr)
        dt = T / steps
        for s in range(steps):
            Y = O.rk2_step(pr, Y, s * dt, dt)
        exact = _rot(Om, np.linalg.norm(Om) * T)
        errs.append(np.abs(Y["B"][0] - exact).max())
        assert np.allclose(Y["B"][0].T @ Y["B"][0], np.eye(3), atol=1e-14)
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_rk2_translates_a_prescribed_body_exactly():
    pr = g.sphere_config(n_force=2, n_quad=4, U=(0.5, -1.0, 2.0), Omega=(0.0, 0.0, 0.0))
    Y = g.initial_state(pr)
    for s in range(5):
        Y = O.rk2_step(pr, Y, s * 0.1, 0.1)
    assert np.allclose(Y["x0"][0], 0.5 * np.array([0.5, -1.0, 2.0]), rtol=1e-15, atol=1e-15)


# --------------------------------------------------------------------------
# velocity at field points and passive tracers (particle tracking)
# --------------------------------------------------------------------------

def test_velocity_far_from_a_point_force_is_the_oseen_flow():
    # one quadrature point of weight w at X carrying the force density f:
    # u(x) = w S^eps(x - X) f / (8 pi mu) -> w (f/r + (f.r) r/r^3) / (8 pi mu)
    # for r >> eps (Sec. 3: the blob solution tends to the stokeslet)
    X = np.array([[0.3, -0.2, 0.1, 0.7]])
    f = np.array([0.4, -1.3, 2.2])
    eps, mu = 1e-3, 1.7
    rng = np.random.default_rng(11)
    xp = np.zeros((6, 4))
    d = rng.normal(size=(6, 3))
    xp[:, :3] = X[0, :3] + 10.0 * d / np.linalg.norm(d, axis=1, keepdims=True)
    u = O.velocity(xp, X, np.array([0], dtype=np.int32), f, eps, mu)
    for p in range(6):
        r = xp[p, :3] - X[0, :3]
        rn = np.linalg.norm(r)
        ref = X[0, 3] * (f / rn + (f @ r) * r / rn ** 3) / (8 * math.pi * mu)
        # the regularisation changes the flow by O(eps^2 / r^2) = 1e-8 of its size
        assert np.linalg.norm(u[p, :3] - ref) <= 1e-7 * np.linalg.norm(ref)
        assert u[p, 3] == 0.0


def test_velocity_at_collocation_points_is_the_assembled_operator():
    # at the force points the boundary integral is the assembled A_s: u(x_m) = (A_s f)_m
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    sh = g.pack_shapes(pr, 0.15)
    Y = g.initial_state(pr)
    x, Xw = O.lab_frame(sh, Y)
    nn = O.nearest(sh["x"], sh["Xw"], sh["n_off"], sh["q_off"])
    A = O.assemble_stokeslet(x, Xw, nn, pr.eps, pr.mu)
    f = np.random.default_rng(12).normal(size=3 * pr.N)
    u = O.velocity(x, Xw, nn, f, pr.eps, pr.mu)
    ref = (A @ f).reshape(-1, 3)
    assert np.allclose(u[:, :3], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_velocity_around_a_translating_sphere_is_the_stokes_flow():
    # the paper's sphere (N = 864, Q = 3456, eps = 0.01) translating with U:
    # off the sphere the computed flow is the exact Stokes solution
    #   u = 3a/4 (U/r + (U.x) x / r^3) + a^3/4 (U/r^3 - 3 (U.x) x / r^5)
    # to the discretisation's accuracy (the drag is within 2 %)
    pr = g.sphere_cells_config(12, 24, eps=0.01, U=(1.0, 0.0, 0.0))
    sh = g.pack_shapes(pr, 0.0)
    Y = g.initial_state(pr)
    A, b, nn, x, Xw = O.system(pr, sh, g.body_table(pr), Y)
    sol = O.solve_lapack(A, b)
    U = np.array([1.0, 0.0, 0.0])
    rng = np.random.default_rng(13)
    d = rng.normal(size=(12, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    xp = np.zeros((24, 4))
    xp[:12, :3] = 1.5 * d
    xp[12:, :3] = 3.0 * d
    u = O.velocity(xp, Xw, nn, sol[:3 * pr.N], pr.eps, pr.mu)
    for p in range(24):
        xv = xp[p, :3]
        r = np.linalg.norm(xv)
        ref = 0.75 * (U / r + (U @ xv) * xv / r ** 3) + 0.25 * (U / r ** 3 - 3 * (U @ xv) * xv / r ** 5)
        assert np.linalg.norm(u[p, :3] - ref) <= 0.02 * np.linalg.norm(U), (p, u[p], ref)


def test_tracer_on_a_translating_body_is_carried_with_it():
    # a tracer at a force point of a rigidly translating body sees the body's
    # velocity at both stages (the collocation condition), so one step moves
    # it by dt U, like the body
    U = np.array([0.5, -1.0, 2.0])
    pr = g.sphere_config(U=tuple(U))
    Y = g.initial_state(pr)
    sh = g.pack_shapes(pr, 0.0)
    tr = np.array(sh["x"][[0, 7, 40]], dtype=np.float64)
    Yn, trn, st = O.rk2_step_tracers(pr, Y, tr, 0.0, 0.1, solver=O.solve_lapack)
    assert np.allclose(st["u1"][:, :3], U, rtol=0, atol=1e-11)
    assert np.allclose(trn[:, :3], tr[:, :3] + 0.1 * U, rtol=0, atol=1e-12)
    assert np.allclose(Yn["x0"][0], 0.1 * U, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# adaptive Dormand-Prince stepping (the ode45 of Sec. 4)
# --------------------------------------------------------------------------

def _rot(axis_rate, angle):
    k = np.asarray(axis_rate, float) / np.linalg.norm(axis_rate)
    Kx = np.array([[0.0, -k[2], k[1]], [k[2], 0.0, -k[0]], [-k[1], k[0], 0.0]])
    return np.eye(3) + math.sin(angle) * Kx + (1 - math.cos(angle)) * (Kx @ Kx)


def test_dormand_prince_is_fifth_order_for_a_prescribed_rotation():
    # fixed steps (tolerance never binding): the global error of B(T) against
    # the exact rotation falls by at least 2^5 per halving of the step (for
    # this linear problem it falls a little faster, ~2^5.8); a wrong
    # coefficient of the tableau drops the order
    Om = np.array([0.3, -1.1, 2.0])
    pr = g.sphere_config(n_force=2, n_quad=4, U=(0.0, 0.0, 0.0), Omega=tuple(Om))
    T = 1.0
    errs = []
    for steps in (4, 8, 16):
        Y = g.initial_state(pr)
        h = T / steps
        K0 = None
        for s in range(steps):
            Y, K, _ = O.dp_step(pr, Y, s * h, h, 1.0, 1.0, K0=K0)
            K0 = K[6]
        errs.append(np.abs(Y["B"][0] - _rot(Om, np.linalg.norm(Om) * T)).max())
    assert errs[0] / errs[1] > 28.0 and errs[1] / errs[2] > 28.0, errs
    assert errs[2] < 1e-9


def test_dormand_prince_error_estimate_scales_as_h5_and_translation_is_exact():
    # the embedded estimate of one step shrinks at least as h^5; a prescribed
    # translation is integrated exactly (every stage has the same rate)
    Om = np.array([0.0, 0.0, 1.5])
    pr = g.sphere_config(n_force=2, n_quad=4, U=(0.4, 0.0, -0.2), Omega=tuple(Om))
    Y0 = g.initial_state(pr)
    e1 = O.dp_step(pr, Y0, 0.0, 0.2, 1e-10, 1e-10)[2]
    e2 = O.dp_step(pr, Y0, 0.0, 0.1, 1e-10, 1e-10)[2]
    assert e1 / e2 > 28.0, (e1, e2)
    Yn = O.dp_step(pr, Y0, 0.0, 0.3, 1.0, 1.0)[0]
    assert np.allclose(Yn["x0"][0], 0.3 * np.array([0.4, 0.0, -0.2]), rtol=0, atol=1e-15)


def test_adaptive_dormand_prince_meets_its_tolerance():
    # a fast rotation over one period: the controller adapts h (steps get
    # rejected from a too-large first step) and the end state is within a
    # small multiple of the tolerance of the exact rotation
    Om = np.array([1.0, 2.0, -2.0])
    pr = g.sphere_config(n_force=2, n_quad=4, U=(0.0, 0.0, 0.0), Omega=tuple(Om))
    T = 2 * math.pi / np.linalg.norm(Om)
    for tol in (1e-6, 1e-9):
        Y, t, acc, rej = O.dp_integrate(pr, g.initial_state(pr), 0.0, T, 1.0, tol, tol)
        assert abs(t - T) <= 1e-12
        err = np.abs(Y["B"][0] - np.eye(3)).max()
        assert err <= 50 * tol, (tol, err, acc, rej)
        assert rej >= 1

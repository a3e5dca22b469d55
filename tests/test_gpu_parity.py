"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (nearest neighbours, segments) must match bit for bit.  Floating
point: lab-frame clouds, right-hand side and the FP64 system matrix bit for
bit (the kernels round every operation on its own, in the oracle's order,
with correctly rounded square root and division); solutions to a relative
error of 1e-10 in the forces f and in the rigid velocities V, the accuracy
the mixed-precision refinement promises.
"""

import math

import numpy as np
import pytest
import torch

import oracle as O
from synth import geometry as g

pytestmark = pytest.mark.gpu

TOL_SOL = 1e-10


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _setup(N, pr, t=0.0, prec="fp32", **kw):
    sh = g.pack_shapes(pr, t)
    ctx = N.Context.from_problem(pr, factor_prec=prec, **kw)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = N.shapes_to_device(sh)
    return ctx, sh, Y, (xi, Xiw, xidot)


def _gpu_system(N, ctx, dev_shapes, nn_frame="body"):
    xi, Xiw, xidot = dev_shapes
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    if nn_frame == "body":
        nn, seg_ptr, perm = ctx.nearest_build(xi, Xiw)
    else:
        nn, seg_ptr, perm = ctx.nearest_build(x, Xw)
    At = ctx.assemble(x, Xw)
    return x, Xw, b, nn, seg_ptr, perm, At


def _oracle_system(pr, sh, Y, ext=None):
    return O.system(pr, sh, g.body_table(pr), Y, ext=ext)


PROBLEMS = {
    "sphere": lambda: g.sphere_config(),
    "swimmer_small": lambda: g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8),
    "swimmer": lambda: g.swimmer_config(),
    "sperm2": lambda: g.sperm_channel_config(count=2, n_head=40, q_head=400, n_flag=60, q_flag=600,
                                             wall_f=(20, 6, 3), wall_q=(60, 18, 9)),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_kinematics_nearest_segments_bit_exact(N, name):
    pr = PROBLEMS[name]()
    ctx, sh, Y, dev = _setup(N, pr, t=0.137)
    Y = {"x0": Y["x0"] + np.array([0.3, -0.1, 0.2]), "B": Y["B"]}
    Rm = np.array([[0.36, 0.48, -0.8], [-0.8, 0.6, 0.0], [0.48, 0.64, 0.6]])
    Y["B"] = np.array([Rm for _ in pr.bodies])
    ctx.set_state(Y["x0"], Y["B"])
    x, Xw, b, nn, seg_ptr, perm, At = _gpu_system(N, ctx, dev)
    A_or, b_or, nn_or, x_or, Xw_or = _oracle_system(pr, sh, Y)
    assert np.array_equal(x.cpu().numpy(), x_or)
    assert np.array_equal(Xw.cpu().numpy(), Xw_or)
    assert np.array_equal(b.cpu().numpy(), b_or)
    assert np.array_equal(nn.cpu().numpy(), nn_or)
    sp_or, perm_or = O.segments(nn_or, pr.N)
    assert np.array_equal(seg_ptr.cpu().numpy(), sp_or)
    assert np.array_equal(perm.cpu().numpy(), perm_or)
    A = At.T.cpu().numpy()
    assert np.array_equal(A, A_or), np.abs(A - A_or).max()


def test_nearest_global_mode_bit_exact(N):
    pr = PROBLEMS["sperm2"]()
    pr.nn_global = True
    ctx, sh, Y, dev = _setup(N, pr, t=0.3)
    x, Xw, b = ctx.kinematics(*dev)
    nn, seg_ptr, perm = ctx.nearest_build(x, Xw)
    x_or, Xw_or = O.lab_frame(sh, Y)
    nn_or = O.nearest(x_or, Xw_or, sh["n_off"], sh["q_off"], global_=True)
    assert np.array_equal(nn.cpu().numpy(), nn_or)


def test_nearest_ties_on_nested_cube_spheres(N):
    # the n=4 lattice is a subset of the n=16 lattice: exact ties by symmetry
    pr = g.sphere_config()
    ctx, sh, Y, dev = _setup(N, pr)
    nn, _, _ = ctx.nearest_build(dev[0], dev[1])
    nn_or = O.nearest(sh["x"], sh["Xw"], sh["n_off"], sh["q_off"])
    assert np.array_equal(nn.cpu().numpy(), nn_or)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "tf32"])
def test_sphere_resistance_solve(N, prec):
    pr = g.sphere_config()
    ctx, sh, Y, dev = _setup(N, pr, prec=prec)
    x, Xw, b, nn, seg_ptr, perm, At = _gpu_system(N, ctx, dev)
    assert ctx.factor(prec) == 0
    xg, rep = ctx.solve(b)
    A_or, b_or, *_ = _oracle_system(pr, sh, Y)
    f_or = O.solve(A_or, b_or)
    assert _rel(xg.cpu().numpy(), f_or) <= TOL_SOL, rep
    assert rep[0]["converged"] == 1 and rep[0]["backward_err"] < 1e-15


@pytest.mark.parametrize("name,prec", [("swimmer_small", "fp32"), ("swimmer", "fp32"),
                                       ("swimmer", "fp64"), ("swimmer", "tf32"), ("sperm2", "fp32"),
                                       ("sperm2", "tf32")])
def test_swimming_solve_matches_oracle(N, name, prec):
    pr = PROBLEMS[name]()
    ctx, sh, Y, dev = _setup(N, pr, t=0.25, prec=prec)
    x, Xw, b, nn, seg_ptr, perm, At = _gpu_system(N, ctx, dev)
    assert ctx.factor(prec) == 0
    xg, rep = ctx.solve(b)
    A_or, b_or, *_ = _oracle_system(pr, sh, Y)
    sol = O.solve(A_or, b_or)
    f, V = O.split_solution(sol, pr.N)
    fg, Vg = O.split_solution(xg.cpu().numpy(), pr.N)
    assert _rel(fg, f) <= TOL_SOL, (rep, _rel(fg, f))
    assert _rel(Vg, V) <= TOL_SOL, (rep, _rel(Vg, V))


@pytest.mark.parametrize("name,prec", [("swimmer", "fp32"), ("swimmer", "tf32"),
                                       ("sperm2", "tf32"), ("sphere", "tf32")])
def test_explicit_inverse_is_accurate(N, name, prec):
    # The FP32 inverse preconditions GMRES: with M ~ A^{-1} to FP32 accuracy,
    # M A = I + E with ||E|| ~ 1e-5, so each refinement step's GMRES meets its
    # 1e-4 tolerance in one or two iterations.  A wrong inverse (a misplaced
    # pivot, a transposed block) still converges -- GMRES is robust -- but
    # needs many more iterations, which this catches.
    pr = PROBLEMS[name]()
    ctx, sh, Y, dev = _setup(N, pr, t=0.25, prec=prec)
    _gpu_system(N, ctx, dev)
    b = ctx.kinematics(*dev)[2]
    assert ctx.factor(prec) == 0
    _, rep = ctx.solve(b)
    assert rep[0]["converged"] and rep[0]["outer"] <= 4, rep
    assert rep[0]["inner"] <= 2 * rep[0]["outer"], rep


@pytest.mark.parametrize("name", ["swimmer_small", "sperm2", "swimmer"])
def test_fused_factor_matches_streamed(N, name):
    # The one-launch factorisation (diagonal inverses on one CTA, updates on
    # the others, counters instead of stream events) runs the same arithmetic
    # in the same order as the separate kernels: the inverse, and so every
    # refinement iterate, is the same bit for bit.
    pr = PROBLEMS[name]()
    sols, reps = [], []
    for schedule in ("fused", "streams"):
        ctx, sh, Y, dev = _setup(N, pr, t=0.25, prec="tf32", factor_schedule=schedule)
        _gpu_system(N, ctx, dev)
        b = ctx.kinematics(*dev)[2]
        assert ctx.factor("tf32") == 0
        x, rep = ctx.solve(b)
        assert rep[0]["converged"], rep
        sols.append(x.cpu().numpy())
        reps.append((rep[0]["outer"], rep[0]["inner"]))
        ctx.close()
    assert reps[0] == reps[1]
    assert np.array_equal(sols[0], sols[1])


@pytest.mark.parametrize("name", ["swimmer", "sperm2"])
def test_two_level_factor_matches_the_oracle_and_the_one_level_inverse(N, name):
    # The two-level elimination (256-column blocks, column panel eliminated in
    # 64-column steps, one rank-256 tensor-core update per block, from scaled
    # FP16 pairs or split TF32) forms the same inverse as the one-level one up
    # to FP32-level rounding: the refinement reaches the oracle's answer from it
    # with the same few GMRES iterations.
    pr = PROBLEMS[name]()
    A_or = b_or = None
    out = {}
    for schedule in ("two_level", "two_level_tf32", "streams"):
        ctx, sh, Y, dev = _setup(N, pr, t=0.25, prec="tf32", factor_schedule=schedule)
        _gpu_system(N, ctx, dev)
        b = ctx.kinematics(*dev)[2]
        assert ctx.factor("tf32") == 0
        x, rep = ctx.solve(b)
        assert rep[0]["converged"] and rep[0]["outer"] <= 4, (schedule, rep)
        assert rep[0]["inner"] <= 2 * rep[0]["outer"], (schedule, rep)
        if A_or is None:
            A_or, b_or, *_ = _oracle_system(pr, sh, Y)
            ref = O.solve(A_or, b_or)
        assert _rel(x.cpu().numpy(), ref) <= TOL_SOL, (schedule, rep)
        out[schedule] = rep[0]
        ctx.close()


def test_warm_start_and_multiple_rhs(N):
    pr = PROBLEMS["swimmer_small"]()
    ctx, sh, Y, dev = _setup(N, pr, t=0.1)
    x, Xw, b, *_ = _gpu_system(N, ctx, dev)
    ctx.factor("fp32")
    B2 = torch.stack([b, 2.0 * b])
    X2, reps = ctx.solve(B2)
    assert _rel(X2[1].cpu().numpy(), 2.0 * X2[0].cpu().numpy()) < 1e-12
    # starting from the answer, refinement stops after one step
    X3, reps3 = ctx.solve(b, x0=X2[0].contiguous())
    assert reps3[0]["outer"] <= 2
    assert _rel(X3.cpu().numpy(), X2[0].cpu().numpy()) < 1e-13


@pytest.mark.parametrize("name,prec", [("swimmer_small", "fp32"), ("sperm2", "fp32"),
                                       ("swimmer", "tf32")])
def test_rk2_step_matches_oracle(N, name, prec):
    pr = PROBLEMS[name]()
    t, dt = 0.05, 0.01
    ctx, sh, Y, dev0 = _setup(N, pr, t=t, prec=prec)
    devh = N.shapes_to_device(g.pack_shapes(pr, t + 0.5 * dt))
    s0, shf = N.Context.shapes(*dev0), N.Context.shapes(*devh)
    sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
    rep = ctx.step(s0, shf, dt, sol=sol)
    Yg = ctx.get_state()
    Yo, stages = O.rk2_step(pr, Y, t, dt, return_stages=True)
    s = sol.cpu().numpy()
    assert _rel(s[:pr.n], stages["sol1"]) <= TOL_SOL, rep
    assert _rel(s[pr.n:], stages["sol2"]) <= TOL_SOL, rep
    assert np.allclose(Yg["x0"], Yo["x0"], rtol=0, atol=1e-13)
    assert np.allclose(Yg["B"], Yo["B"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("name,prec", [("sperm2", "fp32"), ("swimmer", "tf32")])
def test_consecutive_steps_match_oracle(N, name, prec):
    # several steps in a row (for the channel: the wall's map is computed once and kept)
    pr = PROBLEMS[name]()
    dt = 0.01
    ctx, sh, Y, dev = _setup(N, pr, t=0.0, prec=prec)
    Yo = Y
    for k in range(3):
        t = k * dt
        d0 = N.shapes_to_device(g.pack_shapes(pr, t))
        dh = N.shapes_to_device(g.pack_shapes(pr, t + 0.5 * dt))
        ctx.step(N.Context.shapes(*d0), N.Context.shapes(*dh), dt)
        Yo = O.rk2_step(pr, Yo, t, dt)
    Yg = ctx.get_state()
    assert np.allclose(Yg["x0"], Yo["x0"], rtol=0, atol=1e-12)
    assert np.allclose(Yg["B"], Yo["B"], rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec", ["tf32", "fp64"])
def test_factor_reuse_and_warm_start_keep_the_oracle_trajectory(N, prec):
    # the previous stages' factor preconditions later stages; each solve still
    # meets the FP64 residual, so the trajectory stays on the oracle's
    pr = PROBLEMS["swimmer"]()
    dt = 0.01
    ctx, sh, Y, dev = _setup(N, pr, t=0.0, prec=prec, reuse_factor=True, warm_start=True)
    Yo = Y
    facts = 0
    for k in range(3):
        t = k * dt
        d0 = N.shapes_to_device(g.pack_shapes(pr, t))
        dh = N.shapes_to_device(g.pack_shapes(pr, t + 0.5 * dt))
        sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
        rep = ctx.step(N.Context.shapes(*d0), N.Context.shapes(*dh), dt, sol=sol)
        facts += rep["factorizations"]
        Yn, stages = O.rk2_step(pr, Yo, t, dt, return_stages=True)
        s = sol.cpu().numpy()
        assert _rel(s[:pr.n], stages["sol1"]) <= TOL_SOL, rep
        assert _rel(s[pr.n:], stages["sol2"]) <= TOL_SOL, rep
        Yo = Yn
    assert facts < 6  # at least one stage reused an earlier factor
    Yg = ctx.get_state()
    assert np.allclose(Yg["x0"], Yo["x0"], rtol=0, atol=1e-12)
    assert np.allclose(Yg["B"], Yo["B"], rtol=0, atol=1e-12)


def test_external_force_mobility(N):
    # rigid free body pushed by (F, M) from the oracle's resistance problem
    pr = PROBLEMS["swimmer_small"]()
    sh = g.pack_shapes(pr, 0.0)
    sh["xidot"][:] = 0.0
    ext = np.array([[0.01, -0.02, 0.005, 0.001, 0.002, -0.003]])
    ctx = N.Context.from_problem(pr)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    ctx.set_external(ext)
    dev = N.shapes_to_device(sh)
    x, Xw, b, *_ = _gpu_system(N, ctx, dev)
    ctx.factor("fp32")
    xg, _ = ctx.solve(b)
    A_or, b_or, *_ = _oracle_system(pr, sh, Y, ext=ext)
    assert _rel(xg.cpu().numpy(), O.solve(A_or, b_or)) <= TOL_SOL


def test_empty_segment_is_reported_singular(N):
    # a force point that no quadrature point maps to gives zero columns
    n_off, q_off = np.array([0, 3]), np.array([0, 4])
    x = np.zeros((3, 4))
    x[:, :3] = [[0, 0, 0], [1, 0, 0], [50, 0, 0]]
    Xw = np.zeros((4, 4))
    Xw[:, :3] = [[0.1, 0, 0], [-0.1, 0, 0], [0.9, 0, 0], [1.1, 0.1, 0]]
    Xw[:, 3] = 0.25
    ctx = N.Context(n_off, q_off, [N.PRESCRIBED], eps=0.1, U=[[1, 0, 0]], Omega=[[0, 0, 0]])
    xd = torch.from_numpy(x).cuda()
    Xd = torch.from_numpy(Xw).cuda()
    nn, seg_ptr, perm = ctx.nearest_build(xd, Xd)
    assert list(seg_ptr.cpu().numpy()) == [0, 2, 4, 4]
    ctx.assemble(xd, Xd, want_matrix=False)
    assert ctx.factor("fp32") > 0
    assert ctx.factor("fp64") > 0


def test_bad_arguments_are_rejected(N):
    with pytest.raises(N.NrsError) as ei:
        N.Context([0, 3], [0, 4], [N.FREE], eps=-1.0)
    assert ei.value.status == N.NRS_EINVAL
    with pytest.raises(N.NrsError):
        N.Context([0, 0], [0, 4], [N.FREE], eps=0.1)  # quadrature points without force points
    pr = PROBLEMS["swimmer_small"]()
    with pytest.raises(N.NrsError) as ei:
        N.Context.from_problem(pr, factor_prec="bf16")  # no BF16 factorisation is built
    assert ei.value.status == N.NRS_EINVAL
    ctx = N.Context.from_problem(pr)
    with pytest.raises(N.NrsError) as ei:
        ctx.factor("fp32")  # nothing assembled yet
    assert ei.value.status == N.NRS_EINVAL
    sh = g.pack_shapes(pr, 0.0)
    xi, Xiw, xidot = N.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    ctx.assemble(x, Xw, want_matrix=False)
    with pytest.raises(N.NrsError) as ei:
        ctx.factor("bf16")
    assert ei.value.status == N.NRS_EINVAL


def test_single_force_point(N):
    n_off, q_off = np.array([0, 1]), np.array([0, 5])
    x = np.zeros((1, 4))
    Xw = np.zeros((5, 4))
    Xw[:, :3] = np.random.default_rng(0).normal(size=(5, 3)) * 0.01
    Xw[:, 3] = 0.2
    ctx = N.Context(n_off, q_off, [N.PRESCRIBED], eps=0.05, U=[[0, 1, 0]], Omega=[[0, 0, 0]])
    xd, Xd = torch.from_numpy(x).cuda(), torch.from_numpy(Xw).cuda()
    ctx.nearest_build(xd, Xd)
    At = ctx.assemble(xd, Xd)
    A_or = O.assemble_stokeslet(x, Xw, np.zeros(5, dtype=np.int32), 0.05, 1.0)
    assert np.allclose(At.T.cpu().numpy(), A_or, rtol=1e-13)


@pytest.mark.parametrize("name", ["swimmer", "sperm2"])
def test_float_pair_arnoldi_keeps_the_oracle_trajectory(N, name):
    # GMRES products with the float-pair copy of A (about 2^-46 of |A||v|):
    # the residual still uses the FP64 matrix, so every solve reaches the
    # oracle's answer; the iteration counts stay those of the FP64 products
    pr = PROBLEMS[name]()
    dt = 0.01
    runs = {}
    for arnoldi in ("fp64", "df"):
        ctx, sh, Y, dev = _setup(N, pr, t=0.0, prec="tf32", reuse_factor=True, warm_start=True,
                                 reuse_max_inner=40, arnoldi=arnoldi)
        Yo = Y
        inner = 0
        for k in range(3):
            t = k * dt
            d0 = N.shapes_to_device(g.pack_shapes(pr, t))
            dh = N.shapes_to_device(g.pack_shapes(pr, t + 0.5 * dt))
            sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
            rep = ctx.step(N.Context.shapes(*d0), N.Context.shapes(*dh), dt, sol=sol)
            inner += rep["stages"][0]["inner"] + rep["stages"][1]["inner"]
            Yn, stages = O.rk2_step(pr, Yo, t, dt, return_stages=True)
            s = sol.cpu().numpy()
            assert _rel(s[:pr.n], stages["sol1"]) <= TOL_SOL, (arnoldi, rep)
            assert _rel(s[pr.n:], stages["sol2"]) <= TOL_SOL, (arnoldi, rep)
            Yo = Yn
        runs[arnoldi] = inner
        ctx.close()
    assert runs["df"] <= runs["fp64"] + 3, runs

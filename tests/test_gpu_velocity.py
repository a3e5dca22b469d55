"""Fluid velocity at field points and passive tracers (the particle tracking
of the paper's mouse-node and sperm examples) through the C ABI, against the
FP64 oracle.

The velocity u(x_p) = (1/8 pi mu) sum_q S^eps(x_p - X_q) w_q f_n(q) is a plain
sum: the GPU evaluates every term as the oracle does, but adds contiguous
ranges of q separately, so the two agree to rounding of the sum (1e-13 of
the largest |u|).  The tracers move by dt times stage velocities built from
the stage solutions, which agree with the oracle's to 1e-10.
"""

import numpy as np
import pytest
import torch

import oracle as O
from synth import geometry as g

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "swimmer_small": lambda: g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8),
    "sperm2": lambda: g.sperm_channel_config(count=2, n_head=40, q_head=400, n_flag=60, q_flag=600,
                                             wall_f=(20, 6, 3), wall_q=(60, 18, 9)),
}


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


def _field_points(pr, x_lab, count, seed):
    """Seeded points around the bodies: force points pushed outward by a few
    point spacings, and points in the bounding box."""
    rng = np.random.default_rng(seed)
    lo, hi = x_lab[:, :3].min(axis=0), x_lab[:, :3].max(axis=0)
    xp = np.zeros((count, 4))
    xp[:, :3] = lo + (hi - lo) * rng.uniform(size=(count, 3))
    k = count // 2
    idx = rng.integers(0, len(x_lab), size=k)
    xp[:k, :3] = x_lab[idx, :3] + 0.02 * rng.normal(size=(k, 3))
    return xp


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_velocity_matches_oracle(N, name):
    pr = PROBLEMS[name]()
    sh = g.pack_shapes(pr, 0.2)
    Y = g.initial_state(pr)
    ctx = N.Context.from_problem(pr, factor_prec="tf32")
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = N.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    x_or, Xw_or = O.lab_frame(sh, Y)
    nn_or = O.nearest(sh["x"], sh["Xw"], sh["n_off"], sh["q_off"])
    xp = _field_points(pr, x_or, 333, 5)
    f = np.random.default_rng(6).normal(size=3 * pr.N)
    u = ctx.velocity(torch.from_numpy(xp).cuda(), torch.from_numpy(f).cuda(), Xw).cpu().numpy()
    u_or = O.velocity(xp, Xw_or, nn_or, f, pr.eps, pr.mu)
    assert np.all(u[:, 3] == 0.0)
    assert np.abs(u - u_or).max() <= 1e-13 * np.abs(u_or).max()


def test_velocity_of_one_point_is_its_row_of_the_operator(N):
    # at the force points the velocity of a density f is A_s f (first 3N rows
    # of the assembled matrix, which is bit-exact with the oracle's)
    pr = PROBLEMS["swimmer_small"]()
    sh = g.pack_shapes(pr, 0.4)
    Y = g.initial_state(pr)
    ctx = N.Context.from_problem(pr, factor_prec="tf32")
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = N.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    At = ctx.assemble(x, Xw)
    f = torch.from_numpy(np.random.default_rng(7).normal(size=3 * pr.N)).cuda()
    u = ctx.velocity(x, f, Xw)
    ref = (At[:3 * pr.N, :3 * pr.N].T @ f).reshape(-1, 3)
    assert torch.abs(u[:, :3] - ref).max().item() <= 1e-13 * torch.abs(ref).max().item()


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("graph", [False, True])
def test_tracers_step_with_the_bodies_as_the_oracle(N, name, graph):
    pr = PROBLEMS[name]()
    dt = pr.dt
    Y0 = g.initial_state(pr)
    x_or, _ = O.lab_frame(g.pack_shapes(pr, 0.0), Y0)
    tr = _field_points(pr, x_or, 64, 8)
    ctx = N.Context.from_problem(pr, factor_prec="tf32", graph=graph)
    ctx.set_state(Y0["x0"], Y0["B"])
    ctx.set_tracers(tr)
    bufs = None
    Y, T = Y0, tr
    for s in range(3):
        d0 = N.shapes_to_device(g.pack_shapes(pr, s * dt))
        dh = N.shapes_to_device(g.pack_shapes(pr, (s + 0.5) * dt))
        if bufs is None:
            bufs = (d0, dh)
        else:  # graph mode replays the recorded step: same shape buffers
            for src, dst in zip(d0 + dh, bufs[0] + bufs[1]):
                dst.copy_(src)
        ctx.step(N.Context.shapes(*bufs[0]), N.Context.shapes(*bufs[1]), dt)
        Y, T, st = O.rk2_step_tracers(pr, Y, T, s * dt, dt)
        Tg = ctx.get_tracers()
        umax = max(np.abs(st["u1"][:, :3]).max(), np.abs(st["u2"][:, :3]).max())
        assert np.abs(Tg[:, :3] - T[:, :3]).max() <= 1e-10 * (s + 1) * dt * umax + 1e-15, s
        assert np.array_equal(Tg[:, 3], tr[:, 3])

"""The refinement's residual r = b - A x (nrs_residual) against exact rational
arithmetic and the oracle.

With the extended residual (the default) every product's rounded value is
summed exactly as a fixed-point integer and the rounding errors in FP64, so r
is within about u^2 (|A| |x|)_i of the exact b_i - (A x)_i, plus its final
rounding: |r_i - exact_i| <= 2^-52 |exact_i| + 2^-96 (|A| |x|)_i.  The plain
FP64 residual obeys only the classical bound gamma_n (|A| |x|)_i.  The matrix
is the assembled stokeslet system of the CUDA path, which is the oracle's bit
for bit.
"""

from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle as O
from synth import geometry as g

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


def _system(N, pr, residual="extended", t=0.25):
    sh = g.pack_shapes(pr, t)
    ctx = N.Context.from_problem(pr, residual=residual)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = N.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    At = ctx.assemble(x, Xw)
    return ctx, At.T.cpu().numpy(), b.cpu().numpy()


def _exact_rows(A, x, b, rows):
    out = []
    for i in rows:
        s = Fraction(b[i])
        for j in range(A.shape[1]):
            if A[i, j] != 0.0 and x[j] != 0.0:
                s -= Fraction(A[i, j]) * Fraction(x[j])
        out.append(s)
    return out


def _check_extended(A, x, b, r, rows):
    absAx = np.abs(A) @ np.abs(x)
    for i, ex in zip(rows, _exact_rows(A, x, b, rows)):
        err = abs(Fraction(r[i]) - ex)
        bound = abs(ex) * Fraction(2) ** -52 + Fraction(absAx[i]) * Fraction(2) ** -96 \
            + Fraction(2) ** -1074
        assert err <= bound, (i, float(err), float(bound))
    # every row against the oracle's double-double residual (itself within
    # 2^-50 |exact| + 2^-100 |A||x| of exact)
    ro = O.residual_dd(A, x, b)
    tol = 2.0 ** -49 * np.abs(ro) + 2.0 ** -94 * absAx
    assert np.all(np.abs(r - ro) <= tol), np.max(np.abs(r - ro) / np.maximum(tol, 1e-300))


PROBLEMS = {
    "swimmer": lambda: g.swimmer_config(),
    "sperm2": lambda: g.sperm_channel_config(count=2, n_head=40, q_head=400, n_flag=60, q_flag=600,
                                             wall_f=(20, 6, 3), wall_q=(60, 18, 9)),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_residual_at_the_solution_is_exact_to_u2(N, name):
    # at the oracle's solution b - A x cancels to ~1e-16 |b|: the case the
    # refinement's last steps live in
    ctx, A, b = _system(N, PROBLEMS[name]())
    x = O.solve(A, b)
    r = ctx.residual(torch.from_numpy(b).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    rows = np.unique(np.linspace(0, len(b) - 1, 12).astype(int))
    _check_extended(A, x, b, r, rows)
    ctx.close()


def test_residual_wide_dynamic_range(N):
    ctx, A, b = _system(N, PROBLEMS["swimmer"]())
    rng = np.random.default_rng(11)
    n = len(b)
    x = rng.normal(size=n) * 10.0 ** rng.uniform(-30, 30, size=n)
    bb = A @ x * (1 + 1e-9 * rng.normal(size=n))
    r = ctx.residual(torch.from_numpy(bb).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    _check_extended(A, x, bb, r, [0, 7, n // 2, n - 1])
    ctx.close()


@pytest.mark.parametrize("scale", [2.0 ** -990, 2.0 ** -500, 2.0 ** 400])
def test_residual_extreme_magnitudes(N, scale):
    # the fixed-point anchor follows ||A|| ||x|| down towards underflow and up
    ctx, A, b = _system(N, PROBLEMS["sperm2"]())
    rng = np.random.default_rng(12)
    n = len(b)
    x = rng.normal(size=n) * scale
    bb = (A @ x) * (1 + 1e-7 * rng.normal(size=n))
    r = ctx.residual(torch.from_numpy(bb).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(np.isfinite(r))
    rows = [0, 5, n // 3, n - 1]
    absAx = np.abs(A) @ np.abs(x)
    for i, ex in zip(rows, _exact_rows(A, x, bb, rows)):
        err = abs(Fraction(r[i]) - ex)
        # near underflow the subnormal spacing 2^-1074 limits every result
        bound = abs(ex) * Fraction(2) ** -52 + Fraction(absAx[i]) * Fraction(2) ** -96 \
            + 4 * n * Fraction(2) ** -1074
        assert err <= bound, (i, float(err), float(bound))
    ctx.close()


def test_residual_special_cases_are_exact(N):
    ctx, A, b = _system(N, PROBLEMS["sperm2"]())
    n = len(b)
    bd = torch.from_numpy(b).cuda()
    # x = 0: r = b exactly
    r = ctx.residual(bd, torch.zeros(n, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.array_equal(r, b)
    # x = e_j: every product exact, one rounding of b - A[:, j]
    for j in (0, n // 2, n - 1):
        e = torch.zeros(n, dtype=torch.float64, device="cuda")
        e[j] = 1.0
        r = ctx.residual(bd, e).cpu().numpy()
        assert np.array_equal(r, b - A[:, j]), j
    # x = -2 e_j: negative products, still exact
    e = torch.zeros(n, dtype=torch.float64, device="cuda")
    e[3] = -2.0
    r = ctx.residual(bd, e).cpu().numpy()
    assert np.array_equal(r, b + 2.0 * A[:, 3])
    # r may overwrite x
    x = torch.from_numpy(O.solve(A, b)).cuda()
    r1 = ctx.residual(bd, x)
    xx = x.clone()
    assert ctx._check(N._lib.nrs_residual(ctx._h, N._ptr(bd), N._ptr(xx), N._ptr(xx))) == 0
    assert torch.equal(xx, r1)
    ctx.close()


def test_residual_propagates_non_finite(N):
    ctx, A, b = _system(N, PROBLEMS["sperm2"]())
    n = len(b)
    for bad in (float("nan"), float("inf")):
        x = torch.ones(n, dtype=torch.float64, device="cuda")
        x[n // 3] = bad
        r = ctx.residual(torch.from_numpy(b).cuda(), x).cpu().numpy()
        assert not np.any(np.isfinite(r[A[:, n // 3] != 0.0]))
    ctx.close()


def test_plain_fp64_residual_obeys_the_classical_bound(N):
    ctx, A, b = _system(N, PROBLEMS["sperm2"](), residual="fp64")
    x = O.solve(A, b)
    r = ctx.residual(torch.from_numpy(b).cuda(), torch.from_numpy(x).cuda()).cpu().numpy()
    n = len(b)
    gamma = n * U / (1 - n * U)
    ro = O.residual_dd(A, x, b)
    assert np.all(np.abs(r - ro) <= 2 * gamma * (np.abs(A) @ np.abs(x) + np.abs(b)))
    ctx.close()


def test_residual_requires_an_assembly(N):
    pr = PROBLEMS["sperm2"]()
    ctx = N.Context.from_problem(pr)
    z = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    with pytest.raises(N.NrsError) as ei:
        ctx.residual(z, z)
    assert ei.value.status == N.NRS_EINVAL
    ctx.close()


@pytest.mark.parametrize("arnoldi", ["fp64", "df"])
def test_refinement_ends_on_an_exact_residual(N, arnoldi):
    # From a cold start (x = M b, backward error far above 1e-8) the first
    # refinement step keeps a working-precision residual; the refinement may
    # not end on one, so at least one exact residual follows, every step kept
    # one of the two, and the answer is the oracle's to working accuracy
    # (backward error in the oracle's FP64 system, double-double residual).
    pr = g.swimmer_config(ns_f=40, nth_f=6, ns_q=200, nth_q=10)
    sh = g.pack_shapes(pr, 0.25)
    ctx = N.Context.from_problem(pr, factor_prec="tf32", arnoldi=arnoldi)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = N.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    At = ctx.assemble(x, Xw)
    assert ctx.factor("tf32") == 0
    r0, c0 = ctx.residual_counters(), ctx.counters()
    xg, rep = ctx.solve(b)
    r1, c1 = ctx.residual_counters(), ctx.counters()
    assert rep[0]["converged"], rep
    exact, working = r1["exact"] - r0["exact"], r1["working"] - r0["working"]
    outer = c1["outer"] - c0["outer"]
    assert working >= 1 and exact >= 1, (exact, working, rep)
    assert exact + working >= outer >= 2, (exact, working, outer)
    A = At.T.cpu().numpy()
    bh, xs = b.cpu().numpy(), xg.cpu().numpy()
    r = O.residual_dd(A, xs, bh)
    berr = np.max(np.abs(r)) / (np.max(np.sum(np.abs(A), axis=1)) * np.max(np.abs(xs))
                                + np.max(np.abs(bh)))
    assert berr <= 1e-15, berr

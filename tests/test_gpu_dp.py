"""Adaptive Dormand-Prince stepping (the ode45 integrator of Sec. 4) through
the C ABI against the oracle's, and against the exact motion of a body with
prescribed rotation."""

import math

import numpy as np
import pytest
import torch

import oracle as O
from synth import geometry as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


def _shapes_fn(N, pr):
    cache = {}

    def at(t):
        key = round(t, 15)
        if key not in cache:
            cache[key] = N.shapes_to_device(g.pack_shapes(pr, t))
        return N.Context.shapes(*cache[key])
    return at


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_first_dormand_prince_step_matches_oracle(N):
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    Y0 = g.initial_state(pr)
    ctx = N.Context.from_problem(pr, factor_prec="tf32")
    ctx.set_state(Y0["x0"], Y0["B"])
    at = _shapes_fn(N, pr)
    h, rtol, atol = 0.01, 1e-4, 1e-6
    ctx.dp_start(0.0, 1.0, h, rtol, atol)
    times = []
    for _ in range(7):
        times.append(ctx.dp_next_time())
        info = ctx.dp_stage(at(times[-1]))
    assert np.allclose(times, [c * h for c in O.DP_C], rtol=0, atol=1e-15)
    Yn, K, err = O.dp_step(pr, Y0, 0.0, h, rtol, atol)
    assert err < 0.5 and info["last_accepted"] == 1 and info["accepted"] == 1
    assert info["t"] == pytest.approx(h, abs=1e-15)
    assert info["err"] == pytest.approx(err, rel=1e-3)
    Yg = ctx.get_state()
    assert _rel(Yg["x0"], Yn["x0"]) <= 1e-12
    assert _rel(Yg["B"], Yn["B"]) <= 1e-12


def test_dormand_prince_integration_matches_oracle(N):
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    Y0 = g.initial_state(pr)
    ctx = N.Context.from_problem(pr, factor_prec="tf32")
    ctx.set_state(Y0["x0"], Y0["B"])
    tol, T = 1e-8, 0.05
    info = ctx.dp_integrate(_shapes_fn(N, pr), 0.0, T, 0.02, tol, tol)
    assert info["done"] == 1 and info["t"] == pytest.approx(T, abs=1e-14)
    Yo, t, acc, rej = O.dp_integrate(pr, Y0, 0.0, T, 0.02, tol, tol)
    Yg = ctx.get_state()
    scale = np.abs(Yo["x0"]).max() + 1.0
    assert np.abs(Yg["x0"] - Yo["x0"]).max() <= 100 * tol * scale
    assert np.abs(Yg["B"] - Yo["B"]).max() <= 100 * tol


def test_dormand_prince_returns_a_rotating_body_to_its_start(N):
    Om = np.array([1.0, 2.0, -2.0])
    pr = g.sphere_config(n_force=2, n_quad=4, U=(0.0, 0.0, 0.0), Omega=tuple(Om))
    T = 2 * math.pi / np.linalg.norm(Om)
    Y0 = g.initial_state(pr)
    ctx = N.Context.from_problem(pr, factor_prec="tf32")
    ctx.set_state(Y0["x0"], Y0["B"])
    tol = 1e-8
    info = ctx.dp_integrate(_shapes_fn(N, pr), 0.0, T, 1.0, tol, tol)
    assert info["done"] == 1 and info["rejected"] >= 1
    assert np.abs(ctx.get_state()["B"][0] - np.eye(3)).max() <= 50 * tol

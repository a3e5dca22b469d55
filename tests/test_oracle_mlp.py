"""Pins of the FP64 oracle of the learned starting guess (oracle/mlp.py).

The paper has no learned component; these tests fix the oracle MLP to what
mathematics fixes independently of its code: central finite differences of
the loss, PyTorch autograd on the same network, closed forms of Adam, the
special cases of the network, and the rotation invariance of the body-frame
features.  Each is chosen so that a plausible slip (a dropped bias, a
transposed weight, a wrong SiLU derivative, a missing bias correction, a
B instead of B^T) fails at least one of them.
"""

import math

import numpy as np
import pytest
import torch

from oracle import mlp as M
from synth import mlp_batch, mlp_init, mlp_perturb


@pytest.fixture(scope="module")
def case():
    P = mlp_perturb(7, mlp_init(3), 0.2).astype(np.float64)
    X, T = mlp_batch(11, 23)
    return P, X.astype(np.float64), T.astype(np.float64)


def test_layout_size():
    assert M.NPARAM == 64 * 17 + 64 + 64 * 64 + 64 + 3 * 64 + 3 == 5507
    p = M.unpack(np.arange(M.NPARAM, dtype=np.float64))
    assert p["W1"][1, 0] == 17 and p["b1"][0] == 64 * 17 and p["b3"][-1] == M.NPARAM - 1


def test_silu_special_values():
    assert M.silu(0.0) == 0.0
    assert M.silu_grad(0.0) == 0.5
    assert abs(M.silu(40.0) - 40.0) < 1e-12 and abs(M.silu(-40.0)) < 1e-15
    z = np.linspace(-6, 6, 13)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    assert np.allclose(M.silu_grad(z), fd, rtol=1e-8, atol=1e-10)


def test_forward_special_cases(case):
    _, X, _ = case
    # all weights zero: the output is b3
    P = np.zeros(M.NPARAM)
    P[M.OFF_B3:] = [0.5, -1.0, 2.0]
    Y, _ = M.forward(P, X)
    assert np.array_equal(Y, np.tile([0.5, -1.0, 2.0], (X.shape[0], 1)))
    # first layer zero: h1 = SiLU(0) = 0, so y = W3 SiLU(b2) + b3 whatever x is
    rng = np.random.Generator(np.random.PCG64(5))
    P = np.zeros(M.NPARAM)
    b2 = rng.uniform(-1, 1, 64)
    W3 = rng.uniform(-1, 1, (3, 64))
    P[M.OFF_B2:M.OFF_W3] = b2
    P[M.OFF_W3:M.OFF_B3] = W3.ravel()
    Y, _ = M.forward(P, X)
    want = np.array([sum(W3[o, j] * b2[j] / (1 + math.exp(-b2[j])) for j in range(64))
                     for o in range(3)])
    assert np.allclose(Y, want[None, :], rtol=1e-14, atol=1e-14)


def test_forward_matches_torch(case):
    P, X, _ = case
    p = M.unpack(P)
    xt = torch.from_numpy(X)
    h1 = torch.nn.functional.silu(xt @ torch.from_numpy(p["W1"]).T + torch.from_numpy(p["b1"]))
    h2 = torch.nn.functional.silu(h1 @ torch.from_numpy(p["W2"]).T + torch.from_numpy(p["b2"]))
    y = h2 @ torch.from_numpy(p["W3"]).T + torch.from_numpy(p["b3"])
    Y, _ = M.forward(P, X)
    assert np.allclose(Y, y.numpy(), rtol=1e-13, atol=1e-13)


def test_gradient_matches_autograd(case):
    P, X, T = case
    Pt = torch.from_numpy(P.copy()).requires_grad_(True)
    W1 = Pt[M.OFF_W1:M.OFF_B1].reshape(64, 17)
    W2 = Pt[M.OFF_W2:M.OFF_B2].reshape(64, 64)
    W3 = Pt[M.OFF_W3:M.OFF_B3].reshape(3, 64)
    xt = torch.from_numpy(X)
    h1 = torch.nn.functional.silu(xt @ W1.T + Pt[M.OFF_B1:M.OFF_W2])
    h2 = torch.nn.functional.silu(h1 @ W2.T + Pt[M.OFF_B2:M.OFF_W3])
    y = h2 @ W3.T + Pt[M.OFF_B3:]
    lt = torch.mean((y - torch.from_numpy(T)) ** 2)
    lt.backward()
    g, lo = M.grad(P, X, T)
    assert abs(lo - lt.item()) <= 1e-14 * abs(lo)
    assert np.allclose(g, Pt.grad.numpy(), rtol=1e-11, atol=1e-14)


def test_gradient_central_differences(case):
    """Every parameter block, by central differences of the FP64 loss."""
    P, X, T = case
    g, _ = M.grad(P, X, T)
    rng = np.random.Generator(np.random.PCG64(9))
    blocks = [(M.OFF_W1, M.OFF_B1), (M.OFF_B1, M.OFF_W2), (M.OFF_W2, M.OFF_B2),
              (M.OFF_B2, M.OFF_W3), (M.OFF_W3, M.OFF_B3), (M.OFF_B3, M.NPARAM)]
    idx = np.concatenate([rng.choice(np.arange(a, b), size=min(12, b - a), replace=False)
                          for a, b in blocks])
    h = 1e-5
    gmax = np.max(np.abs(g))
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (M.loss(M.forward(Pp, X)[0], T) - M.loss(M.forward(Pm, X)[0], T)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * (abs(g[k]) + 1e-3 * gmax), (k, fd, g[k])
    # and a directional derivative over all parameters at once
    d = rng.uniform(-1, 1, M.NPARAM)
    fd = (M.loss(M.forward(P + h * d, X)[0], T) - M.loss(M.forward(P - h * d, X)[0], T)) / (2 * h)
    assert abs(fd - g @ d) <= 1e-7 * np.abs(g) @ np.abs(d)


def test_grad_abs_bounds_gradient(case):
    P, X, T = case
    g, _ = M.grad(P, X, T)
    ga = M.grad_abs(P, X, T)
    assert np.all(np.abs(g) <= ga * (1 + 1e-12) + 1e-300)


def test_adam_first_step_is_lr_times_sign():
    g = np.array([3.0, -0.25, 1e-3, -7.0])
    P0 = np.array([1.0, 2.0, 3.0, 4.0])
    P1, m, v = M.adam(P0, np.zeros(4), np.zeros(4), g, 0.01, 1)
    # mhat = g, vhat = g^2 after bias correction
    assert np.allclose(P1, P0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_steps_are_constant():
    g = np.array([0.5, -2.0])
    P = np.zeros(2)
    m = np.zeros(2)
    v = np.zeros(2)
    for t in range(1, 8):
        Pn, m, v = M.adam(P, m, v, g, 0.1, t)
        assert np.allclose(Pn - P, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        P = Pn


def test_adam_zero_gradient_leaves_parameters():
    P = np.array([1.0, -1.0])
    P1, _, _ = M.adam(P, np.zeros(2), np.zeros(2), np.zeros(2), 0.5, 1)
    assert np.array_equal(P1, P)


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _toy():
    """Two bodies: a free one with 3 points and a static one with 2."""
    xi = np.array([[1.0, 0, 0, 0], [0, 2.0, 0, 0], [0, 0, -0.5, 0],
                   [3.0, 0, 0, 0], [0, 0, 1.0, 0]])
    xidot = np.array([[0, 0.1, 0, 0], [0.2, 0, 0, 0], [0, 0, 0.3, 0],
                      [0, 0, 0, 0], [0, 0, 0, 0]])
    W = np.array([1.0, 2.0, 3.0, 5.0, 5.0])
    n_off = np.array([0, 3, 5])
    kind = np.array([M.FREE, M.STATIC])
    return xi, xidot, W, n_off, kind


def test_features_hand_computed():
    xi, xidot, W, n_off, kind = _toy()
    B = np.stack([_rot([0, 0, 1], math.pi / 2), np.eye(3)])
    vprev = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 2.0])  # U = e_x, Omega = 2 e_z (lab frame)
    scl = np.array([2.0, 0.5, 1.0])
    X = M.features(xi, xidot, W, n_off, kind, B, np.zeros((2, 3)), np.zeros((2, 3)), vprev, scl)
    assert X.shape == (5, 17)
    assert np.allclose(X[1, 0:3], [0, 1.0, 0]) and np.allclose(X[0, 3:6], [0, 0.2, 0])
    assert np.allclose(X[:3, 6], [0, 0.5, 1.0]) and np.allclose(X[3:, 6], [0, 1.0])
    assert np.allclose(X[:3, 7], [0.5, 1.0, 1.5]) and np.allclose(X[3:, 7], [1.0, 1.0])
    assert np.array_equal(X[:3, 8:11], np.tile([1, 0, 0], (3, 1)))
    assert np.array_equal(X[3:, 8:11], np.tile([0, 0, 1], (2, 1)))
    # B rotates body x to lab y: lab U = e_x is body -y; lab Omega = 2 e_z is body 2 e_z
    assert np.allclose(X[0, 11:14], [0, -2.0, 0]) and np.allclose(X[0, 14:17], [0, 0, 8.0])
    assert np.allclose(X[3:, 11:17], 0.0)


def test_features_and_targets_are_rotation_invariant():
    xi, xidot, W, n_off, kind = _toy()
    rng = np.random.Generator(np.random.PCG64(2))
    B = np.stack([_rot(rng.normal(size=3), 0.7), _rot(rng.normal(size=3), -1.1)])
    vprev = rng.normal(size=6)
    f = rng.normal(size=15)
    scl = np.array([1.5, 0.7, 2.0])
    X = M.features(xi, xidot, W, n_off, kind, B, np.zeros((2, 3)), np.zeros((2, 3)), vprev, scl)
    T = M.targets(f, n_off, B, scl[2])
    R = _rot([1, 2, 3], 0.4)
    B2 = np.stack([R @ B[0], R @ B[1]])
    v2 = np.concatenate([R @ vprev[:3], R @ vprev[3:]])
    f2 = (f.reshape(5, 3) @ R.T).ravel()
    X2 = M.features(xi, xidot, W, n_off, kind, B2, np.zeros((2, 3)), np.zeros((2, 3)), v2, scl)
    T2 = M.targets(f2, n_off, B2, scl[2])
    assert np.allclose(X, X2, atol=1e-14) and np.allclose(T, T2, atol=1e-14)


def test_start_vector_inverts_targets():
    xi, xidot, W, n_off, kind = _toy()
    rng = np.random.Generator(np.random.PCG64(4))
    B = np.stack([_rot(rng.normal(size=3), 0.3), _rot(rng.normal(size=3), 2.0)])
    f = rng.normal(size=15)
    vprev = rng.normal(size=6)
    T = M.targets(f, n_off, B, 3.0)
    x = M.start_vector(T, n_off, B, 3.0, vprev, 1)
    assert np.allclose(x[:15], f, atol=1e-14) and np.array_equal(x[15:], vprev)


def test_prescribed_body_uses_its_motion():
    xi, xidot, W, n_off, _ = _toy()
    kind = np.array([M.PRESCRIBED, M.STATIC])
    B = np.stack([np.eye(3), np.eye(3)])
    U = np.array([[1.0, 2.0, 3.0], [9.0, 9.0, 9.0]])
    Om = np.array([[0.0, 0.0, 1.0], [9.0, 9.0, 9.0]])
    X = M.features(xi, xidot, W, n_off, kind, B, U, Om, None, np.array([1.0, 1.0, 1.0]))
    assert np.allclose(X[:3, 11:14], [1, 2, 3]) and np.allclose(X[:3, 14:17], [0, 0, 1])
    assert np.allclose(X[3:, 11:17], 0.0)
    assert np.array_equal(X[:3, 8:11], np.tile([0, 1, 0], (3, 1)))


def test_scales():
    xi = np.array([[3.0, 4.0, 0, 0], [1.0, 0, 0, 0]])
    b = np.array([0, 0, 2.0, 1.0, 0, 0])
    f = np.array([1.0, 0, 0, 0, 1.0, 1.0])
    s = M.scales(xi, b, f)
    assert np.allclose(s, [5.0, 2.0, math.sqrt(1.5)])
    assert np.array_equal(M.scales(np.zeros((2, 4)), np.zeros(6), np.zeros(6)), [1.0, 1.0, 1.0])

"""FP64 oracle of the learned starting guess (the point-wise MLP).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests, the smoke run
and the CPU-baseline legs of the benchmark may import it.

The paper has no learned component.  This module states, in plain numpy
float64, what the CUDA path computes for the MLP that predicts the starting
vector of the refinement of Sec. 4 step 3:

* features of each force point (body frame) and the body-frame targets;
* a two-hidden-layer perceptron with SiLU activations and its loss (mean
  squared error);
* the gradient of that loss by reverse-mode differentiation written out
  layer by layer (Rumelhart, Hinton & Williams 1986);
* one step of Adam (Kingma & Ba 2015, Algorithm 1; beta1 = 0.9,
  beta2 = 0.999, epsilon = 1e-8);
* the scales and the start vector built from a prediction.

The parameter vector has the layout of the C interface:
W1 [64][17] row-major, b1 [64], W2 [64][64], b2 [64], W3 [3][64], b3 [3].

Parity pins: the gradient against central finite differences of the loss;
Adam against its closed forms (first step = lr * sign(g); a constant gradient
gives a step of lr * g / (|g| + eps') at every t); the features against
rotation invariance and hand-computed values.
"""

from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

IN, HID, OUT = 17, 64, 3
OFF_W1 = 0
OFF_B1 = OFF_W1 + HID * IN
OFF_W2 = OFF_B1 + HID
OFF_B2 = OFF_W2 + HID * HID
OFF_W3 = OFF_B2 + HID
OFF_B3 = OFF_W3 + OUT * HID
NPARAM = OFF_B3 + OUT

FREE, PRESCRIBED, STATIC = 0, 1, 2


def unpack(P: np.ndarray) -> Dict[str, np.ndarray]:
    """Views of the parameter vector as the weight matrices and biases."""
    P = np.asarray(P, dtype=np.float64)
    return {
        "W1": P[OFF_W1:OFF_B1].reshape(HID, IN),
        "b1": P[OFF_B1:OFF_W2],
        "W2": P[OFF_W2:OFF_B2].reshape(HID, HID),
        "b2": P[OFF_B2:OFF_W3],
        "W3": P[OFF_W3:OFF_B3].reshape(OUT, HID),
        "b3": P[OFF_B3:NPARAM],
    }


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, np.ravel(W3), b3]).astype(np.float64)


def silu(z):
    """SiLU(z) = z * sigmoid(z) = z / (1 + e^-z)."""
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    """d/dz [z sigma(z)] = sigma(z) (1 + z (1 - sigma(z)))."""
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(P: np.ndarray, X: np.ndarray) -> Tuple[np.ndarray, Dict[str, np.ndarray]]:
    """Y = W3 SiLU(W2 SiLU(W1 x + b1) + b2) + b3 for every row x of X."""
    p = unpack(P)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = silu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = silu(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, {"X": X, "Z1": Z1, "H1": H1, "Z2": Z2, "H2": H2}


def loss(Y: np.ndarray, T: np.ndarray) -> float:
    """Mean of the squared error over all points and components."""
    D = np.asarray(Y, dtype=np.float64) - np.asarray(T, dtype=np.float64)
    return float(np.mean(D * D))


def grad(P: np.ndarray, X: np.ndarray, T: np.ndarray) -> Tuple[np.ndarray, float]:
    """Gradient of loss(forward(P, X), T) with respect to P, by the chain rule
    applied layer by layer from the output back to the input."""
    p = unpack(P)
    Y, c = forward(P, X)
    npts = Y.shape[0]
    dY = 2.0 * (Y - T) / (OUT * npts)          # d loss / d Y
    gW3 = dY.T @ c["H2"]
    gb3 = dY.sum(axis=0)
    D2 = (dY @ p["W3"]) * silu_grad(c["Z2"])   # d loss / d Z2
    gW2 = D2.T @ c["H1"]
    gb2 = D2.sum(axis=0)
    D1 = (D2 @ p["W2"]) * silu_grad(c["Z1"])   # d loss / d Z1
    gW1 = D1.T @ c["X"]
    gb1 = D1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3), loss(Y, T)


def grad_abs(P: np.ndarray, X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """The gradient's sums taken over absolute values of every term (the
    magnitude that rounding errors of a reordered evaluation scale with)."""
    p = unpack(P)
    Y, c = forward(P, X)
    npts = Y.shape[0]
    dY = np.abs(2.0 * (Y - T) / (OUT * npts))
    gW3 = dY.T @ np.abs(c["H2"])
    gb3 = dY.sum(axis=0)
    D2 = (dY @ np.abs(p["W3"])) * np.abs(silu_grad(c["Z2"]))
    gW2 = D2.T @ np.abs(c["H1"])
    gb2 = D2.sum(axis=0)
    D1 = (D2 @ np.abs(p["W2"])) * np.abs(silu_grad(c["Z1"]))
    gW1 = D1.T @ np.abs(c["X"])
    gb1 = D1.sum(axis=0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def forward_abs(P: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Output magnitudes |b3| + |W3| |SiLU(Z2)| (with |Z2| from absolute
    sums as well): the scale of the rounding error of the forward pass."""
    p = unpack(P)
    Y, c = forward(P, X)
    A1 = np.abs(c["X"]) @ np.abs(p["W1"]).T + np.abs(p["b1"])
    A2 = np.abs(c["H1"]) @ np.abs(p["W2"]).T + np.abs(p["b2"]) + A1 @ np.abs(p["W2"]).T
    return np.abs(c["H2"]) @ np.abs(p["W3"]).T + np.abs(p["b3"]) + A2 @ np.abs(p["W3"]).T


def adam(P, m, v, g, lr: float, t: int):
    """One Adam step at step count t (>= 1): biased moments, bias correction,
    update P - lr * mhat / (sqrt(vhat) + 1e-8).  Returns (P, m, v)."""
    b1, b2, eps = 0.9, 0.999, 1e-8
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return np.asarray(P, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def scales(xi: np.ndarray, b: np.ndarray, f: np.ndarray) -> np.ndarray:
    """L = max |xi_m|, V = max |b_m| over the force rows, F = RMS of |f_m|;
    a zero scale becomes 1."""
    N = xi.shape[0]
    L = float(np.max(np.linalg.norm(xi[:, :3], axis=1)))
    V = float(np.max(np.linalg.norm(np.asarray(b[:3 * N]).reshape(N, 3), axis=1)))
    F = float(np.sqrt(np.mean(np.sum(np.asarray(f).reshape(N, 3) ** 2, axis=1))))
    return np.array([L if L > 0 else 1.0, V if V > 0 else 1.0, F if F > 0 else 1.0])


def features(xi, xidot, W, n_off, kind, B, U_pres, Om_pres, vprev, scl) -> np.ndarray:
    """Feature rows (N x 17) of every force point, body by body:
    xi/L, xidot/V, the position s in the body's point order, W_m over the
    body's mean W, the one-hot kind, and B^T U / V, B^T Omega L / V with
    (U, Omega) from vprev for a free body (zero without vprev), prescribed for
    a prescribed body, zero for a static body."""
    L, V = float(scl[0]), float(scl[1])
    N = int(n_off[-1])
    X = np.zeros((N, IN))
    f = 0
    for b in range(len(kind)):
        lo, hi = int(n_off[b]), int(n_off[b + 1])
        Bb = np.asarray(B[b], np.float64).reshape(3, 3)
        if kind[b] == PRESCRIBED:
            U, Om = np.asarray(U_pres[b], float), np.asarray(Om_pres[b], float)
        elif kind[b] == FREE and vprev is not None:
            U, Om = np.asarray(vprev[6 * f:6 * f + 3]), np.asarray(vprev[6 * f + 3:6 * f + 6])
        else:
            U, Om = np.zeros(3), np.zeros(3)
        if kind[b] == FREE:
            f += 1
        cnt = hi - lo
        if cnt == 0:
            continue
        mean_w = float(np.mean(W[lo:hi]))
        X[lo:hi, 0:3] = xi[lo:hi, :3] / L
        X[lo:hi, 3:6] = xidot[lo:hi, :3] / V
        X[lo:hi, 6] = np.arange(cnt) / max(1, cnt - 1)
        X[lo:hi, 7] = W[lo:hi] / mean_w if mean_w > 0 else 0.0
        X[lo:hi, 8 + int(kind[b])] = 1.0
        X[lo:hi, 11:14] = (Bb.T @ U) / V
        X[lo:hi, 14:17] = (Bb.T @ Om) * L / V
    return X


def targets(f: np.ndarray, n_off, B, F: float) -> np.ndarray:
    """Body-frame force densities B^T f_m / F (N x 3)."""
    N = int(n_off[-1])
    f = np.asarray(f, np.float64).reshape(N, 3)
    T = np.zeros((N, 3))
    for b in range(len(n_off) - 1):
        lo, hi = int(n_off[b]), int(n_off[b + 1])
        T[lo:hi] = f[lo:hi] @ np.asarray(B[b], np.float64).reshape(3, 3) / F
    return T


def start_vector(Y: np.ndarray, n_off, B, F: float, vprev, nfree: int) -> np.ndarray:
    """Start vector of the refinement from a prediction: f_m = F B y_m for
    every force point, then the free bodies' (U, Omega) from vprev (zero if
    None)."""
    N = int(n_off[-1])
    x = np.zeros(3 * N + 6 * nfree)
    for b in range(len(n_off) - 1):
        lo, hi = int(n_off[b]), int(n_off[b + 1])
        x[3 * lo:3 * hi] = (F * (np.asarray(Y[lo:hi], np.float64)
                                 @ np.asarray(B[b], np.float64).reshape(3, 3).T)).ravel()
    if vprev is not None and nfree:
        x[3 * N:] = vprev
    return x

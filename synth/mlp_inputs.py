"""Seeded inputs of the learned starting guess: initial MLP parameters and
random feature / target batches for the parity tests.

Random numbers only; the MLP's arithmetic lives on each side of the parity
tests separately.  Draws use numpy's PCG64 generator (O'Neill 2014) seeded
with the given integer, which gives the same stream on every platform.
"""

from __future__ import annotations

import numpy as np

IN, HID, OUT = 17, 64, 3
NPARAM = HID * IN + HID + HID * HID + HID + OUT * HID + OUT


def mlp_init(seed: int = 0) -> np.ndarray:
    """Parameters in the interface layout (W1 [64][17], b1, W2 [64][64], b2,
    W3 [3][64], b3), float32: weights uniform in +-sqrt(6 / (fan_in +
    fan_out)) (Glorot & Bengio 2010), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def glorot(fan_out, fan_in):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size=(fan_out, fan_in))

    parts = [glorot(HID, IN).ravel(), np.zeros(HID), glorot(HID, HID).ravel(), np.zeros(HID),
             glorot(OUT, HID).ravel(), np.zeros(OUT)]
    return np.concatenate(parts).astype(np.float32)


def mlp_batch(seed: int, npts: int, scale: float = 1.0):
    """Random features X (npts, 17) uniform in [-scale, scale] and targets
    T (npts, 3) uniform in [-1, 1], float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(-scale, scale, size=(npts, IN)).astype(np.float32)
    T = rng.uniform(-1.0, 1.0, size=(npts, OUT)).astype(np.float32)
    return X, T


def mlp_perturb(seed: int, params: np.ndarray, size: float) -> np.ndarray:
    """params plus uniform noise in [-size, size] (float32): non-zero biases
    for tests that need every parameter to matter."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (params + rng.uniform(-size, size, size=params.shape)).astype(np.float32)

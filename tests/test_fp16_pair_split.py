"""The scaled FP16-pair products of the two-level factorisation's update, as
a numerical claim checked in numpy (no GPU): each row of A and each row of B
(K-major) is scaled by the power of two 2^e that puts its largest magnitude in
[2^14, 2^15), split into hi = fp16(x) and lo = fp16(x - hi), and the product
hi hi + hi lo + lo hi, accumulated in FP32 and unscaled by 2^-(e_i + f_j),
reproduces A B^T to about 2^-21 of |A| |B|^T -- the accuracy of the split-TF32
form it replaces -- even where rows differ by many orders of magnitude, where
unscaled FP16 would overflow or flush to zero."""

import numpy as np


def _scale_exp(rowmax):
    e = np.zeros_like(rowmax, dtype=np.int64)
    nz = rowmax > 0
    e[nz] = np.clip(14 - np.floor(np.log2(rowmax[nz])).astype(np.int64), -100, 100)
    return e


def _split(X):
    e = _scale_exp(np.max(np.abs(X), axis=1))
    Xs = (X * np.exp2(e)[:, None]).astype(np.float32)
    hi = Xs.astype(np.float16)
    lo = (Xs - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float64), lo.astype(np.float64), e


def _product(A, B):
    ah, al, ea = _split(A)
    bh, bl, eb = _split(B)
    acc = (ah @ bh.T) + (ah @ bl.T) + (al @ bh.T)  # exact products, FP64 sums
    acc = acc.astype(np.float32).astype(np.float64)  # one FP32 rounding of the sum
    return acc * np.exp2(-ea)[:, None] * np.exp2(-eb)[None, :]


def test_scaled_fp16_pairs_reproduce_the_product():
    rng = np.random.default_rng(0)
    m, k, n = 64, 256, 48
    A = (rng.normal(size=(m, k)) * 10.0 ** rng.uniform(-20, 20, size=(m, 1))).astype(np.float32)
    B = (rng.normal(size=(n, k)) * 10.0 ** rng.uniform(-20, 20, size=(n, 1))).astype(np.float32)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = A64 @ B64.T
    bound = np.abs(A64) @ np.abs(B64).T
    err = np.abs(_product(A64, B64) - ref)
    assert np.all(err <= 2.0 ** -20 * bound)
    # rows this far apart are out of FP16's range unscaled
    assert np.max(np.abs(A)) > 65504 or np.min(np.max(np.abs(A), axis=1)) < 2.0 ** -24


def test_zero_rows_and_ranges_inside_a_row():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(8, 256))
    A[3] = 0.0
    A[5, :128] *= 1e-6  # a row whose entries span six orders of magnitude
    B = rng.normal(size=(16, 256))
    err = np.abs(_product(A, B) - A @ B.T)
    assert np.all(err[3] == 0.0)
    assert np.all(err <= 2.0 ** -20 * (np.abs(A) @ np.abs(B).T))

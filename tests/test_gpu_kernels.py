"""Kernel-level parity: the rank-64 update of the Gauss-Jordan inverse on the
tensor cores (tcgen05, split-precision 3xTF32, FP32 accumulation) and on the
CUDA cores (FP32), element by element against an FP64 product on the host.

Both keep FP32-level accuracy: the split-precision products are within about
2^-21 of exact and FP32 accumulation of 64 terms adds at most ~64 * 2^-24, so
every entry is within 1e-5 of sum_c |C_ic R_jc|.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


@pytest.fixture(scope="module")
def ctx(N):
    # any context provides the stream and the status word
    return N.Context([0, 1], [0, 1], [N.PRESCRIBED], eps=0.1)


def _case(n, seed):
    rng = np.random.default_rng(seed)
    lda = ((n + 31) // 32) * 32
    M = rng.normal(size=(n, lda)).astype(np.float32)  # Mt[j, i] = M[i, j]
    C = rng.normal(size=(n, 64)).astype(np.float32)
    R = rng.normal(size=(n, 64)).astype(np.float32)
    return M, C, R


def _reference(M, C, R):
    n = C.shape[0]
    upd = C.astype(np.float64) @ R.astype(np.float64).T  # upd[i, j]
    ref = M.astype(np.float64).copy()
    ref[:, :n] -= upd.T  # Mt[j, i] -= upd[i, j]
    bound = np.abs(C).astype(np.float64) @ np.abs(R).astype(np.float64).T
    return ref, bound.T


@pytest.mark.parametrize("prec,rel", [("fp32", 1e-5), ("tf32", 1e-5)])
@pytest.mark.parametrize("n", [64, 300, 1000])
def test_rank64_update_matches_fp64_product(N, ctx, prec, rel, n):
    M, C, R = _case(n, 11 + n)
    Mt = torch.from_numpy(M).cuda()
    ctx.rank64_update(Mt, torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda(), prec)
    torch.cuda.synchronize()
    got = Mt.cpu().numpy().astype(np.float64)
    ref, bound = _reference(M, C, R)
    err = np.abs(got[:, :n] - ref[:, :n])
    assert np.all(err <= rel * bound + 1e-6 * np.abs(ref[:, :n])), err.max()
    # rows between n and lda (padding) are never written
    assert np.array_equal(got[:, n:], M[:, n:].astype(np.float64))


def test_tensor_core_update_is_deterministic(N, ctx):
    n = 700
    M, C, R = _case(n, 5)
    Cd, Rd = torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda()
    first = None
    for _ in range(20):
        Mt = torch.from_numpy(M).cuda()
        ctx.rank64_update(Mt, Cd, Rd, "tf32")
        out = Mt.cpu().numpy()
        if first is None:
            first = out
        assert np.array_equal(out, first)


def test_tensor_core_update_is_far_more_accurate_than_one_tf32_pass(N, ctx):
    # one TF32 pass would leave errors near 2^-11; the split form must be far below
    n = 256
    M, C, R = _case(n, 9)
    Mt = torch.from_numpy(M).cuda()
    ctx.rank64_update(Mt, torch.from_numpy(C).cuda(), torch.from_numpy(R).cuda(), "tf32")
    got = Mt.cpu().numpy().astype(np.float64)
    ref, bound = _reference(M, C, R)
    assert np.max(np.abs(got[:, :n] - ref[:, :n]) / bound[:, :n]) < 2.0 ** -16

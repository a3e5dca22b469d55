"""nrs_nearest_build_static, the allocation-free variant of nrs_nearest_build.

It serves callers that cannot allocate device memory where they need the
nearest-neighbour map (a memory pool or arena they do not own, a loop where
cudaMalloc would synchronise the device, a process that reserved all device
memory up front).  Its scratch is a fixed file-scope device array shared by
every call.  These tests call it through the C ABI twice in a row, on two
problems of different sizes (so stale scratch from the first call would show
in the second), and require the same bit-exact integer outputs as the
context-based entry point.  This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

from synth import geometry as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


def _reference(N, pr, sh):
    ctx = N.Context.from_problem(pr)
    xi, Xiw, _ = N.shapes_to_device(sh)
    nn, seg_ptr, perm = ctx.nearest_build(xi, Xiw)
    torch.cuda.synchronize()
    return xi, Xiw, nn.cpu().numpy(), seg_ptr.cpu().numpy(), perm.cpu().numpy()


def test_static_variant_matches_context_entry_point_on_two_calls_in_a_row(N):
    problems = [
        g.sperm_channel_config(count=2, n_head=40, q_head=400, n_flag=60, q_flag=600,
                               wall_f=(20, 6, 3), wall_q=(60, 18, 9)),
        g.swimmer_config(),
    ]
    for pr in problems:
        sh = g.pack_shapes(pr, 0.07)
        xi, Xiw, nn_ref, sp_ref, perm_ref = _reference(N, pr, sh)
        nn, seg_ptr, perm = N.nearest_build_static(xi, Xiw, sh["n_off"], sh["q_off"])
        torch.cuda.synchronize()
        assert np.array_equal(nn.cpu().numpy(), nn_ref)
        assert np.array_equal(seg_ptr.cpu().numpy(), sp_ref)
        assert np.array_equal(perm.cpu().numpy(), perm_ref)


def test_static_variant_rejects_sizes_beyond_its_scratch(N):
    from paper_2001_06468_gb300.nrs import NRS_STATIC_LIMITS
    too_many = NRS_STATIC_LIMITS["N"] + 1
    x = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    Xw = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(N.NrsError) as ei:
        N.nearest_build_static(x, Xw, [0, too_many], [0, 1],
                               nn=torch.empty(1, dtype=torch.int32, device="cuda"),
                               seg_ptr=torch.empty(1, dtype=torch.int32, device="cuda"),
                               perm=torch.empty(1, dtype=torch.int32, device="cuda"))
    assert ei.value.status == N.NRS_EINVAL

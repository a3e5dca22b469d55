"""nrs_nearest_build_static, the allocation-free variant of nrs_nearest_build.

It serves callers that cannot allocate device memory where they need the
nearest-neighbour map (a memory pool or arena they do not own, a loop where
cudaMalloc would synchronise the device, a process that reserved all device
memory up front).  Its scratch is a fixed file-scope device array shared by
every call.  These tests call it through the C ABI twice in a row, on two
problems of different sizes (so stale scratch from the first call would show
in the second), and require the same bit-exact integer outputs as the
context-based entry point and the oracle, in per-body and global mode and at
the largest size it accepts; a non-finite coordinate is reported through the
caller's status word.  This file is collected last on purpose.
"""

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


def test_static_variant_matches_the_oracle_in_global_mode_and_at_its_largest_size(N):
    # global mode (every force point a candidate, lab frame) against the
    # context entry point and the oracle; then N = NRS_STATIC_MAX_N force points
    from paper_2001_06468_gb300.nrs import NRS_STATIC_LIMITS
    pr = g.sperm_channel_config(count=2, n_head=40, q_head=400, n_flag=60, q_flag=600,
                                wall_f=(20, 6, 3), wall_q=(60, 18, 9))
    pr.nn_global = True
    sh = g.pack_shapes(pr, 0.3)
    Y = g.initial_state(pr)
    x_lab, Xw_lab = O.lab_frame(sh, Y)
    xd, Xd = torch.from_numpy(x_lab).cuda(), torch.from_numpy(Xw_lab).cuda()
    nn, seg_ptr, perm = N.nearest_build_static(xd, Xd, sh["n_off"], sh["q_off"], global_=True)
    ctx = N.Context.from_problem(pr)
    nn_c, sp_c, pm_c = ctx.nearest_build(xd, Xd)
    nn_or = O.nearest(x_lab, Xw_lab, sh["n_off"], sh["q_off"], global_=True)
    sp_or, pm_or = O.segments(nn_or, pr.N)
    for got, ctx_v, ref in ((nn, nn_c, nn_or), (seg_ptr, sp_c, sp_or), (perm, pm_c, pm_or)):
        assert np.array_equal(got.cpu().numpy(), ref)
        assert np.array_equal(got.cpu().numpy(), ctx_v.cpu().numpy())
    # the largest accepted problem: N = NRS_STATIC_MAX_N force points on a
    # random cloud, 3000 quadrature points, one body
    Nmax = NRS_STATIC_LIMITS["N"]
    rng = np.random.default_rng(3)
    x = np.zeros((Nmax, 4))
    x[:, :3] = rng.uniform(-1.0, 1.0, size=(Nmax, 3))
    Xw = np.zeros((3000, 4))
    Xw[:, :3] = rng.uniform(-1.0, 1.0, size=(3000, 3))
    Xw[:, 3] = 1.0
    n_off, q_off = np.array([0, Nmax]), np.array([0, 3000])
    nn, seg_ptr, perm = N.nearest_build_static(torch.from_numpy(x).cuda(),
                                               torch.from_numpy(Xw).cuda(), n_off, q_off)
    nn_or = O.nearest(x, Xw, n_off, q_off)
    sp_or, pm_or = O.segments(nn_or, Nmax)
    assert np.array_equal(nn.cpu().numpy(), nn_or)
    assert np.array_equal(seg_ptr.cpu().numpy(), sp_or)
    assert np.array_equal(perm.cpu().numpy(), pm_or)


def test_static_variant_reports_non_finite_input(N):
    # a NaN quadrature coordinate: that point gets nn < 0 and no segment, and
    # the caller's status word says so (the wrapper raises NRS_ENONFINITE);
    # the next call with finite input clears it
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    sh = g.pack_shapes(pr, 0.0)
    Xiw = sh["Xw"].copy()
    Xiw[17, 1] = np.nan
    xi = torch.from_numpy(sh["x"]).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    nn, seg_ptr, perm = N.nearest_build_static(xi, torch.from_numpy(Xiw).cuda(), sh["n_off"],
                                               sh["q_off"], status=status, check=False)
    torch.cuda.synchronize()
    assert int(status.item()) == 4
    assert int(nn[17].item()) < 0
    assert int(seg_ptr[-1].item()) == pr.Q - 1
    with pytest.raises(N.NrsError) as ei:
        N.nearest_build_static(xi, torch.from_numpy(Xiw).cuda(), sh["n_off"], sh["q_off"])
    assert ei.value.status == N.NRS_ENONFINITE
    N.nearest_build_static(xi, torch.from_numpy(sh["Xw"]).cuda(), sh["n_off"], sh["q_off"],
                           status=status)
    assert int(status.item()) == 0


def test_static_variant_rejects_sizes_beyond_its_scratch(N):
    # the library's own check, through the C ABI directly: N above the limit
    # is refused before anything is enqueued (nothing is read or written)
    import ctypes
    from paper_2001_06468_gb300 import nrs
    too_many = nrs.NRS_STATIC_LIMITS["N"] + 1
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    ibuf = torch.zeros(4, dtype=torch.int32, device="cuda")
    n_off = np.array([0, too_many], dtype=np.int64)
    q_off = np.array([0, 1], dtype=np.int64)
    p = ctypes.c_void_p
    rc = nrs._lib.nrs_nearest_build_static(
        p(buf.data_ptr()), p(buf.data_ptr()), 1, n_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        q_off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 0, p(ibuf.data_ptr()),
        p(ibuf.data_ptr()), p(ibuf.data_ptr()), None, None)
    assert rc == N.NRS_EINVAL
    # and the wrapper refuses tensors that do not match the offsets
    with pytest.raises(ValueError):
        N.nearest_build_static(buf.reshape(1, 4), buf.reshape(1, 4), [0, 2], [0, 1])

"""nrs_get_trace: the timed spans of a factorisation as a timeline.

The separate-kernel factorisation puts the chain of diagonal-block inverses on
a second stream and the finish on a third; the trace must show one inverse and
one update per 64-column block, every span with begin <= end, the inverses one
after the other, and the same totals as nrs_get_timing.
"""

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


def test_trace_of_a_factorisation(N):
    pr = g.swimmer_config()
    sh = g.pack_shapes(pr, 0.25)
    ctx = N.Context.from_problem(pr, factor_prec="tf32")
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = N.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    ctx.assemble(x, Xw, want_matrix=False)
    ctx.set_timing(True)
    assert ctx.factor("tf32") == 0
    tr = ctx.get_trace()
    totals, _ = ctx.get_timing()
    nblk = -(-pr.n // 64)
    phases = [p for p, _, _ in tr]
    assert phases.count("lu_diag") == nblk
    assert phases.count("lu_update") == nblk
    assert all(0.0 <= t0 <= t1 for _, t0, t1 in tr)
    assert min(t0 for _, t0, _ in tr) == 0.0
    diag = [(t0, t1) for p, t0, t1 in tr if p == "lu_diag"]
    # each inverse needs the previous one's D^{-1}: they run one after the other
    assert all(diag[i][1] <= diag[i + 1][0] + 1e-3 for i in range(nblk - 1))
    for p in ("lu_diag", "lu_update", "lu_panel"):
        s = sum(t1 - t0 for q, t0, t1 in tr if q == p)
        assert s == pytest.approx(totals[p][0], rel=1e-4, abs=1e-4)
        assert totals[p][1] == phases.count(p)
    ctx.close()

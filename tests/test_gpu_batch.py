"""The recorded step (CUDA graph) and the batch of independent problems.

* Graph mode replays exactly the kernels of the eager step: bit-identical
  results over consecutive steps (the shape buffers are reused, their
  contents rewritten each step).
* A batch of uneven problems (ventral-node-like: rotating cilia, a static
  floor, free spheres, at reduced sizes) gives each problem the solution the
  FP64 oracle gives, to the solver's 1e-10, over consecutive steps; and the
  same as stepping each problem on its own context to 1e-12 (the solve kernel
  may run with a different CTA count, which reorders its sums).
* The autotuner restores the state it started from, and its cache is reused.
"""

import numpy as np
import pytest
import torch

import oracle as O
from synth import geometry as g

pytestmark = pytest.mark.gpu

TOL_SOL = 1e-10


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_06468_gb300 import nrs
    return nrs


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def small_node(i):
    return g.node_config(i, cilia=(2, 4), floor=(60, 120), n_rod=8, q_rod=48, n_sphere=2,
                         q_sphere=6, n_spheres=2)


class Buffers:
    """Fixed device shape buffers whose contents are rewritten every step."""

    def __init__(self, N, pr):
        self.N, self.pr = N, pr
        sh = g.pack_shapes(pr, 0.0)
        self.b0 = tuple(torch.empty_like(torch.from_numpy(sh[k]), device="cuda")
                        for k in ("x", "Xw", "xidot"))
        self.bh = tuple(torch.empty_like(t) for t in self.b0)

    def load(self, t, dt):
        for buf, tt in ((self.b0, t), (self.bh, t + 0.5 * dt)):
            for dst, src in zip(buf, self.N.shapes_to_device(g.pack_shapes(self.pr, tt))):
                dst.copy_(src)
        return self.b0, self.bh


@pytest.mark.parametrize("warm", [False, True])
def test_graph_mode_replays_the_eager_step_bit_for_bit(N, warm):
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    Y = g.initial_state(pr)
    out = {}
    for graph in (False, True):
        ctx = N.Context.from_problem(pr, factor_prec="tf32", graph=graph, warm_start=warm)
        ctx.set_state(Y["x0"], Y["B"])
        bufs = Buffers(N, pr)
        sols = []
        for k in range(4):
            b0, bh = bufs.load(k * 0.01, 0.01)
            sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
            rep = ctx.step(N.Context.shapes(*b0), N.Context.shapes(*bh), 0.01, sol=sol)
            assert rep["status"] == 0
            sols.append(sol.cpu().numpy())
        out[graph] = (np.array(sols), ctx.get_state())
    assert np.array_equal(out[False][0], out[True][0])
    assert np.array_equal(out[False][1]["B"], out[True][1]["B"])
    assert np.array_equal(out[False][1]["x0"], out[True][1]["x0"])


def test_graph_mode_rejects_unsupported_options(N):
    pr = g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)
    with pytest.raises(N.NrsError):
        N.Context.from_problem(pr, factor_prec="fp64", graph=True)
    with pytest.raises(N.NrsError):
        N.Context.from_problem(pr, factor_prec="tf32", graph=True, reuse_factor=True)


def _batch_problems():
    return [small_node(i) for i in range(4)] + [
        g.swimmer_config(ns_f=20, nth_f=4, ns_q=100, nth_q=8)]


def test_batch_matches_oracle_and_single_contexts(N):
    probs = _batch_problems()
    dt, steps = 0.01, 3
    batch = N.Batch(probs, factor_prec="tf32")
    Ys = [g.initial_state(pr) for pr in probs]
    for c, Y in zip(batch.contexts, Ys):
        c.set_state(Y["x0"], Y["B"])
    bufs = [Buffers(N, pr) for pr in probs]
    sols = [torch.empty(2 * pr.n, dtype=torch.float64, device="cuda") for pr in probs]
    got = []
    for k in range(steps):
        pairs = [b.load(k * dt, dt) for b in bufs]
        reps = batch.step(pairs, dt, sols=sols, report=True)
        assert all(r["stages"][s]["status"] == 0 for r in reps for s in (0, 1))
        got.append([s.cpu().numpy() for s in sols])
    assert batch.info()["graph_kernels"] > 0
    # each problem alone on an eager context
    for i, pr in enumerate(probs):
        ctx = N.Context.from_problem(pr, factor_prec="tf32")
        ctx.set_state(Ys[i]["x0"], Ys[i]["B"])
        Yo = Ys[i]
        for k in range(steps):
            d0 = N.shapes_to_device(g.pack_shapes(pr, k * dt))
            dh = N.shapes_to_device(g.pack_shapes(pr, k * dt + 0.5 * dt))
            sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
            ctx.step(N.Context.shapes(*d0), N.Context.shapes(*dh), dt, sol=sol)
            assert _rel(got[k][i], sol.cpu().numpy()) <= 1e-12
            if i in (0, 4):  # the oracle on two of them (a node problem, the swimmer)
                Yo, stg = O.rk2_step(pr, Yo, k * dt, dt, return_stages=True)
                assert _rel(got[k][i][:pr.n], stg["sol1"]) <= TOL_SOL
                assert _rel(got[k][i][pr.n:], stg["sol2"]) <= TOL_SOL
        st_b, st_s = batch.contexts[i].get_state(), ctx.get_state()
        assert np.allclose(st_b["B"], st_s["B"], rtol=0, atol=1e-13)
    batch.close()


def test_batch_tune_restores_state_and_uses_its_cache(N, tmp_path):
    probs = _batch_problems()
    dt = 0.01
    batch = N.Batch(probs, factor_prec="tf32")
    for c, pr in zip(batch.contexts, probs):
        Y = g.initial_state(pr)
        c.set_state(Y["x0"], Y["B"])
    bufs = [Buffers(N, pr) for pr in probs]
    batch.step([b.load(0.0, dt) for b in bufs], dt)
    before = [c.get_state() for c in batch.contexts]
    pairs = [b.load(dt, dt) for b in bufs]
    cache = str(tmp_path / "tune.txt")
    res = batch.tune(pairs, dt, cache_path=cache)
    assert res["chains"] >= 1 and res["grid"] >= 1 and res["ms"] > 0
    after = [c.get_state() for c in batch.contexts]
    for a, b in zip(before, after):
        assert np.array_equal(a["B"], b["B"]) and np.array_equal(a["x0"], b["x0"])
    res2 = batch.tune(pairs, dt, cache_path=cache)
    assert res2["ms"] == -1.0 and (res2["chains"], res2["grid"]) == (res["chains"], res["grid"])
    with open(cache) as f:
        assert len(f.read().strip().splitlines()) == 1
    with pytest.raises(N.NrsError):
        batch.config(0, 10)
    with pytest.raises(N.NrsError):
        batch.config(len(probs) + 1, 10)
    batch.close()


def test_full_size_node_problems_in_a_batch_match_the_oracle(N):
    # the two smallest full-size ventral-node problems of the 128 (n = 5322
    # and 5466) and a reduced one, stepped twice as a batch (the second step
    # replayed from the recorded graph), against the oracle's trajectory
    probs = [g.node_config(4), g.node_config(106), small_node(0)]
    assert (probs[0].n, probs[1].n) == (5322, 5466)
    dt = 0.01
    batch = N.Batch(probs, factor_prec="tf32")
    Ys = [g.initial_state(pr) for pr in probs]
    for c, Y in zip(batch.contexts, Ys):
        c.set_state(Y["x0"], Y["B"])
    bufs = [Buffers(N, pr) for pr in probs]
    sols = [torch.empty(2 * pr.n, dtype=torch.float64, device="cuda") for pr in probs]
    Yo = list(Ys)
    for k in range(2):
        reps = batch.step([b.load(k * dt, dt) for b in bufs], dt, sols=sols, report=True)
        assert all(r["stages"][s]["status"] == 0 for r in reps for s in (0, 1))
        for i in range(2):
            pr = probs[i]
            Yo[i], stg = O.rk2_step(pr, Yo[i], k * dt, dt, solver=O.solve_lapack,
                                    return_stages=True)
            s = sols[i].cpu().numpy()
            assert _rel(s[:pr.n], stg["sol1"]) <= TOL_SOL, (i, k)
            assert _rel(s[pr.n:], stg["sol2"]) <= TOL_SOL, (i, k)
    assert batch.info()["graph_kernels"] > 0
    batch.close()

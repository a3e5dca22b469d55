"""Write the oracle's solutions of the first explicit-midpoint step of the
full-size workloads -- the eight-cell channel (9200 force / 92000 quadrature
points, n = 27648) and the four interacting swimmers (8000 / 80000,
n = 24024) -- to ``<workload>_step0.npz``, for the full-size GPU parity
test.

Only ``oracle/`` computes anything here; ``synth`` supplies the seeded
inputs, whose SHA-1 is stored beside the solutions so that the test can
check it is comparing against the same inputs (the test recomputes the
oracle when the digest differs).  The oracle's system (Sec. 4 steps 1-2) is
solved by LAPACK's LU refined with a double-double residual to working
accuracy (oracle.solve_lapack).

    python tests/golden/make_fullsize_golden.py [sperm_channel] [swimmers4]
                                        # about two minutes each on 8 cores
"""

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from synth import geometry as g  # noqa: E402



def input_digest(pr, dt):
    """SHA-1 of every input of the first step: body-frame shapes at t = 0 and
    t = dt/2 and the initial state."""
    m = hashlib.sha1()
    for t in (0.0, 0.5 * dt):
        d = g.pack_shapes(pr, t)
        for k in ("x", "Xw", "xidot"):
            m.update(np.ascontiguousarray(d[k], dtype=np.float64).tobytes())
    Y = g.initial_state(pr)
    m.update(np.ascontiguousarray(Y["x0"], dtype=np.float64).tobytes())
    m.update(np.ascontiguousarray(Y["B"], dtype=np.float64).tobytes())
    return m.hexdigest()


def oracle_first_step(pr):
    """(Y after the step, stage solutions) of the oracle's first RK2 step."""
    Y0 = g.initial_state(pr)
    return O.rk2_step(pr, Y0, 0.0, pr.dt, solver=O.solve_lapack, return_stages=True)


def main(names):
    for name in names:
        pr = g.workload(name)
        out = os.path.join(HERE, f"{name}_step0.npz")
        t0 = time.time()
        Yn, st = oracle_first_step(pr)
        np.savez(out, digest=np.array(input_digest(pr, pr.dt)), sol1=st["sol1"],
                 sol2=st["sol2"], x0=Yn["x0"], B=Yn["B"], n=np.array(pr.n))
        print(f"wrote {out} (n = {pr.n}) in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1:] or ["sperm_channel", "swimmers4"])

"""Checks of the seeded input generators (inputs only, no method arithmetic)."""

import math

import numpy as np

from synth import geometry as g


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 1234567 (published test vector
    # of the reference C implementation by Vigna)
    rng = g.SplitMix64(1234567)
    got = [rng.next_u64() for _ in range(3)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_cube_sphere_counts_and_weights():
    for n in (4, 16):
        p, w = g.cube_sphere_vertices(n)
        assert len(p) == 6 * n * n + 2
        assert np.allclose(np.linalg.norm(p, axis=1), 1.0, rtol=1e-15)
        assert abs(w.sum() - 4 * math.pi) < 1e-12
        assert np.all(w > 0)
    p, w = g.cube_sphere_cells(12)
    assert len(p) == 864 and abs(w.sum() - 4 * math.pi) < 1e-12


def test_coarse_cube_sphere_vertices_are_quadrature_points_bit_for_bit():
    xi, _ = g.cube_sphere_vertices(4)
    Xi, _ = g.cube_sphere_vertices(16)
    rows = {tuple(r) for r in Xi}
    assert all(tuple(r) in rows for r in xi)


def test_tube_velocity_is_the_time_derivative_of_position():
    h = 1e-5
    p0, _, v = g.tube_shape(0.3, 12, 6, phase=0.7)
    pp, _, _ = g.tube_shape(0.3 + h, 12, 6, phase=0.7)
    pm, _, _ = g.tube_shape(0.3 - h, 12, 6, phase=0.7)
    assert np.abs((pp - pm) / (2 * h) - v).max() < 1e-8


def test_tube_weights_converge_to_the_surface_area():
    areas = [g.tube_shape(0.0, ns, nth)[1].sum() for ns, nth in ((100, 20), (400, 40), (1600, 80))]
    assert abs(areas[1] - areas[2]) < abs(areas[0] - areas[2])
    assert abs(areas[1] / areas[2] - 1) < 2e-3


def test_workload_sizes():
    assert (g.sphere_config().N, g.sphere_config().Q, g.sphere_config().n) == (98, 1538, 294)
    sw = g.swimmer_config()
    assert (sw.N, sw.Q, sw.n) == (800, 8000, 2406)
    sw4 = g.swimmers_config()
    assert (sw4.N, sw4.Q, sw4.n) == (8000, 80000, 24024)
    sc = g.sperm_channel_config()
    assert (sc.N, sc.Q, sc.n) == (9200, 92000, 27648)


def test_swimmers_are_seeded_and_separated():
    a = g.swimmers_config()
    b = g.swimmers_config()
    assert all(np.array_equal(x.x0, y.x0) for x, y in zip(a.bodies, b.bodies))
    c = [bd.x0 for bd in a.bodies]
    assert min(np.linalg.norm(c[i] - c[j]) for i in range(4) for j in range(i)) >= 1.2


def test_pack_layout():
    pr = g.sperm_channel_config(count=2)
    sh = g.pack_shapes(pr, 0.1)
    assert sh["x"].shape == (pr.N, 4) and sh["Xw"].shape == (pr.Q, 4)
    assert list(sh["n_off"]) == [0, 6000, 6400, 6800]
    assert np.all(sh["Xw"][:, 3] > 0)

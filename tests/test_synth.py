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


def test_node_batch_sizes_and_structure():
    # n = 3 (40 c + N_f + 5 * 98) + 6 * 5 = 120 c + 3 N_f + 1500 for every problem
    for i in (0, 5, 77):
        pr = g.node_config(i)
        c = sum(1 for b in pr.bodies if b.name.startswith("cilium"))
        nf = pr.bodies[0].N
        assert 10 <= c <= 60 and 800 <= nf <= 2500
        assert pr.bodies[0].Q == 10 * nf and pr.n == 120 * c + 3 * nf + 1500
        assert [b.kind for b in pr.bodies].count(g.FREE) == 5
    # seeded: the same index gives the same problem, another index another one
    a, b, c2 = g.node_config(3), g.node_config(3), g.node_config(4)
    assert a.n == b.n and np.array_equal(a.bodies[1].x0, b.bodies[1].x0)
    assert (a.n, a.bodies[1].x0.tolist()) != (c2.n, c2.bodies[1].x0.tolist())


def test_node_cilia_rotate_on_their_cone():
    pr = g.node_config(2, cilia=(3, 3), floor=(100, 100), n_rod=8, q_rod=40)
    for b in pr.bodies[1:4]:
        a = -b.Omega / np.linalg.norm(b.Omega)       # cone axis (clockwise from above)
        d = b.B[:, 0]                                  # the rod, body x-axis, lab frame
        assert abs(np.linalg.norm(b.Omega) - 2 * np.pi) < 1e-12
        assert abs(np.dot(a, d) - np.cos(np.radians(30.0))) < 1e-12   # semi-angle 30 degrees
        tilt = np.degrees(np.arccos(a[2]))
        assert 30.0 - 1e-9 <= tilt <= 45.0 + 1e-9 and a[1] <= 0.0     # tilted towards -y
        assert np.allclose(b.B.T @ b.B, np.eye(3), atol=1e-14)
        assert b.x0[2] == 0.0 and np.hypot(*b.x0[:2]) <= 1.6 + 1e-12  # base on the floor disc


def test_vogel_disc_weights_sum_to_the_area():
    P, w = g.vogel_disc(1000, 2.0)
    assert abs(w.sum() - np.pi * 4.0) < 1e-12
    assert np.max(np.hypot(P[:, 0], P[:, 1])) < 2.0 and np.all(P[:, 2] == 0.0)

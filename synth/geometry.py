"""Body-frame geometries and prescribed kinematics of the synthetic workloads.

Every function here returns plain numpy arrays in float64.  Nothing in this
file evaluates the regularized stokeslet, searches for nearest neighbours,
assembles or solves anything: it only describes *where* the points are, how
much surface each quadrature point carries, and how fast each force point
moves in its body frame (the prescribed beat).

Workloads (sizes follow the method's use in Sec. 4 and Sec. 5 of the paper,
with synthetic bodies standing in for the cited beat patterns):

* ``sphere``        rigid unit sphere, force points = cube-sphere vertices with
                    4 cells per face edge (N=98), quadrature = 16 cells per edge
                    (Q=1538), prescribed translation U=(1,0,0), eps=0.01.
* ``sphere_cells``  the paper's Sec. 3 sphere example sizes: cube-sphere face
                    cell centres, N=864 (12 per edge), Q=3456 (24 per edge).
* ``swimmer``       one undulating slender tube, N=800, Q=8000, eps=0.005,
                    free (U, Omega unknown): 2406 unknowns.
* ``swimmers4``     four such tubes at 2000/20000 points each: 24024 unknowns.
* ``sperm_channel`` eight sperm-like swimmers (ellipsoid head + beating
                    flagellum) in a closed static box: 27648 unknowns.
* ``node``          one problem of the batch workload: 10-60 tilted cilia
                    rotating on cones over a static floor disc, plus five free
                    spheres (n = 120 c + 3 N_f + 1500, 5100-16200 unknowns);
                    ``node_batch(128)`` is the batch.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood 2014).

    state += 0x9E3779B97F4A7C15; z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
    return z ^ (z >> 31)          (all arithmetic mod 2**64)

    ``uniform()`` maps the top 53 bits to [0, 1): (z >> 11) * 2**-53.
    """

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


# --------------------------------------------------------------------------
# spherical-triangle area (Van Oosterom & Strackee 1983 solid-angle formula)
# --------------------------------------------------------------------------

def _solid_angle(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Solid angle of the spherical triangles with unit-vector corners a, b, c
    (rows).  tan(Omega/2) = |a.(b x c)| / (1 + a.b + a.c + b.c)."""
    num = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c)))
    den = 1.0 + np.einsum("ij,ij->i", a, b) + np.einsum("ij,ij->i", a, c) \
        + np.einsum("ij,ij->i", b, c)
    return 2.0 * np.arctan2(num, den)


def _cube_faces(n: int):
    """Yield (axis, side) for the 6 faces of the lattice cube {0..n}^3."""
    for axis in range(3):
        for side in (0, n):
            yield axis, side


def _lattice_point(axis: int, side: int, u: int, v: int) -> tuple:
    """Integer lattice point on face (axis, side) at in-face coordinates (u, v)."""
    p = [0, 0, 0]
    p[axis] = side
    others = [d for d in range(3) if d != axis]
    p[others[0]] = u
    p[others[1]] = v
    return tuple(p)


def _project(ijk: np.ndarray, n: int, a: float) -> np.ndarray:
    """Cube coordinate c = 2 i / n - 1, projected to the sphere p = a c / |c|."""
    c = 2.0 * ijk.astype(np.float64) / n - 1.0
    return a * c / np.sqrt((c * c).sum(axis=1))[:, None]


def cube_sphere_vertices(n: int, a: float = 1.0):
    """Cube-sphere vertices and their quarter-cell area weights.

    Points: integer lattice (i,j,k) in {0..n}^3 with at least one coordinate
    in {0, n}, in lexicographic order (6 n^2 + 2 points), projected radially
    onto the sphere of radius a.  Weight of a vertex: one quarter of the area
    of every projected face cell that has it as a corner, each cell split into
    two spherical triangles.  The weights sum to 4 pi a^2.
    """
    rng = np.arange(n + 1)
    I, J, K = np.meshgrid(rng, rng, rng, indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    onb = np.any((ijk == 0) | (ijk == n), axis=1)
    ijk = ijk[onb]
    index = {tuple(p): q for q, p in enumerate(map(tuple, ijk))}
    pts = _project(ijk, n, a)
    unit = pts / a
    w = np.zeros(len(ijk))
    for axis, side in _cube_faces(n):
        for u in range(n):
            for v in range(n):
                c00 = index[_lattice_point(axis, side, u, v)]
                c10 = index[_lattice_point(axis, side, u + 1, v)]
                c11 = index[_lattice_point(axis, side, u + 1, v + 1)]
                c01 = index[_lattice_point(axis, side, u, v + 1)]
                t1 = _solid_angle(unit[[c00]], unit[[c10]], unit[[c11]])[0]
                t2 = _solid_angle(unit[[c00]], unit[[c11]], unit[[c01]])[0]
                area = (t1 + t2) * a * a
                for c in (c00, c10, c11, c01):
                    w[c] += 0.25 * area
    return pts, w


def cube_sphere_cells(n: int, a: float = 1.0):
    """Cube-sphere face-cell centres (6 n^2 points) and projected cell areas.

    The centre of cell (u, v) of a face is the lattice point (u+1/2, v+1/2)
    projected radially; its weight is the area of the projected cell (two
    spherical triangles on the cell's corners).  Face order as in
    ``_cube_faces``, cells in (u, v) lexicographic order.
    """
    centres, w = [], []
    for axis, side in _cube_faces(n):
        others = [d for d in range(3) if d != axis]
        for u in range(n):
            for v in range(n):
                cc = np.zeros(3)
                cc[axis] = side
                cc[others[0]] = u + 0.5
                cc[others[1]] = v + 0.5
                c = 2.0 * cc / n - 1.0
                centres.append(a * c / math.sqrt((c * c).sum()))
                corners = np.array([_lattice_point(axis, side, u, v),
                                    _lattice_point(axis, side, u + 1, v),
                                    _lattice_point(axis, side, u + 1, v + 1),
                                    _lattice_point(axis, side, u, v + 1)])
                un = _project(corners, n, 1.0)
                t1 = _solid_angle(un[[0]], un[[1]], un[[2]])[0]
                t2 = _solid_angle(un[[0]], un[[2]], un[[3]])[0]
                w.append((t1 + t2) * a * a)
    return np.array(centres), np.array(w)


# --------------------------------------------------------------------------
# undulating slender tube (C. elegans-like body)
# --------------------------------------------------------------------------

def tube_shape(t: float, ns: int, nth: int, amp: float = 0.1, rad: float = 0.04,
               phase: float = 0.0):
    """Body-frame surface of a tube around the planar centreline
    c(s,t) = (s/2, amp s sin(2 pi (s - t) + phase), 0), s in [-1, 1], with
    radius r(s) = rad sqrt(1 - s^2), sampled at cell midpoints of an
    ns x nth (s, theta) grid (index i*nth + l).

    The cross-section circle lies in the plane spanned by the in-plane unit
    normal nu = (-g_s, 1/2, 0)/|c_s| and z.  Returns (points, weights,
    velocities): weights are |p_s x p_theta| ds dtheta, velocities the exact
    time derivative dp/dt at fixed (s, theta).  The body-frame origin is the
    centreline point s = 0 for every t.
    """
    ds = 2.0 / ns
    dth = 2.0 * math.pi / nth
    s = -1.0 + (np.arange(ns) + 0.5) * ds
    th = (np.arange(nth) + 0.5) * dth
    S, TH = np.meshgrid(s, th, indexing="ij")
    S = S.ravel()
    TH = TH.ravel()
    tp = 2.0 * math.pi
    phi = tp * (S - t) + phase
    sn, cs = np.sin(phi), np.cos(phi)
    g = amp * S * sn
    g_s = amp * sn + amp * S * tp * cs
    g_ss = 2.0 * amp * tp * cs - amp * S * tp * tp * sn
    g_t = -amp * S * tp * cs
    g_st = -amp * tp * cs + amp * S * tp * tp * sn
    zero = np.zeros_like(S)
    one = np.ones_like(S)
    c = np.stack([0.5 * S, g, zero], axis=1)
    c_s = np.stack([0.5 * one, g_s, zero], axis=1)
    c_t = np.stack([zero, g_t, zero], axis=1)
    L = np.sqrt(0.25 + g_s * g_s)
    m = np.stack([-g_s, 0.5 * one, zero], axis=1)
    nu = m / L[:, None]
    # L * L * L rather than L ** 3: numpy's power may round differently on
    # other machines, and the inputs must be the same bits everywhere
    L3 = L * L * L
    nu_s = np.stack([-g_ss, zero, zero], axis=1) / L[:, None] \
        - m * (g_s * g_ss / L3)[:, None]
    nu_t = np.stack([-g_st, zero, zero], axis=1) / L[:, None] \
        - m * (g_s * g_st / L3)[:, None]
    ez = np.stack([zero, zero, one], axis=1)
    r = rad * np.sqrt(1.0 - S * S)
    r_s = -rad * S / np.sqrt(1.0 - S * S)
    cth, sth = np.cos(TH)[:, None], np.sin(TH)[:, None]
    e = cth * nu + sth * ez
    p = c + r[:, None] * e
    p_s = c_s + r_s[:, None] * e + (r[:, None] * cth) * nu_s
    p_th = r[:, None] * (-sth * nu + cth * ez)
    p_t = c_t + (r[:, None] * cth) * nu_t
    w = np.linalg.norm(np.cross(p_s, p_th), axis=1) * ds * dth
    return p, w, p_t


def flagellum_line(t: float, n: int, k: float, phase: float, amp: float = 0.1,
                   x_start: float = -0.1, length: float = 1.0):
    """Body-frame flagellum of a sperm-like cell: a line of points leaving the
    head's rear at (x_start, 0, 0) along -x, projected length ``length``, with
    the planar wave y = amp s sin(k s - 2 pi t + phase) for the projected
    arclength s in [0, length] (the factor s keeps the junction at the head
    continuous).  Midpoints of n equal cells; weight = |dX/ds| ds.
    Returns (points, weights, velocities)."""
    ds = length / n
    s = (np.arange(n) + 0.5) * ds
    arg = k * s - 2.0 * math.pi * t + phase
    y = amp * s * np.sin(arg)
    y_s = amp * np.sin(arg) + amp * s * k * np.cos(arg)
    y_t = -2.0 * math.pi * amp * s * np.cos(arg)
    zero = np.zeros_like(s)
    p = np.stack([x_start - s, y, zero], axis=1)
    w = np.sqrt(1.0 + y_s * y_s) * ds
    v = np.stack([zero, y_t, zero], axis=1)
    return p, w, v


def ellipsoid_fibonacci(npts: int, a: float, b: float, c: float):
    """Fibonacci lattice on the unit sphere, z_i = 1 - (2i+1)/npts,
    azimuth i * pi (3 - sqrt 5), mapped to the ellipsoid (a p_x, b p_y, c p_z);
    area weight (4 pi / npts) sqrt(b^2 c^2 p_x^2 + a^2 c^2 p_y^2 + a^2 b^2 p_z^2)
    (the surface Jacobian of that map)."""
    i = np.arange(npts)
    z = 1.0 - (2.0 * i + 1.0) / npts
    r = np.sqrt(1.0 - z * z)
    ga = math.pi * (3.0 - math.sqrt(5.0))
    phi = i * ga
    p = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    pts = p * np.array([a, b, c])
    w = (4.0 * math.pi / npts) * np.sqrt(
        (b * c * p[:, 0]) ** 2 + (a * c * p[:, 1]) ** 2 + (a * b * p[:, 2]) ** 2)
    return pts, w


def box_cells(L: tuple, counts: tuple):
    """Face-cell centres and areas of the closed box [0,Lx]x[0,Ly]x[0,Lz];
    ``counts`` = cells along (x, y, z).  Faces in the order z=0, z=Lz, y=0,
    y=Ly, x=0, x=Lx; cells in lexicographic order of the two in-face axes."""
    pts, w = [], []
    for axis in (2, 1, 0):
        others = [d for d in range(3) if d != axis]
        nu_, nv_ = counts[others[0]], counts[others[1]]
        hu, hv = L[others[0]] / nu_, L[others[1]] / nv_
        for side in (0.0, L[axis]):
            U, V = np.meshgrid((np.arange(nu_) + 0.5) * hu, (np.arange(nv_) + 0.5) * hv,
                               indexing="ij")
            P = np.zeros((nu_ * nv_, 3))
            P[:, axis] = side
            P[:, others[0]] = U.ravel()
            P[:, others[1]] = V.ravel()
            pts.append(P)
            w.append(np.full(nu_ * nv_, hu * hv))
    return np.concatenate(pts), np.concatenate(w)


# --------------------------------------------------------------------------
# bodies and problems
# --------------------------------------------------------------------------

FREE, PRESCRIBED, STATIC = 0, 1, 2
KIND_NAMES = {FREE: "free", PRESCRIBED: "prescribed", STATIC: "static"}


@dataclass
class Body:
    """One body: body-frame clouds as a function of time plus its initial
    rigid-body state.  ``shape(t)`` returns (xi (N,3), Xi (Q,3), w (Q,),
    xidot (N,3)) in the body frame."""
    kind: int
    N: int
    Q: int
    shape: Callable[[float], tuple]
    rigid: bool
    x0: np.ndarray
    B: np.ndarray
    U: np.ndarray = field(default_factory=lambda: np.zeros(3))
    Omega: np.ndarray = field(default_factory=lambda: np.zeros(3))
    name: str = ""


@dataclass
class Problem:
    name: str
    bodies: List[Body]
    eps: float
    mu: float = 1.0
    dt: float = 0.01
    steps: int = 1
    nn_global: bool = False

    @property
    def N(self) -> int:
        return sum(b.N for b in self.bodies)

    @property
    def Q(self) -> int:
        return sum(b.Q for b in self.bodies)

    @property
    def n_free(self) -> int:
        return sum(1 for b in self.bodies if b.kind == FREE)

    @property
    def n(self) -> int:
        return 3 * self.N + 6 * self.n_free

    @property
    def pairs(self) -> int:
        return self.N * self.Q


def _rigid(points_xi, Xi, w):
    xidot = np.zeros_like(points_xi)

    def shape(t):
        return points_xi, Xi, w, xidot
    return shape


def sphere_config(n_force: int = 4, n_quad: int = 16, a: float = 1.0, eps: float = 0.01,
                  U=(1.0, 0.0, 0.0), Omega=(0.0, 0.0, 0.0), mu: float = 1.0) -> Problem:
    """Rigid sphere, cube-sphere vertex clouds, prescribed (U, Omega)."""
    xi, _ = cube_sphere_vertices(n_force, a)
    Xi, w = cube_sphere_vertices(n_quad, a)
    body = Body(PRESCRIBED, len(xi), len(Xi), _rigid(xi, Xi, w), True,
                np.zeros(3), np.eye(3), np.array(U, float), np.array(Omega, float), "sphere")
    return Problem("sphere", [body], eps, mu)


def sphere_cells_config(n_force: int = 12, n_quad: int = 24, a: float = 1.0,
                        eps: float = 0.01, U=(1.0, 0.0, 0.0), Omega=(0.0, 0.0, 0.0)) -> Problem:
    """Rigid sphere with cube-sphere face-cell-centre clouds (6 n^2 points)."""
    xi, _ = cube_sphere_cells(n_force, a)
    Xi, w = cube_sphere_cells(n_quad, a)
    body = Body(PRESCRIBED, len(xi), len(Xi), _rigid(xi, Xi, w), True,
                np.zeros(3), np.eye(3), np.array(U, float), np.array(Omega, float),
                "sphere_cells")
    return Problem("sphere_cells", [body], eps, 1.0)


def _tube_body(ns_f, nth_f, ns_q, nth_q, phase, x0, name):
    def shape(t):
        xi, _, xidot = tube_shape(t, ns_f, nth_f, phase=phase)
        Xi, w, _ = tube_shape(t, ns_q, nth_q, phase=phase)
        return xi, Xi, w, xidot
    return Body(FREE, ns_f * nth_f, ns_q * nth_q, shape, False,
                np.array(x0, float), np.eye(3), name=name)


def swimmer_config(ns_f: int = 80, nth_f: int = 10, ns_q: int = 400, nth_q: int = 20,
                   eps: float = 0.005) -> Problem:
    """Single free undulating tube (N = ns_f*nth_f, Q = ns_q*nth_q)."""
    body = _tube_body(ns_f, nth_f, ns_q, nth_q, 0.0, (0.0, 0.0, 0.0), "tube")
    return Problem("swimmer", [body], eps, 1.0, dt=0.01, steps=100)


def swimmers_config(count: int = 4, ns_f: int = 200, nth_f: int = 10, ns_q: int = 1000,
                    nth_q: int = 20, eps: float = 0.005, seed: int = 2,
                    box=(4.0, 4.0, 1.0), min_sep: float = 1.2) -> Problem:
    """``count`` free tubes; centres uniform in the box (x, y, z drawn in that
    order), redrawn while closer than ``min_sep`` to an earlier centre; then
    one phase in [0, 2 pi) per swimmer."""
    rng = SplitMix64(seed)
    centres: List[np.ndarray] = []
    while len(centres) < count:
        c = np.array([rng.uniform(0, box[0]), rng.uniform(0, box[1]), rng.uniform(0, box[2])])
        if all(np.linalg.norm(c - o) >= min_sep for o in centres):
            centres.append(c)
    phases = [rng.uniform(0.0, 2.0 * math.pi) for _ in range(count)]
    bodies = [_tube_body(ns_f, nth_f, ns_q, nth_q, phases[i], centres[i], f"tube{i}")
              for i in range(count)]
    return Problem("swimmers4", bodies, eps, 1.0, dt=0.01, steps=100)


def sperm_channel_config(count: int = 8, n_head: int = 150, q_head: int = 1500,
                         n_flag: int = 250, q_flag: int = 2500,
                         wall_f=(90, 21, 10), wall_q=(279, 70, 30),
                         eps: float = 0.005, seed: int = 3) -> Problem:
    """Closed static box [0,4]x[0,1]x[0,0.5] plus ``count`` free sperm-like
    cells (ellipsoid head 0.1 x 0.08 x 0.03 centred on the body origin,
    flagellum of projected length 1 towards -x).  Each cell draws, in order,
    wavenumber k in [2 pi, 4 pi], phase in [0, 2 pi), and a centre jitter
    (dx, dy) in [-0.05, 0.05]^2 around a 2 x 4 grid of lanes
    x in {1.6, 3.2}, y in {0.2, 0.4, 0.6, 0.8}, z = 0.25."""
    rng = SplitMix64(seed)
    wall_x, wall_w = box_cells((4.0, 1.0, 0.5), wall_f)
    wall_X, wall_wq = box_cells((4.0, 1.0, 0.5), wall_q)
    wall = Body(STATIC, len(wall_x), len(wall_X), _rigid(wall_x, wall_X, wall_wq), True,
                np.zeros(3), np.eye(3), name="channel")
    hx, _ = ellipsoid_fibonacci(n_head, 0.1, 0.08, 0.03)
    hX, hw = ellipsoid_fibonacci(q_head, 0.1, 0.08, 0.03)
    bodies = [wall]
    lanes = [(x, y) for x in (1.6, 3.2) for y in (0.2, 0.4, 0.6, 0.8)]
    for i in range(count):
        k = rng.uniform(2.0 * math.pi, 4.0 * math.pi)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        jx = rng.uniform(-0.05, 0.05)
        jy = rng.uniform(-0.05, 0.05)
        lx, ly = lanes[i % len(lanes)]

        def shape(t, k=k, ph=ph):
            fx, _, fv = flagellum_line(t, n_flag, k, ph)
            fX, fw, _ = flagellum_line(t, q_flag, k, ph)
            xi = np.concatenate([hx, fx])
            Xi = np.concatenate([hX, fX])
            w = np.concatenate([hw, fw])
            xidot = np.concatenate([np.zeros_like(hx), fv])
            return xi, Xi, w, xidot
        bodies.append(Body(FREE, n_head + n_flag, q_head + q_flag, shape, False,
                           np.array([lx + jx, ly + jy, 0.25]), np.eye(3), name=f"sperm{i}"))
    return Problem("sperm_channel", bodies, eps, 1.0, dt=0.01, steps=200)


def vogel_disc(npts: int, R: float):
    """Vogel spiral on the disc of radius R in the plane z = 0: point k at
    radius R sqrt((k + 1/2) / npts), angle k times the golden angle
    pi (3 - sqrt 5); equal weights pi R^2 / npts."""
    k = np.arange(npts, dtype=np.float64)
    r = R * np.sqrt((k + 0.5) / npts)
    th = k * (math.pi * (3.0 - math.sqrt(5.0)))
    P = np.stack([r * np.cos(th), r * np.sin(th), np.zeros(npts)], axis=1)
    return P, np.full(npts, math.pi * R * R / npts)


def rod_line(npts: int, length: float):
    """Midpoints of npts equal segments of the body x-axis from 0 to length,
    with the segment length as weight."""
    s = (np.arange(npts, dtype=np.float64) + 0.5) * (length / npts)
    P = np.stack([s, np.zeros(npts), np.zeros(npts)], axis=1)
    return P, np.full(npts, length / npts)


def node_config(index: int = 0, cilia=(10, 60), floor=(800, 2500), n_rod: int = 40,
                q_rod: int = 400, rod_len: float = 0.5, n_sphere: int = 4, q_sphere: int = 16,
                n_spheres: int = 5, eps: float = 0.005) -> Problem:
    """One ventral-node-like problem of the batch workload, seeded by (4, index).
    Draws, in order: the cilium count c in [cilia], the floor count N_f in
    [floor]; c cilium bases uniform in the disc r <= 1.6 (redrawn while closer
    than 0.4 to an earlier base; after 1000 redraws in a row the spacing
    shrinks by 10 %, since random packing cannot place more than about 35
    bases 0.4 apart in that disc); per cilium a tilt theta in [30, 45] degrees
    and a starting phase in [0, 2 pi); per sphere a centre (x, y) uniform in
    r <= 1.6 and a height in [0.7, 0.9].

    * floor: static disc of radius 2, Vogel spirals with N_f force points and
      10 N_f quadrature points;
    * cilia: rigid rods of length rod_len (n_rod / q_rod points on a line),
      prescribed rotation about the base at 2 pi clockwise seen from above,
      on a cone of semi-angle 30 degrees whose axis is tilted by theta
      towards -y; the body x-axis is the rod;
    * spheres: free rigid spheres of radius 0.05 (cube-sphere vertex clouds).
    n = 3 (n_rod c + N_f + n_spheres N_sphere) + 6 n_spheres."""
    rng = SplitMix64((4 << 32) | (index & 0xFFFFFFFF))
    c = int(cilia[0] + min(cilia[1] - cilia[0], int(rng.uniform() * (cilia[1] - cilia[0] + 1))))
    nf = int(floor[0] + min(floor[1] - floor[0], int(rng.uniform() * (floor[1] - floor[0] + 1))))
    bases: List[np.ndarray] = []
    sep, misses = 0.4, 0
    while len(bases) < c:
        r = 1.6 * math.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2.0 * math.pi)
        p = np.array([r * math.cos(th), r * math.sin(th), 0.0])
        if all(np.linalg.norm(p - o) >= sep for o in bases):
            bases.append(p)
            misses = 0
        else:
            misses += 1
            if misses == 1000:  # random packing at this spacing is full: shrink it
                sep *= 0.9
                misses = 0
    tilts = []
    for _ in range(c):
        tilts.append((math.radians(rng.uniform(30.0, 45.0)), rng.uniform(0.0, 2.0 * math.pi)))
    fx, fw = vogel_disc(nf, 2.0)
    fX, fwq = vogel_disc(10 * nf, 2.0)
    bodies = [Body(STATIC, nf, 10 * nf, _rigid(fx, fX, fwq), True, np.zeros(3), np.eye(3),
                   name="floor")]
    rx, _ = rod_line(n_rod, rod_len)
    rX, rw = rod_line(q_rod, rod_len)
    cone = math.radians(30.0)
    for i, (theta, phi) in enumerate(tilts):
        a = np.array([0.0, -math.sin(theta), math.cos(theta)])
        e1 = np.array([1.0, 0.0, 0.0])
        e2 = np.cross(a, e1)
        d = math.cos(cone) * a + math.sin(cone) * (math.cos(phi) * e1 + math.sin(phi) * e2)
        b2 = np.cross(a, d)
        b2 /= np.linalg.norm(b2)
        B = np.stack([d, b2, np.cross(d, b2)], axis=1)
        bodies.append(Body(PRESCRIBED, n_rod, q_rod, _rigid(rx, rX, rw), True, bases[i].copy(), B,
                           np.zeros(3), -2.0 * math.pi * a, name=f"cilium{i}"))
    sx, _ = cube_sphere_vertices(n_sphere, 0.05)
    sX, sw = cube_sphere_vertices(q_sphere, 0.05)
    for k in range(n_spheres):
        r = 1.6 * math.sqrt(rng.uniform())
        th = rng.uniform(0.0, 2.0 * math.pi)
        z = rng.uniform(0.7, 0.9)
        bodies.append(Body(FREE, len(sx), len(sX), _rigid(sx, sX, sw), True,
                           np.array([r * math.cos(th), r * math.sin(th), z]), np.eye(3),
                           name=f"sphere{k}"))
    return Problem(f"node{index}", bodies, eps, 1.0, dt=0.01, steps=20)


def node_batch(count: int = 128, **kw) -> List[Problem]:
    """The batch workload: node_config(i) for i < count."""
    return [node_config(i, **kw) for i in range(count)]


WORKLOADS: Dict[str, Callable[..., Problem]] = {
    "sphere": sphere_config,
    "sphere_cells": sphere_cells_config,
    "swimmer": swimmer_config,
    "swimmers4": swimmers_config,
    "sperm_channel": sperm_channel_config,
    "node": node_config,
}


def workload(name: str, **kw) -> Problem:
    return WORKLOADS[name](**kw)


def pack_shapes(problem: Problem, t: float) -> dict:
    """Concatenate the bodies' body-frame clouds at time t into the packed
    device layout: x (N,4) = [xi, 0], Xw (Q,4) = [Xi, w], xidot (N,4) =
    [xidot, 0]; plus point offsets per body (int64, length bodies+1)."""
    xs, Xs, vs = [], [], []
    n_off, q_off = [0], [0]
    for b in problem.bodies:
        xi, Xi, w, xidot = b.shape(t)
        assert xi.shape == (b.N, 3) and Xi.shape == (b.Q, 3) and w.shape == (b.Q,)
        xs.append(np.concatenate([xi, np.zeros((b.N, 1))], axis=1))
        Xs.append(np.concatenate([Xi, w[:, None]], axis=1))
        vs.append(np.concatenate([xidot, np.zeros((b.N, 1))], axis=1))
        n_off.append(n_off[-1] + b.N)
        q_off.append(q_off[-1] + b.Q)
    return {
        "x": np.ascontiguousarray(np.concatenate(xs), dtype=np.float64),
        "Xw": np.ascontiguousarray(np.concatenate(Xs), dtype=np.float64),
        "xidot": np.ascontiguousarray(np.concatenate(vs), dtype=np.float64),
        "n_off": np.array(n_off, dtype=np.int64),
        "q_off": np.array(q_off, dtype=np.int64),
    }


def body_table(problem: Problem) -> dict:
    """Per-body constants: kind, prescribed U and Omega (nb,3)."""
    return {
        "kind": np.array([b.kind for b in problem.bodies], dtype=np.int32),
        "U": np.array([b.U for b in problem.bodies], dtype=np.float64).reshape(-1, 3),
        "Omega": np.array([b.Omega for b in problem.bodies], dtype=np.float64).reshape(-1, 3),
        "rigid": np.array([b.rigid for b in problem.bodies], dtype=bool),
    }


def initial_state(problem: Problem) -> dict:
    """Initial rigid-body state Y = [x0; B] per body: x0 (nb,3), B (nb,3,3)
    (B's columns are the body-frame basis vectors in the lab frame)."""
    return {
        "x0": np.array([b.x0 for b in problem.bodies], dtype=np.float64).reshape(-1, 3),
        "B": np.array([b.B for b in problem.bodies], dtype=np.float64).reshape(-1, 3, 3),
    }

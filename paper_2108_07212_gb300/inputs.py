"""Seeded synthetic inputs for the PeriDEM force loop.

This module is shared by the GPU library's tests/benchmarks and by the CPU
oracle's tests.  It only *describes* problems -- grain outlines, grain
placements, material and run parameters -- and holds none of the method's
arithmetic (no meshing, no bonds, no forces).

Shapes follow Sec. 6.2 of the paper (perturbed disk, square, plus, annulus)
plus the disk / hexagon / triangle / drop shapes of the synthetic settling
workloads.  Every shape is a list of closed polygon loops in units of the grain
radius R (the radius of the grain's security disk): loop 0 is the outer
boundary in counter-clockwise order, further loops are holes in clockwise
order, so the material is always on the left of each directed edge.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ----------------------------------------------------------------------------
# shapes (units of R)


def regular_polygon(n: int, radius: float = 1.0, phase: float = 0.0) -> np.ndarray:
    """Counter-clockwise regular n-gon inscribed in a circle of ``radius``."""
    k = np.arange(n, dtype=np.float64)
    ang = phase + 2.0 * math.pi * k / n
    return np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1)


def disk_shape(n_vertices: int = 48) -> list[np.ndarray]:
    return [regular_polygon(n_vertices)]


def hexagon_shape() -> list[np.ndarray]:
    return [regular_polygon(6)]


def triangle_shape() -> list[np.ndarray]:
    return [regular_polygon(3, phase=math.pi / 2)]


def square_shape() -> list[np.ndarray]:
    """Square inscribed in the unit circle: side sqrt(2) (Sec. 6.2)."""
    return [regular_polygon(4, phase=math.pi / 4)]


def drop_shape(tail_radius: float = 0.5, n_arc: int = 40) -> list[np.ndarray]:
    """Convex tear drop: convex hull of a tip at (1, 0) and a circle of radius
    ``tail_radius`` touching the unit circle at (-1, 0)."""
    b = tail_radius
    cx = -1.0 + b
    dist = 1.0 - cx                      # tip to circle centre
    alpha = math.asin(b / dist)          # half opening angle at the tip
    # tangent points sit at polar angle +-(pi/2 - alpha) around the circle centre
    a0 = math.pi / 2 - alpha
    a1 = 2 * math.pi - a0
    ang = np.linspace(a0, a1, n_arc)
    arc = np.stack([cx + b * np.cos(ang), b * np.sin(ang)], axis=1)
    # the arc already runs counter-clockwise from the upper tangent point
    return [np.vstack([[1.0, 0.0], arc])]


def annulus_shape(tau: float = 0.6, n_outer: int = 48, n_inner: int = 32) -> list[np.ndarray]:
    """Ring with inner radius tau (Sec. 6.2, tau = 0.6); the hole is clockwise."""
    outer = regular_polygon(n_outer)
    inner = regular_polygon(n_inner, radius=tau)[::-1].copy()
    return [outer, inner]


def plus_shape(c: float = 0.2) -> list[np.ndarray]:
    """Plus (cross) of arm half-width c with arm tips on the unit circle."""
    r = c
    a = math.sqrt(1.0 - r * r)
    pts = [(a, -r), (a, r), (r, r), (r, a), (-r, a), (-r, r), (-a, r), (-a, -r),
           (-r, -r), (-r, -a), (r, -a), (r, -r)]
    return [np.array(pts, dtype=np.float64)]


def perturbed_disk_shape(rng: np.random.Generator, n: int = 20, phi: float = 0.6) -> list[np.ndarray]:
    """Disk perturbed inward at n vertices, r_i = 1 - X_i, X_i ~ U[0, 1-phi] (Sec. 6.2)."""
    x = rng.uniform(0.0, 1.0 - phi, size=n)
    r = 1.0 - x
    ang = 2.0 * math.pi * np.arange(n) / n
    return [np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)]


SHAPE_MAKERS = {
    "disk": disk_shape,
    "hexagon": hexagon_shape,
    "triangle": triangle_shape,
    "drop": drop_shape,
    "annulus": annulus_shape,
    "plus": plus_shape,
    "square": square_shape,
}

MIX_SETTLING = ("disk", "hexagon", "triangle", "drop", "annulus", "plus")


# ----------------------------------------------------------------------------
# workload description


@dataclasses.dataclass
class Workload:
    """A complete synthetic problem.

    shapes      list of shapes, each a list of (n_i, 2) float64 loops (units of R)
    grain_shape (G,) int32 index into ``shapes``
    grain_geom  (G, 7) float64 rows (cx, cy, R, theta, vx, vy, h) in SI units;
                h is the lattice spacing of that grain
    params      material / contact / wall / time-step parameters (SI units)
    n_steps     number of time steps of the full run
    name        label used in reports
    """

    shapes: list
    grain_shape: np.ndarray
    grain_geom: np.ndarray
    params: dict
    n_steps: int
    name: str = ""
    grain_agg: np.ndarray | None = None     # aggregate of each grain (batched ensembles)
    agg_walls: np.ndarray | None = None     # (A, 8): x_lo, x_hi, y_lo, y_hi and their normal velocities
    # (props (M, 4): E, k_bulk, rho, Gc per material; grain_material (G,)); None: params is the one material
    materials: tuple | None = None

    @property
    def n_grains(self) -> int:
        return int(self.grain_shape.shape[0])

    def flat_shapes(self):
        """(shape_loop_start[int32, S+1], loop_vtx_start[int32, L+1], vtx[float64, V*2])."""
        shape_loop_start = [0]
        loop_vtx_start = [0]
        vtx = []
        for loops in self.shapes:
            for lp in loops:
                vtx.append(np.asarray(lp, dtype=np.float64).reshape(-1, 2))
                loop_vtx_start.append(loop_vtx_start[-1] + vtx[-1].shape[0])
            shape_loop_start.append(shape_loop_start[-1] + len(loops))
        return (np.asarray(shape_loop_start, dtype=np.int32),
                np.asarray(loop_vtx_start, dtype=np.int32),
                np.ascontiguousarray(np.vstack(vtx)).reshape(-1))


def default_params(**over) -> dict:
    """Material M of the synthetic workloads: E = 1e7 Pa, rho = 1200 kg/m^3, Gc = 50 J/m^2.

    nu is fixed to 1/3 by the bond-based model (Remark after Table 1).  The bulk
    modulus k only enters the contact stiffness K_n = 18 k / (pi eps^5); with
    k = E / (3 (1 - 2 nu)) = E the damped contact pair is unstable under explicit
    Verlet at the workloads' time steps, so each workload picks a smaller k
    (see :func:`contact_cfl`).
    """
    p = dict(
        E=1.0e7, nu=1.0 / 3.0, k_bulk=1.0e7, rho=1200.0, Gc=50.0,
        horizon_ratio=3.0,          # eps = 3 h
        rc_ratio=0.95,              # R_c = 0.95 h_min
        damping_ratio=0.8, friction=0.5,
        gx=0.0, gy=-5000.0,
        dt=1.0e-7,
        wall_lo=(-5e-3, 0.0), wall_hi=(5e-3, 20e-3),
        wall_vel_lo=(0.0, 0.0), wall_vel_hi=(0.0, 0.0),
        micromodulus=0,             # 0 constant, 1 conic (Table 1)
    )
    p.update(over)
    return p


def contact_cfl(params: dict, h_min: float) -> dict:
    """Stability numbers of the stiffest node-node contact pair (equal volumes h_min^2).

    omega_dt   relative-motion angular frequency sqrt(2 K_n V^2 / (rho V)) times dt
    damp_dt    relative damping rate 2 c / (rho V) times dt, c = beta_d V^2
    Explicit velocity Verlet with the start-of-step velocity in the damping is
    stable for damp_dt below about 2 and omega_dt below 2.
    """
    eps = params["horizon_ratio"] * h_min
    kn = 18.0 * params["k_bulk"] / (math.pi * eps ** 5)
    V = h_min * h_min
    m = params["rho"] * V
    beta = 2.0 * params["damping_ratio"] * math.sqrt(kn * params["rho"] / V)
    c = beta * V * V
    dt = params["dt"]
    return dict(omega_dt=math.sqrt(2.0 * kn * V * V / m) * dt, damp_dt=2.0 * c / m * dt)


def _mk(shapes, gshape, ggeom, params, n_steps, name):
    return Workload(shapes=shapes, grain_shape=np.asarray(gshape, dtype=np.int32),
                    grain_geom=np.ascontiguousarray(np.asarray(ggeom, dtype=np.float64).reshape(-1, 7)),
                    params=params, n_steps=int(n_steps), name=name)


def two_disks(h_ratio: int = 8, gap: float = 0.5e-3, floor_gap: float | None = None,
              v_upper: float = 0.0, n_steps: int = 10_000, **over) -> Workload:
    """Two disks of radius 1 mm, h = R / h_ratio; the upper one falls ``gap`` onto
    the lower one, which rests ``floor_gap`` (default R_c / 2) above the floor."""
    R = 1e-3
    h = R / h_ratio
    params = default_params(k_bulk=1.0e6)
    params.update(over)
    rc = params["rc_ratio"] * h
    if floor_gap is None:
        floor_gap = rc / 2
    y0 = R + floor_gap
    y1 = y0 + 2 * R + gap
    ggeom = [(0.0, y0, R, 0.0, 0.0, 0.0, h), (0.0, y1, R, 0.0, 0.0, v_upper, h)]
    return _mk([disk_shape()], [0, 0], ggeom, params, n_steps, f"two_disks_h{h_ratio}")


def two_material_disks(**over) -> Workload:
    """Two disks of different materials (the material table of Sec. 5 lists a
    stiff and a soft one): the lower disk has the default soft material (E =
    1e7 Pa, k = 1e6 Pa, rho = 1200 kg/m^3, Gc = 50 J/m^2), the upper one twice
    its E, density and Gc and three times its bulk modulus (the same elastic
    wave speed, so the same stable time step).  They start R_c / 4 above the
    floor and 1.05 R_c apart, the upper one moving down at 1 m/s."""
    w = two_disks(**over)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + 0.25 * rc
    w.grain_geom[1, 0] = 0.25e-3
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 14 * h + 1.05 * rc
    w.grain_geom[1, 5] = -1.0
    p = w.params
    soft = (p["E"], p["k_bulk"], p["rho"], p["Gc"])
    stiff = (2 * p["E"], 3 * p["k_bulk"], 2 * p["rho"], 2 * p["Gc"])
    w.materials = (np.array([soft, stiff], dtype=np.float64), np.array([0, 1], dtype=np.int32))
    w.name = "two_material_disks"
    return w


def notched_square_shape(notch_w: float, notch_y: float) -> list[np.ndarray]:
    """Square of side 2 (units of R) with a straight notch of width notch_w from
    the middle of its left edge to its centre, centred at height notch_y."""
    yb, yt = notch_y - 0.5 * notch_w, notch_y + 0.5 * notch_w
    return [np.array([(-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0), (-1.0, yt), (0.0, yt), (0.0, yb),
                      (-1.0, yb)], dtype=np.float64)]


def rectangle_shape(aspect: float = 0.5) -> list[np.ndarray]:
    """Rectangle 2 x 2 aspect (units of R)."""
    return [np.array([(-1.0, -aspect), (1.0, -aspect), (1.0, aspect), (-1.0, aspect)], dtype=np.float64)]


def three_particles(gc_a: float = 135.0, h_ratio: int = 10, v: float = 20.0, n_steps: int = 2500,
                    **over) -> Workload:
    """The symmetric-impact test of Sec. 5.3: particle A, a 1 mm square with a
    0.5 mm notch from its left edge to its centre, is hit from below and from
    above by particles B and C, 1 mm x 0.5 mm rectangles at +v and -v (20 m/s).
    Damping and friction are off; dt = 20 ns (Sec. 5.1).  The paper gives no
    material for this test: all three take E and rho of M2 of the material
    table (E = 1.23 GPa, rho = 1200 kg/m^3), A with fracture energy gc_a (135
    or 13.5 J/m^2 in the paper), B and C with 135 J/m^2.  The contact bulk
    modulus is 5 MPa, not M2's 2 GPa: with K_n = 18 k / (pi eps^5) at h = 50 um
    and dt = 20 ns, 2 GPa gives a contact pair omega dt of 16 (explicit Verlet
    needs < 2), 5 MPa gives 0.8 (see contact_cfl).  Lattice h = R / h_ratio
    (R = 0.5 mm); the notch, 2 % of h wide, lies between two lattice rows, so
    it removes the bonds across it and no node; B and C start 1.02 R_c from A."""
    R = 0.5e-3
    h = R / h_ratio
    params = default_params(E=1.23e9, k_bulk=5.0e6, rho=1200.0, Gc=135.0, damping_ratio=0.0, friction=0.0,
                            gx=0.0, gy=0.0, dt=2.0e-8, wall_lo=(-5e-3, -5e-3), wall_hi=(5e-3, 5e-3))
    params.update(over)
    rc = params["rc_ratio"] * h
    na = h_ratio - 1                  # outermost lattice row of A (nodes strictly inside)
    nb = h_ratio // 2 - 1             # outermost lattice row of B and C (half-height R / 2)
    off = (na + nb) * h + 1.02 * rc   # centre distance: node rows 1.02 R_c apart
    shapes = [notched_square_shape(0.02 / h_ratio, 0.5 / h_ratio), rectangle_shape(0.5)]
    ggeom = [(0.0, 0.0, R, 0.0, 0.0, 0.0, h), (0.0, -off, R, 0.0, 0.0, v, h), (0.0, off, R, 0.0, 0.0, -v, h)]
    w = _mk(shapes, [0, 1, 1], ggeom, params, n_steps, f"three_particles_gc{gc_a:g}")
    p = w.params
    w.materials = (np.array([[p["E"], p["k_bulk"], p["rho"], gc_a], [p["E"], p["k_bulk"], p["rho"], p["Gc"]]]),
                   np.array([0, 1, 1], dtype=np.int32))
    return w


def _rsa_place(rng, radii, box_lo, box_hi, margin, max_tries=200000):
    """Random sequential addition of non-overlapping disks of radius radii+margin."""
    n = len(radii)
    P = np.zeros((n, 2))
    Rr = np.zeros(n)
    for k, r in enumerate(radii):
        rr = r + margin
        for _ in range(max_tries):
            x = rng.uniform(box_lo[0] + rr + margin, box_hi[0] - rr - margin)
            y = rng.uniform(box_lo[1] + rr + margin, box_hi[1] - rr - margin)
            if k == 0 or np.all((P[:k, 0] - x) ** 2 + (P[:k, 1] - y) ** 2 >= (Rr[:k] + rr) ** 2):
                P[k] = (x, y)
                Rr[k] = rr
                break
        else:
            raise RuntimeError("random sequential addition failed; box too small")
    return P


def settling(n_grains: int = 50, box=(20e-3, 30e-3), r_range=(1e-3, 1.5e-3), h_ratio: int = 15,
             mix=MIX_SETTLING, seed: int = 1, n_steps: int = 20_000, dt: float = 5e-8,
             **over) -> Workload:
    """Seeded mixed-shape grains in a rectangular wall box under gravity.

    Radii ~ U[r_range], shapes drawn uniformly from ``mix``, lattice spacing
    h = R / h_ratio per grain, random rotations, zero initial velocity.  Grains
    are placed by random sequential addition of security disks of radius
    R + R_c / 2 (so no contact force acts at t = 0) kept R_c away from the walls.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = rng.uniform(r_range[0], r_range[1], size=n_grains)
    kinds = rng.integers(0, len(mix), size=n_grains)
    theta = rng.uniform(0.0, 2 * math.pi, size=n_grains)
    params = default_params(dt=dt, friction=0.8, damping_ratio=0.8, k_bulk=5.0e5,
                            wall_lo=(0.0, 0.0), wall_hi=(box[0], box[1]))
    params.update(over)
    h_min = float(np.min(radii)) / h_ratio
    rc = params["rc_ratio"] * h_min
    order = np.argsort(-radii, kind="stable")          # place big grains first
    centres = np.empty((n_grains, 2))
    centres[order] = _rsa_place(rng, radii[order], (0.0, 0.0), box, rc / 2)
    shapes = []
    shape_index = {}
    gshape = []
    for g in range(n_grains):
        name = mix[kinds[g]]
        if name not in shape_index:
            shape_index[name] = len(shapes)
            shapes.append(SHAPE_MAKERS[name]())
        gshape.append(shape_index[name])
    ggeom = [(centres[g, 0], centres[g, 1], radii[g], theta[g], 0.0, 0.0, radii[g] / h_ratio)
             for g in range(n_grains)]
    return _mk(shapes, gshape, ggeom, params, n_steps, f"settling_{n_grains}g_seed{seed}")


def compaction(n_grains: int = 500, width: float = 40e-3, r_range=(0.8e-3, 1.6e-3), h_ratio: int = 23,
               wall_speed: float = 0.1, seed: int = 3, n_steps: int = 2000, dt: float = 2e-8,
               agitation: float = 0.0, **over) -> Workload:
    """Mixed-shape grains in a box of given width whose top wall moves down
    (no gravity).  dt = 2e-8 s keeps the damped contact of the h = R/23
    lattice (h_min = 35 um) stable at k = 5e5 Pa.  With agitation > 0 every
    grain starts with that speed in a seeded random direction, so that grains
    collide, load and fracture within a few hundred steps (a loaded window
    without the long compaction run that would lead to it)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = rng.uniform(r_range[0], r_range[1], size=n_grains)
    area = float(np.sum(math.pi * (radii + 0.1e-3) ** 2))
    height = area / 0.42 / width
    w = settling(n_grains=n_grains, box=(width, height), r_range=r_range, h_ratio=h_ratio,
                 seed=seed, n_steps=n_steps, dt=dt, gy=0.0, **over)
    w.params["wall_vel_hi"] = (0.0, -wall_speed)
    if agitation > 0:
        ang = np.random.Generator(np.random.PCG64(seed + 77)).uniform(0.0, 2 * math.pi, size=n_grains)
        w.grain_geom[:, 4] = agitation * np.cos(ang)
        w.grain_geom[:, 5] = agitation * np.sin(ang)
    w.name = f"compaction_{n_grains}g_seed{seed}"
    return w


def perturbed_disks(n_grains: int, seed: int = 7, **kw) -> Workload:
    """Settling workload made only of perturbed disks (one random outline per grain)."""
    w = settling(n_grains=n_grains, mix=("disk",), seed=seed, **kw)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    w.shapes = [perturbed_disk_shape(rng) for _ in range(n_grains)]
    w.grain_shape = np.arange(n_grains, dtype=np.int32)
    w.name = f"perturbed_{n_grains}g_seed{seed}"
    return w


def ensemble(n_agg: int = 64, grains_range=(20, 200), r_range=(0.8e-3, 1.2e-3), h_ratio: int = 21,
             seed: int = 11, dt: float = 2e-8, n_steps: int = 5000) -> Workload:
    """Batched ensemble of independent settling aggregates of uneven size.

    Aggregate a has n_a ~ U{grains_range} grains (seeded), radii ~ U[r_range],
    the settling shape mix, its own wall box (width ~ sqrt of its grain count,
    packing ~0.35 of the box) and its own seed; all aggregates share the
    material and time step (dt = 2e-8 s keeps the damped contact of the finer
    h = R/21 lattice stable at k = 5e5 Pa).  Returns one Workload whose grains carry their
    aggregate id; :func:`split_ensemble` gives the aggregates back one by one.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.integers(grains_range[0], grains_range[1] + 1, size=n_agg)
    parts = []
    for a in range(n_agg):
        n = int(counts[a])
        rmean = 0.5 * (r_range[0] + r_range[1])
        area = n * math.pi * (rmean + 0.1e-3) ** 2 / 0.35
        width = math.sqrt(area / 1.5)
        parts.append(settling(n_grains=n, box=(width, 1.5 * width), r_range=r_range, h_ratio=h_ratio,
                              seed=seed * 1000 + a, dt=dt, n_steps=n_steps))
    return merge_aggregates(parts, name=f"ensemble_{n_agg}agg_seed{seed}")


def merge_aggregates(parts, name="ensemble") -> Workload:
    """Concatenate independent workloads (same material and dt) into one batched workload."""
    shapes, gshape, ggeom, gagg, walls = [], [], [], [], []
    for a, w in enumerate(parts):
        base = len(shapes)
        shapes.extend(w.shapes)
        gshape.extend(int(s) + base for s in w.grain_shape)
        ggeom.append(w.grain_geom)
        gagg.extend([a] * w.n_grains)
        p = w.params
        walls.append([p["wall_lo"][0], p["wall_hi"][0], p["wall_lo"][1], p["wall_hi"][1],
                      p["wall_vel_lo"][0], p["wall_vel_hi"][0], p["wall_vel_lo"][1], p["wall_vel_hi"][1]])
    out = _mk(shapes, gshape, np.vstack(ggeom), dict(parts[0].params), parts[0].n_steps, name)
    out.grain_agg = np.asarray(gagg, dtype=np.int32)
    out.agg_walls = np.asarray(walls, dtype=np.float64)
    out.parts = parts
    return out


def surrogate_settling(n_grains: int = 2000, r_range=(1.0e-3, 1.5e-3), h_ratio: int = 23, seed: int = 5,
                       dt: float = 2.5e-8, n_steps: int = 5000) -> Workload:
    """Large settling aggregate for the surrogate: ~1000-node grains (h = R/23) of
    the settling shape mix in a box of packing ~0.35 (dt = 2.5e-8 s for the finer
    lattice)."""
    rmean = 0.5 * (r_range[0] + r_range[1])
    area = n_grains * math.pi * (rmean + 0.1e-3) ** 2 / 0.35
    width = math.sqrt(area / 2.0)
    w = settling(n_grains=n_grains, box=(width, 2.0 * width), r_range=r_range, h_ratio=h_ratio, seed=seed,
                 n_steps=n_steps, dt=dt)
    w.name = f"surrogate_settling_{n_grains}g_seed{seed}"
    return w


def free_grains(shapes=("hexagon", "disk"), n_per_shape: int = 8, R: float = 1e-3, h_ratio: int = 10,
                seed: int = 9, dt: float = 5e-8, n_steps: int = 2000) -> Workload:
    """Grains of equal size on a grid 3R apart, at rest, no gravity, random
    orientations: no contact, only the bond forces of whatever deformation a
    test gives them."""
    rng = np.random.default_rng(seed)
    names = [n for n in shapes for _ in range(n_per_shape)]
    G = len(names)
    cols = int(math.ceil(math.sqrt(G)))
    rows = int(math.ceil(G / cols))
    pitch = 3.0 * R
    shape_list = [SHAPE_MAKERS[n]() for n in shapes]
    gs = [shapes.index(n) for n in names]
    geom = []
    for k in range(G):
        cx = (k % cols + 1) * pitch
        cy = (k // cols + 1) * pitch
        geom.append([cx, cy, R, rng.uniform(0.0, 2.0 * math.pi), 0.0, 0.0, R / h_ratio])
    params = default_params(gy=0.0, dt=dt, wall_lo=(0.0, 0.0), wall_hi=((cols + 1) * pitch, (rows + 1) * pitch))
    return _mk(shape_list, gs, geom, params, n_steps, f"free_grains_{G}g_h{h_ratio}")

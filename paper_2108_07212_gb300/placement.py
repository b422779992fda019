"""Shape-agnostic initial placement of grains in security disks (Sec. 6.1).

Host-side set-up, before the time loop.  The construction follows the steps of
Sec. 6.1 ("Generating an initial particle distribution"):

1. a triangular mesh of the container (here a structured mesh of the wall
   box, its interior nodes jittered by a seeded amount, in place of the
   paper's mesh generator);
2. the inscribed circle of every triangle: centre
   c_T = (v1 l1 + v2 l2 + v3 l3) / (l1 + l2 + l3) with l_k the length of the
   side opposite v_k, radius r_T = 2 |T| / (l1 + l2 + l3);
3. one nodal circle per mesh node, as large as its constraints allow: it may
   not overlap the inscribed circle of any triangle around the node, may not
   leave the container, and (a reading: the paper is silent on two nodal
   circles) stays on the node's side of the perpendicular bisector of every
   mesh edge at the node, so nodal circles of different nodes are disjoint;
4. the radius r_v and centre c_v maximise the smallest distance to those
   constraints (the largest empty circle of the node's star), found by a
   pattern search started at the node;
5. every security disk shrinks by R_c / 2, so that no contact force acts at
   the start;
6. a grain whose shape is inscribed in the unit circle is placed in every
   disk with radius equal to the disk's and a seeded random rotation.

Disks smaller than a given minimum radius are dropped (a grain must hold a
lattice of nodes).
"""
from __future__ import annotations

import math

import numpy as np


def structured_mesh(lo, hi, spacing: float, jitter: float = 0.2, seed: int = 0):
    """Triangles of the box [lo, hi]: a grid of about ``spacing``, interior nodes
    moved by up to jitter * spacing (seeded), each cell cut along a diagonal
    chosen at random.  Returns (nodes (n, 2), triangles (t, 3) int, boundary
    flags (n,) bool)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx = max(1, int(round((hi[0] - lo[0]) / spacing)))
    ny = max(1, int(round((hi[1] - lo[1]) / spacing)))
    xs = np.linspace(lo[0], hi[0], nx + 1)
    ys = np.linspace(lo[1], hi[1], ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    nodes = np.stack([X.ravel(), Y.ravel()], 1)
    bnd = ((np.isclose(nodes[:, 0], lo[0]) | np.isclose(nodes[:, 0], hi[0]) |
            np.isclose(nodes[:, 1], lo[1]) | np.isclose(nodes[:, 1], hi[1])))
    hx, hy = (hi[0] - lo[0]) / nx, (hi[1] - lo[1]) / ny
    d = rng.uniform(-jitter, jitter, nodes.shape) * np.array([hx, hy])
    nodes = nodes + np.where(bnd[:, None], 0.0, d)
    tris = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, e = a + 1, a + nx + 1, a + nx + 2
            if rng.random() < 0.5:
                tris += [(a, b, e), (a, e, c)]
            else:
                tris += [(a, b, c), (b, e, c)]
    return nodes, np.asarray(tris, dtype=np.int64), bnd


def incircles(nodes: np.ndarray, tris: np.ndarray):
    """Centres (t, 2) and radii (t,) of the inscribed circles (step 2)."""
    v1, v2, v3 = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    l1 = np.linalg.norm(v2 - v3, axis=1)
    l2 = np.linalg.norm(v1 - v3, axis=1)
    l3 = np.linalg.norm(v1 - v2, axis=1)
    per = l1 + l2 + l3
    c = (v1 * l1[:, None] + v2 * l2[:, None] + v3 * l3[:, None]) / per[:, None]
    area = 0.5 * np.abs((v2[:, 0] - v1[:, 0]) * (v3[:, 1] - v1[:, 1]) - (v3[:, 0] - v1[:, 0]) * (v2[:, 1] - v1[:, 1]))
    return c, 2.0 * area / per


def _clearance(c, cT, rT, lo, hi, v, nbrs):
    """Largest radius of a circle at c that keeps out of the incircles (cT, rT),
    inside the box and on v's side of the bisectors of the edges v - w."""
    r = np.min(np.linalg.norm(cT - c, axis=1) - rT) if len(rT) else math.inf
    r = min(r, c[0] - lo[0], hi[0] - c[0], c[1] - lo[1], hi[1] - c[1])
    for w in nbrs:
        m, n = 0.5 * (v + w), w - v
        n = n / np.linalg.norm(n)
        r = min(r, float(np.dot(m - c, n)))          # signed distance to the bisector, towards v
    return r


# 16 search directions: the clearance is a minimum of distances, so its
# maximum sits on a ridge that few directions can climb
_DIRS = [np.array([math.cos(a), math.sin(a)]) for a in np.linspace(0.0, 2.0 * math.pi, 16, endpoint=False)]


def nodal_circles(nodes, tris, cT, rT, lo, hi, iters: int = 60):
    """Centre and radius of every node's circle (steps 3-4): pattern search for
    the centre maximising the clearance, started at the node."""
    n = nodes.shape[0]
    star = [[] for _ in range(n)]
    nbr = [set() for _ in range(n)]
    for t, (a, b, c) in enumerate(tris):
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):
            star[p].append(t)
            nbr[p].update((q, r))
    centres = np.zeros((n, 2))
    radii = np.zeros(n)
    for v in range(n):
        ts = np.asarray(star[v], dtype=np.int64)
        ws = [nodes[w] for w in sorted(nbr[v])]
        f = lambda c: _clearance(c, cT[ts], rT[ts], lo, hi, nodes[v], ws)
        c = nodes[v].copy()
        best = f(c)
        step = 0.5 * (np.min(rT[ts]) if len(ts) else 1.0)
        for _ in range(iters):
            moved = False
            for ang in _DIRS:
                cand = c + step * ang
                val = f(cand)
                if val > best:
                    c, best, moved = cand, val, True
            if not moved:
                step *= 0.5
        centres[v], radii[v] = c, max(best, 0.0)
    return centres, radii


def security_disks(lo, hi, spacing: float, rc_ratio: float, h_ratio: int, r_min: float, jitter: float = 0.2,
                   seed: int = 0):
    """Centres and radii of the security disks after the R_c / 2 shrink (steps
    1-5), dropping disks below r_min, and the packing ratio of the jammed
    configuration before the shrink.  A grain of radius R has lattice spacing
    R / h_ratio and R_c = rc_ratio h_min; the shrink uses the R_c of the
    largest disk, an upper bound on the aggregate's R_c, so that grains start
    at least R_c apart."""
    nodes, tris, _ = structured_mesh(lo, hi, spacing, jitter, seed)
    cT, rT = incircles(nodes, tris)
    cN, rN = nodal_circles(nodes, tris, cT, rT, lo, hi)
    centres = np.vstack([cT, cN])
    radii = np.concatenate([rT, rN])
    area = (hi[0] - lo[0]) * (hi[1] - lo[1])
    packing = float(np.sum(math.pi * radii ** 2) / area)
    rc = rc_ratio * float(radii.max()) / h_ratio
    radii = radii - 0.5 * rc
    keep = radii >= r_min
    return centres[keep], radii[keep], packing, rc


def jammed_settling(box=(20e-3, 30e-3), spacing: float = 3.2e-3, h_ratio: int = 15, mix=None, seed: int = 1,
                    n_steps: int = 50_000, dt: float = 2e-8, r_min_ratio: float = 0.15, **over):
    """The settling workload with the shape-agnostic jammed placement in place
    of random sequential addition: every security disk of the box holds one
    grain (shapes cycled through the settling mix), of radius equal to the
    disk's, lattice spacing R / h_ratio, rotated at random (step 6).  Disks
    smaller than r_min_ratio * spacing are left empty.  The smallest grains
    (R ~ 0.5 mm, h ~ 32 um) make the bond and contact stiffness those of the
    finest lattices here, so dt = 2e-8 s, as for the other h ~ 35 um
    workloads (at 5e-8 s the first contacts blow up)."""
    from . import inputs as I

    mix = I.MIX_SETTLING if mix is None else mix
    params = I.default_params(dt=dt, friction=0.8, damping_ratio=0.8, k_bulk=5.0e5, wall_lo=(0.0, 0.0),
                              wall_hi=(box[0], box[1]))
    params.update(over)
    centres, radii, packing, rc = security_disks((0.0, 0.0), box, spacing, params["rc_ratio"], h_ratio,
                                                 r_min=r_min_ratio * spacing, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    n = len(radii)
    shapes = [I.SHAPE_MAKERS[name]() for name in mix]
    gshape = np.arange(n) % len(mix)
    theta = rng.uniform(0.0, 2.0 * math.pi, n)
    geom = np.zeros((n, 7))
    geom[:, 0], geom[:, 1], geom[:, 2], geom[:, 3] = centres[:, 0], centres[:, 1], radii, theta
    geom[:, 6] = radii / h_ratio
    w = I.Workload(shapes=shapes, grain_shape=gshape.astype(np.int32), grain_geom=geom, params=params,
                   n_steps=int(n_steps), name="jammed_settling")
    w.packing_jammed = packing
    w.shrink_rc = rc
    return w

"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

None of these tests re-types an oracle formula: each checks a closed form
obtained by a different route (a numerical integral, an energy gradient, the
analytic motion of a linear oscillator), an invariant, a special value the
paper prints, or a brute-force evaluation of a definition.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O
from paper_2108_07212_gb300 import inputs as I

E, NU, GC = 1.0e7, 1.0 / 3.0, 50.0


def _prm(Kn, Rc, rho=1200.0, dt=1e-8, rd=0.0, mu=0.0, g=(0.0, 0.0), walls=(-1.0, 1.0, -1.0, 1.0),
         wall_vel=(0.0, 0.0, 0.0, 0.0), micro=0, grid=True):
    p = np.zeros(O.P_NPARAM)
    p[O.P_RHO], p[O.P_KN], p[O.P_RC], p[O.P_DT] = rho, Kn, Rc, dt
    p[O.P_RD], p[O.P_MU] = rd, mu
    p[O.P_GX], p[O.P_GY] = g
    p[O.P_WX0], p[O.P_WX1], p[O.P_WY0], p[O.P_WY1] = walls
    p[O.P_VX0], p[O.P_VX1], p[O.P_VY0], p[O.P_VY1] = wall_vel
    p[O.P_MICRO] = micro
    p[O.P_SEARCH] = 1.0 if grid else 0.0
    return p


# ---------------------------------------------------------------------------
# Table 1: spring constant and critical stretch


@pytest.mark.parametrize("micro", [0, 1])
def test_spring_constant_reproduces_continuum_energy(micro):
    """Under uniform dilation e0 the peridynamic energy density
    W = 1/2 int_H 1/2 c w(|xi|) e0^2 |xi| dA must equal the 2D continuum value
    E e0^2 / (1 - nu) (the calibration behind Table 1)."""
    eps = 3.75e-4
    cw, _ = O.bond_constants(E, NU, GC, eps, micro)
    w = (lambda r: 1.0) if micro == 0 else (lambda r: 1.0 - r / eps)
    e0 = 1e-3
    integral, _ = quad(lambda r: 0.5 * cw * w(r) * e0 ** 2 * r * 2.0 * math.pi * r, 0.0, eps)
    assert 0.5 * integral == pytest.approx(E * e0 ** 2 / (1.0 - NU), rel=1e-10)


@pytest.mark.parametrize("micro", [0, 1])
def test_critical_stretch_reproduces_fracture_energy(micro):
    """Sec. 3.1: s0 makes the work to break every bond across a unit crack equal Gc:
    G = int_0^eps dz int_z^eps dr 2 acos(z/r) * 1/2 c w(r) s0^2 r * r."""
    eps = 3.75e-4
    cw, s0 = O.bond_constants(E, NU, GC, eps, micro)
    w = (lambda r: 1.0) if micro == 0 else (lambda r: 1.0 - r / eps)

    def inner(z):
        return quad(lambda r: 2.0 * math.acos(z / r) * 0.5 * cw * w(r) * s0 ** 2 * r * r, z, eps)[0]

    G, _ = quad(inner, 0.0, eps, limit=200)
    assert G == pytest.approx(GC, rel=1e-8)


def test_contact_stiffness_scaling():
    """K_n = 18 k / (pi eps^5): linear in k, eps^-5 (Sec. 4.1)."""
    k0 = O.contact_stiffness(1e7, 1e-4)
    assert O.contact_stiffness(2e7, 1e-4) / k0 == pytest.approx(2.0, rel=1e-14)
    assert O.contact_stiffness(1e7, 2e-4) / k0 == pytest.approx(1.0 / 32.0, rel=1e-14)


def test_contact_stiffness_is_the_3d_bond_micromodulus_over_the_horizon():
    """Reading of Sec. 4.1: K_n = 18 k / (pi eps^5) is the micromodulus of the
    3D bond-based model, c = 18 k / (pi eps^4), per unit length of the horizon
    (the contact law is linear in the overlap R_c - |d|, a length, where the
    bond law is linear in the stretch).  Here c comes from its own definition:
    under a uniform dilation with stretch s every bond of the 3D horizon stores
    (1/2) c s^2 |xi| (half per node), and the energy density, integrated by
    quadrature over the ball, must equal the bulk energy (1/2) k (3 s)^2.  A
    transcription with another constant (9/pi, 18 pi, ...) fails."""
    k, eps, s = 1.3e6, 2.7e-4, 1e-3
    # energy density per unit c: the integral over the ball of (1/4) s^2 |xi|
    per_c = quad(lambda r: 0.25 * s * s * r * 4.0 * math.pi * r * r, 0.0, eps)[0]
    c = 0.5 * k * (3.0 * s) ** 2 / per_c
    assert O.contact_stiffness(k, eps) * eps == pytest.approx(c, rel=1e-12)


# ---------------------------------------------------------------------------
# bond law


def _two_node(u1, h=1e-4, micro=0, theta=0.3):
    eps = 3 * h
    cw, s0 = O.bond_constants(E, NU, GC, eps, micro)
    X = np.array([[0.0, 0.0], [h * math.cos(theta), h * math.sin(theta)]])
    P = O.OracleProblem(X, [h * h] * 2, [0, 0], [0, 1, 2], [1, 0], [cw], [s0], [eps], _prm(1.0, 0.0, micro=micro))
    P.u[1] = u1
    return P, cw, s0


@pytest.mark.parametrize("micro", [0, 1])
def test_bond_force_is_minus_energy_gradient(micro):
    """The pairwise force density of eq. (pmb) derives from the PMB pair potential
    1/2 c w s^2 |xi|: compare the oracle force with a finite-difference gradient
    of the oracle bond energy."""
    P, cw, s0 = _two_node(np.array([3e-6, -2e-6]), micro=micro)
    F, parts = P.forces()
    delta = 1e-10
    grad = np.zeros(2)
    for k in range(2):
        P.u[0, k] += delta
        ep = P.diagnostics()["E_bond"]
        P.u[0, k] -= 2 * delta
        em = P.diagnostics()["E_bond"]
        P.u[0, k] += delta
        grad[k] = (ep - em) / (2 * delta)
    assert np.allclose(parts[0, 0], -grad, rtol=1e-6, atol=0)
    # tension pulls node 0 towards node 1
    d = (P.X[1] + P.u[1]) - (P.X[0] + P.u[0])
    assert np.dot(parts[0, 0], d) > 0
    assert np.allclose(parts[0, 0], -parts[0, 1], rtol=0, atol=1e-15 * np.abs(parts[0, 0]).max())


def test_rigid_motion_gives_zero_bond_force():
    """eq:pmb depends on the deformed bond length only: a rigid rotation plus
    translation of every grain (non-convex plus, holed annulus, drop) leaves
    every stretch and so every bond force at zero, to rounding, while a uniform
    dilation of 1e-3 gives forces of its own size.  A law that used displacement
    differences instead of lengths would give forces of the rotation's size."""
    w = I.free_grains(shapes=("plus", "annulus", "drop"), n_per_shape=1, h_ratio=10)
    P = O.OracleProblem.from_workload(w)
    rng = np.random.default_rng(4)
    u_rigid = np.zeros_like(P.X)
    u_dil = np.zeros_like(P.X)
    for g in range(w.n_grains):
        m = P.grain == g
        c = P.X[m].mean(axis=0)
        th = rng.uniform(0.3, 2.5)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        r = P.X[m] - c
        u_rigid[m] = r @ R.T - r + rng.uniform(-1e-3, 1e-3, 2)
        u_dil[m] = 1e-3 * r
    P.u[:] = u_dil
    _, parts = P.forces()
    scale = np.abs(parts[0]).max()
    assert scale > 0
    P.u[:] = u_rigid
    F, parts = P.forces()
    assert np.abs(parts[0]).max() <= 1e-9 * scale
    assert np.abs(F).max() <= 1e-9 * scale
    assert not P.broken.any()


def test_bond_breaks_beyond_critical_stretch_and_stays_broken():
    """Sec. 3.1: |s| > s0 breaks the bond; it remains broken afterwards; also in
    compression (absolute value)."""
    h = 1e-4
    for sign in (+1, -1):
        P, cw, s0 = _two_node(np.zeros(2), theta=0.0)
        P.u[1, 0] = sign * 0.99 * s0 * h
        F, _ = P.forces(keep_broken=False)
        assert P.broken.sum() == 0 and abs(F[0, 0]) > 0
        P.u[1, 0] = sign * 1.01 * s0 * h
        F, _ = P.forces(keep_broken=False)
        assert P.broken.sum() == 2 and np.all(F == 0)
        P.u[1, 0] = 0.5 * s0 * h
        F, _ = P.forces(keep_broken=False)
        assert P.broken.sum() == 2 and np.all(F == 0)


def test_damage_is_broken_over_reference_bonds():
    """Sec. 3.1: damage = broken / reference bonds of the node."""
    h = 1e-4
    eps = 3 * h
    cw, s0 = O.bond_constants(E, NU, GC, eps, 0)
    X = np.array([[0, 0], [h, 0], [0, h], [h, h]], dtype=float)
    row = [0, 3, 6, 9, 12]
    col = [1, 2, 3, 0, 2, 3, 0, 1, 3, 0, 1, 2]
    P = O.OracleProblem(X, [h * h] * 4, [0] * 4, row, col, [cw], [s0], [eps], _prm(1.0, 0.0))
    P.u[3] = [0.5 * h, 0.5 * h]          # node 3 pulled far away: its 3 bonds break
    P.forces(keep_broken=False)
    assert np.allclose(P.damage(), [1 / 3, 1 / 3, 1 / 3, 1.0])


def test_bond_forces_sum_to_zero_force_and_moment():
    """Central, pairwise-antisymmetric bond forces: zero net force and zero net
    moment about the origin for any deformation (to round-off)."""
    w = I.Workload(shapes=[I.plus_shape()], grain_shape=np.array([0], np.int32),
                   grain_geom=np.array([[1e-3, 2e-3, 1e-3, 0.4, 0, 0, 1e-3 / 15]]),
                   params=I.default_params(), n_steps=1)
    P = O.OracleProblem.from_workload(w)
    rng = np.random.default_rng(5)
    P.u[:] = rng.normal(scale=2e-7, size=P.u.shape)
    F, parts = P.forces()
    Fb = parts[0]
    p = P.positions
    scale = np.abs(Fb).sum()
    assert abs(Fb[:, 0].sum()) < 1e-13 * scale
    assert abs(Fb[:, 1].sum()) < 1e-13 * scale
    mom = np.sum(p[:, 0] * Fb[:, 1] - p[:, 1] * Fb[:, 0])
    assert abs(mom) < 1e-12 * scale * np.abs(p).max()


def test_uniform_dilation_interior_force_and_energy():
    """u = e0 (X - c): every bond has s = e0; nodes with a full 24-bond horizon
    feel zero net force (lattice symmetry), and the bond energy equals
    sum over directed bonds of 1/4 c e0^2 |xi| V^2 with |xi| = h sqrt(di^2 + dj^2)."""
    h = 1e-3 / 15
    w = I.Workload(shapes=[I.disk_shape()], grain_shape=np.array([0], np.int32),
                   grain_geom=np.array([[0.0, 0.0, 1e-3, 0.0, 0, 0, h]]), params=I.default_params(), n_steps=1)
    P = O.OracleProblem.from_workload(w)
    e0 = 1e-3
    P.u[:] = e0 * P.X
    F, parts = P.forces()
    counts = np.diff(P.row_ptr)
    full = counts == 24
    cw = P.g_cw[0]
    assert full.sum() > 300
    assert np.abs(parts[0][full]).max() < 1e-8 * cw * e0 * h ** 4
    assert np.abs(parts[0][~full]).max() > 1e-2 * cw * e0 * h ** 4
    rows = np.repeat(np.arange(P.N), counts)
    dl = P.lat[P.col] - P.lat[rows]
    xi = h * np.sqrt((dl ** 2).sum(axis=1))
    expected = np.sum(0.25 * cw * e0 ** 2 * xi * h ** 4)
    assert P.diagnostics()["E_bond"] == pytest.approx(expected, rel=1e-9)


# ---------------------------------------------------------------------------
# contact laws


def _two_grain_nodes(Rc, h, gap, v_rel, rd=0.0, mu=0.0, dt=None, k_bulk=1e6, rho=1200.0):
    V = h * h
    Kn = O.contact_stiffness(k_bulk, 3 * h)
    omega = math.sqrt(2 * Kn * V * V / (rho * V))
    if dt is None:
        dt = 0.01 / omega
    X = np.array([[0.0, 0.0], [Rc + gap, 0.0]])
    v0 = np.array([[v_rel / 2, 0.0], [-v_rel / 2, 0.0]])
    P = O.OracleProblem(X, [V, V], [0, 1], [0, 0, 0], [], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0],
                        _prm(Kn, Rc, rho=rho, dt=dt, rd=rd, mu=mu), v0)
    return P, Kn, omega, dt


def _collide(P, Rc, max_steps=100000):
    P.init_accel()
    contact_steps = 0
    started = False
    for _ in range(max_steps):
        P.run(1)
        d = np.linalg.norm(P.positions[1] - P.positions[0])
        if d < Rc:
            started = True
            contact_steps += 1
        elif started:
            break
    return contact_steps


def test_normal_contact_is_linear_spring_half_period():
    """Eq. (law-repulsive) between two single-node grains is a linear spring of
    stiffness K_n V^2 on the reduced mass rho V / 2: the contact lasts half a
    period pi / omega and the rebound speed equals the impact speed."""
    h, Rc = 1e-4, 0.95e-4
    P, Kn, omega, dt = _two_grain_nodes(Rc, h, gap=1e-9, v_rel=0.1)
    steps = _collide(P, Rc)
    assert steps * dt == pytest.approx(math.pi / omega, rel=0.01)
    v_out = P.v[0, 0] - P.v[1, 0]
    assert v_out == pytest.approx(-0.1, rel=1e-4)


def test_friction_is_continuous_at_the_stick_slip_switch():
    """Sec. 4.2 with the small-velocity sticking: the tangential contact force
    is linear in the relative tangential velocity below the switch (sticking)
    and of constant size above it (sliding), and the two branches meet where
    they switch: the threshold is chosen so that the law is continuous.  The
    force opposes the relative tangential velocity.  Located from the oracle's
    own outputs (the slope of the small-speed branch and the size of the
    large-speed one), not from the threshold formula."""
    h, Rc = 1e-4, 0.95e-4
    P, *_ = _two_grain_nodes(Rc, h, gap=-0.3 * Rc, v_rel=0.0, mu=0.5, dt=1e-8)   # overlapping: F_r > 0

    def tangential(vt):
        P.v[:] = 0.0
        P.v[0, 1] = vt                          # normal along x, tangential along y
        F, parts = P.forces()
        return parts[2][0, 1]                   # contact part on node 0, tangential component

    small, big = 1e-9, 10.0
    f1, f2 = tangential(small), tangential(2 * small)
    assert f1 < 0 and f2 == pytest.approx(2 * f1, rel=1e-9)            # sticking: linear, opposing
    g1, g2 = tangential(big), tangential(2 * big)
    assert g1 < 0 and g2 == pytest.approx(g1, rel=1e-12)               # sliding: constant size
    assert tangential(-big) == pytest.approx(-g1, rel=1e-12)           # opposing either way
    v_switch = g1 / (f1 / small)                 # where the linear branch reaches the sliding size
    for side in (1.0 - 1e-6, 1.0 + 1e-6):
        assert tangential(side * v_switch) == pytest.approx(g1, rel=2e-6)
    # and the switch is there, not elsewhere: linear just below, constant well above
    assert tangential(0.9 * v_switch) == pytest.approx(0.9 * g1, rel=1e-9)
    assert tangential(1.5 * v_switch) == pytest.approx(g1, rel=1e-12)
    assert abs(tangential(0.5 * v_switch)) == pytest.approx(0.5 * abs(g1), rel=1e-9)


def test_normal_damping_restitution_matches_kelvin_voigt():
    """Sec. 4.3: spring K_n V^2 + dashpot beta_d V^2 with beta_d = 2 r_d sqrt(K_n rho / V)
    on reduced mass rho V / 2 has damping ratio zeta = sqrt(2) r_d and restitution
    exp(-pi zeta / sqrt(1 - zeta^2))."""
    h, Rc, rd = 1e-4, 0.95e-4, 0.1
    P, Kn, omega, dt = _two_grain_nodes(Rc, h, gap=1e-9, v_rel=0.1, rd=rd, dt=None)
    P.prm[O.P_DT] = 0.002 / omega
    _collide(P, Rc, max_steps=400000)
    zeta = math.sqrt(2.0) * rd
    e = math.exp(-math.pi * zeta / math.sqrt(1 - zeta ** 2))
    v_out = -(P.v[0, 0] - P.v[1, 0]) / 0.1
    assert v_out == pytest.approx(e, rel=0.01)


def test_self_contact_equals_contact_when_cw_over_Rc_is_Kn():
    """Sec. 4.4 remark: for |xi| > R_c the self-contact force equals the
    inter-grain contact force when c_w / R_c = K_n (damping and friction too)."""
    h, Rc = 1e-4, 0.95e-4
    V = h * h
    Kn = O.contact_stiffness(1e6, 3 * h)
    prm = _prm(Kn, Rc, dt=1e-9, rd=0.5, mu=0.4)
    X = np.array([[0.0, 0.0], [3 * Rc, 0.0]])          # reference distance beyond R_c, no bond
    u = np.array([[0.0, 0.0], [-2.2 * Rc, 0.1 * Rc]])   # now closer than R_c
    v = np.array([[0.3, 0.1], [-0.2, 0.05]])
    self_p = O.OracleProblem(X, [V, V], [0, 0], [0, 0, 0], [], [Kn * Rc], [1.0], [1.0], prm, v)
    pair_p = O.OracleProblem(X, [V, V], [0, 1], [0, 0, 0], [], [Kn * Rc] * 2, [1.0] * 2, [1.0] * 2, prm, v)
    self_p.u[:] = u
    pair_p.u[:] = u
    Fs, ps = self_p.forces()
    Fp, pp = pair_p.forces()
    assert np.abs(ps[1]).max() > 0 and np.abs(pp[2]).max() > 0
    assert np.allclose(ps[1], pp[2], rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# self-contact of nodes whose reference distance is below R_c (Sec. 4.4, first branch)


def _self_pair(xi, Rc, Kn, d, v_rel=0.0, dt=1e-9):
    """Two unbonded nodes of one grain, reference distance xi, current distance d."""
    h = 1e-4
    V = h * h
    prm = _prm(Kn, Rc, dt=dt)
    X = np.array([[0.0, 0.0], [xi, 0.0]])
    v = np.array([[v_rel / 2, 0.0], [-v_rel / 2, 0.0]])
    P = O.OracleProblem(X, [V, V], [0, 0], [0, 0, 0], [], [Kn * Rc], [1.0], [3 * h], prm, v)
    P.u[1, 0] = d - xi
    return P, V


def test_self_contact_below_Rc_is_a_one_sided_spring_about_the_reference_distance():
    """For |xi| < R_c the self-contact force c_w (d - |xi|) / |xi| V_x V_y acts only
    while d < |xi|: a linear spring of stiffness c_w V^2 / |xi| on the reduced mass
    rho V / 2 that is compressed from its rest length.  An approaching pair
    therefore stays in contact for half a period pi / omega and leaves with its
    impact speed (no damping, no friction), and the pair feels nothing while
    |xi| <= d < R_c (no attraction back to the reference distance)."""
    h, Rc = 1e-4, 0.95e-4
    Kn = O.contact_stiffness(1e6, 3 * h)
    cw = Kn * Rc
    xi = 0.5 * Rc
    V = h * h
    omega = math.sqrt(2.0 * (cw * V * V / xi) / (1200.0 * V))
    dt = 0.005 / omega
    P, _ = _self_pair(xi, Rc, Kn, d=xi + 1e-9, v_rel=0.1, dt=dt)
    P.init_accel()
    inside = 0
    started = False
    for _ in range(20000):
        P.run(1)
        dist = np.linalg.norm(P.positions[1] - P.positions[0])
        if dist < xi:
            started = True
            inside += 1
        elif started:
            break
    assert inside * dt == pytest.approx(math.pi / omega, rel=0.01)
    assert (P.v[0, 0] - P.v[1, 0]) == pytest.approx(-0.1, rel=1e-4)
    # between |xi| and R_c: inside the contact radius, yet no force
    for frac in (0.55, 0.75, 0.99):
        Q, _ = _self_pair(xi, Rc, Kn, d=frac * Rc, v_rel=0.3)
        F, parts = Q.forces()
        assert np.all(F == 0.0) and np.all(parts == 0.0)


def test_self_contact_branches_meet_at_Rc():
    """The two self-contact branches (|xi| < R_c: rest length |xi|; |xi| >= R_c:
    rest length R_c) give the same force as |xi| crosses R_c from either side,
    at any compression d < R_c."""
    h, Rc = 1e-4, 0.95e-4
    Kn = O.contact_stiffness(1e6, 3 * h)
    for frac in (0.3, 0.7, 0.95):
        d = frac * Rc
        below, _ = _self_pair(Rc * (1 - 1e-10), Rc, Kn, d)
        above, _ = _self_pair(Rc * (1 + 1e-10), Rc, Kn, d)
        Fb, pb = below.forces()
        Fa, pa = above.forces()
        assert np.abs(pb[1]).max() > 0
        assert np.allclose(pb[1], pa[1], rtol=1e-8, atol=0)


def test_friction_on_floor_gives_coulomb_deceleration_then_sticks():
    """Sec. 4.2 + 4.5: a node resting on the floor (|F_r| = rho V g) sliding at v0
    decelerates at mu g (slip) and then sticks (zero relative speed kept)."""
    h = 1e-4
    Rc = 0.95 * h
    V = h * h
    Kn = O.contact_stiffness(1e6, 3 * h)
    g, mu = 5000.0, 0.5
    prm = _prm(Kn, Rc, dt=2e-9, rd=0.8, mu=mu, g=(0.0, -g), walls=(-1.0, 1.0, 0.0, 1.0))
    P = O.OracleProblem(np.array([[0.0, Rc]]), [V], [0], [0, 0], [], [1.0], [1.0], [1.0], prm)
    P.init_accel()
    P.run(150000)                                  # settle on the floor
    assert abs(P.v[0, 1]) < 1e-9
    v0 = 0.05
    P.v[0, 0] = v0
    ts, vs = [], []
    for k in range(12000):
        P.run(1)
        ts.append(P.step * prm[O.P_DT])
        vs.append(P.v[0, 0])
    ts, vs = np.array(ts), np.array(vs)
    sl = (vs > 0.2 * v0) & (vs < 0.8 * v0)
    slope = np.polyfit(ts[sl], vs[sl], 1)[0]
    assert slope == pytest.approx(-mu * g, rel=0.01)
    assert abs(vs[-1]) < 1e-6 * v0


# ---------------------------------------------------------------------------
# wall regions (Sec. 4.5)


def test_wall_segment_area_and_centroid_by_quadrature():
    Rc = 1.3e-4
    A0, c0 = O.wall_segment(0.0, Rc)
    assert A0 == pytest.approx(math.pi * Rc ** 2 / 2, rel=1e-15)        # half disk (paper)
    for f in (0.0, 0.2, 0.5, 0.8, 0.97):
        d = f * Rc
        A, c = O.wall_segment(d, Rc)
        # x = Rc sin(phi) removes the square-root end-point singularity
        f0 = math.asin(d / Rc)
        Aq = quad(lambda f: 2 * Rc * math.cos(f) * Rc * math.cos(f), f0, math.pi / 2, epsabs=0, epsrel=1e-13)[0]
        Mq = quad(lambda f: Rc * math.sin(f) * 2 * Rc * math.cos(f) * Rc * math.cos(f), f0, math.pi / 2,
                  epsabs=0, epsrel=1e-13)[0]
        assert A == pytest.approx(Aq, rel=1e-9)
        assert c == pytest.approx(Mq / Aq, rel=1e-9)


def test_wall_segment_stays_accurate_as_it_vanishes():
    """As d -> R_c the region shrinks to nothing; area and R_c - |c - p| must keep
    full relative precision (50-digit evaluation of the same integrals)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    Rc = 1.3e-4
    for f in (0.99, 0.9999, 0.999999, 0.99999999):
        d = f * Rc
        R, D = mpmath.mpf(Rc), mpmath.mpf(d)
        A = R * R * mpmath.acos(D / R) - D * mpmath.sqrt(R * R - D * D)
        c = mpmath.mpf(2) / 3 * (R * R - D * D) ** mpmath.mpf(1.5) / A
        A_o, c_o = O.wall_segment(d, Rc)
        assert float(abs(A_o - A) / A) < 1e-12
        assert float(abs((Rc - c_o) - (R - c)) / (R - c)) < 1e-9


def test_corner_region_area_and_moments_by_quadrature():
    Rc = 1.3e-4
    A, Ix, Iy = O.corner_region(0.0, 0.0, Rc)
    assert A == pytest.approx(math.pi * Rc ** 2 / 4, rel=1e-14)         # quarter disk (paper)
    assert Ix == pytest.approx(Iy, rel=1e-14)
    for fi, fj in [(0.1, 0.3), (0.5, 0.2), (0.6, 0.7), (0.0, 0.9), (0.3, 0.0), (0.6, 0.79), (0.7071, 0.7071)]:
        di, dj = fi * Rc, fj * Rc
        if di * di + dj * dj >= Rc * Rc:
            continue
        b = math.sqrt(Rc * Rc - dj * dj)
        f0, f1 = math.asin(di / Rc), math.asin(b / Rc)
        kw = dict(epsabs=0, epsrel=1e-13)

        def jac(f):
            return Rc * math.cos(f)

        Aq = quad(lambda f: (Rc * math.cos(f) - dj) * jac(f), f0, f1, **kw)[0]
        Ixq = quad(lambda f: Rc * math.sin(f) * (Rc * math.cos(f) - dj) * jac(f), f0, f1, **kw)[0]
        Iyq = quad(lambda f: 0.5 * ((Rc * math.cos(f)) ** 2 - dj * dj) * jac(f), f0, f1, **kw)[0]
        A, Ix, Iy = O.corner_region(di, dj, Rc)
        assert A == pytest.approx(Aq, rel=1e-8)
        assert Ix == pytest.approx(Ixq, rel=1e-8)
        assert Iy == pytest.approx(Iyq, rel=1e-8)


# ---------------------------------------------------------------------------
# geometry: mesh and non-convex horizon


def _poly_area(loops):
    a = 0.0
    for lp in loops:
        x, y = lp[:, 0], lp[:, 1]
        a += 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
    return a


@pytest.mark.parametrize("name", ["disk", "hexagon", "triangle", "drop", "annulus", "plus", "square"])
def test_mesh_volume_converges_to_polygon_area(name):
    """Sum of nodal volumes h^2 -> grain area; the lattice-count error is bounded
    by the boundary layer, |n h^2 - A| <= 1.5 * perimeter * h."""
    loops = I.SHAPE_MAKERS[name]()
    R = 1e-3
    area = _poly_area(loops) * R * R
    perim = sum(np.sum(np.hypot(*(np.roll(lp, -1, axis=0) - lp).T)) for lp in loops) * R
    for ratio in (15, 30, 60, 120):
        h = R / ratio
        X, lat = O.mesh_grain(loops, R, h)
        assert abs(X.shape[0] * h * h - area) <= 1.5 * perim * h
    assert abs(X.shape[0] * h * h - area) / area < 0.02


def _inside_closed(pts, loops, scale, tol):
    """Brute force: even-odd test plus distance-to-boundary tolerance."""
    px, py = pts[:, 0], pts[:, 1]
    inside = np.zeros(len(pts), dtype=bool)
    dist = np.full(len(pts), np.inf)
    for lp in loops:
        v = np.asarray(lp) * scale
        w = np.roll(v, -1, axis=0)
        for (x0, y0), (x1, y1) in zip(v, w):
            cond = (y0 > py) != (y1 > py)
            with np.errstate(divide="ignore", invalid="ignore"):
                xc = x0 + (py - y0) * (x1 - x0) / (y1 - y0)
            inside ^= cond & (px < xc)
            ex, ey = x1 - x0, y1 - y0
            t = np.clip(((px - x0) * ex + (py - y0) * ey) / (ex * ex + ey * ey), 0, 1)
            dist = np.minimum(dist, np.hypot(x0 + t * ex - px, y0 + t * ey - py))
    return inside | (dist <= tol)


def _notched_square():
    s = 1 / math.sqrt(2)
    return [np.array([[-s, -s], [s, -s], [s, s], [0.1, s], [0.0, 0.1], [-0.1, s], [-s, s]])]


@pytest.mark.parametrize("case", ["plus8", "plus15", "annulus12", "notch10", "pert0", "pert1", "drop10"])
def test_nonconvex_horizon_matches_sampled_visibility(case):
    """Sec. 4 (set C_x): a bond exists iff the whole segment stays in the grain.
    Compare the oracle's bond lists with dense sampling of every candidate segment."""
    rng = np.random.default_rng(11)
    shapes = {
        "plus8": (I.plus_shape(), 8), "plus15": (I.plus_shape(), 15), "annulus12": (I.annulus_shape(), 12),
        "notch10": (_notched_square(), 10), "pert0": (I.perturbed_disk_shape(rng), 12),
        "pert1": (I.perturbed_disk_shape(np.random.default_rng(3)), 12), "drop10": (I.drop_shape(), 10),
    }
    loops, ratio = shapes[case]
    R = 1e-3
    h = R / ratio
    X, lat = O.mesh_grain(loops, R, h)
    row, col = O.grain_bonds(loops, R, h, lat, 3.0)
    got = {(i, int(j)) for i in range(len(lat)) for j in col[row[i]:row[i + 1]]}
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(lat)}
    ts = np.linspace(0.0, 1.0, 201)
    expected = set()
    n_excluded = 0
    for i, (a, b) in enumerate(lat):
        for dj in range(-3, 4):
            for di in range(-3, 4):
                if (di, dj) == (0, 0) or di * di + dj * dj >= 9:
                    continue
                j = index.get((int(a) + di, int(b) + dj))
                if j is None:
                    continue
                p0 = np.array([a, b], dtype=float) * h
                p1 = np.array([a + di, b + dj], dtype=float) * h
                pts = p0[None, :] + ts[:, None] * (p1 - p0)[None, :]
                if _inside_closed(pts, loops, R, 1e-9 * h).all():
                    expected.add((i, j))
                else:
                    n_excluded += 1
    assert got == expected
    if case not in ("drop10", "plus15"):
        assert n_excluded > 0          # the shape really is non-convex at this mesh
    # plus15: arm half-width 3h puts the re-entrant corners on lattice points; bonds
    # that only touch a corner stay inside the closed grain and must be kept


# ---------------------------------------------------------------------------
# time integration and global invariants


def test_free_fall_is_exact_under_velocity_verlet():
    """Algorithm 1 integrates constant acceleration exactly: u = 1/2 g t^2."""
    h = 1e-4
    prm = _prm(1.0, 0.95 * h, dt=1e-6, g=(0.0, -9.81))
    P = O.OracleProblem(np.array([[0.0, 0.5]]), [h * h], [0], [0, 0], [], [1.0], [1.0], [1.0], prm)
    P.init_accel()
    P.run(1000)
    t = 1000 * 1e-6
    assert P.u[0, 1] == pytest.approx(-0.5 * 9.81 * t * t, rel=1e-12)
    assert P.v[0, 1] == pytest.approx(-9.81 * t, rel=1e-12)


def _colliding_disks(mu, rd, Gc, v=1.0, h_ratio=8):
    w = I.two_disks(h_ratio=h_ratio, gap=0.02e-3, gy=0.0, friction=mu, damping_ratio=rd, Gc=Gc,
                    wall_lo=(-1.0, -1.0), wall_hi=(1.0, 1.0), dt=2e-8)
    h = 1e-3 / h_ratio
    rc = w.params["rc_ratio"] * h
    w.grain_geom[1, 0] = 0.3e-3           # off-centre impact: tangential sliding too
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 2 * (h_ratio - 1) * h + 1.2 * rc   # nodes just apart
    w.grain_geom[1, 5] = -v
    return O.OracleProblem.from_workload(w)


def test_momentum_is_conserved_in_collision_with_damping_and_friction():
    """Equal volumes, no walls, no gravity: all pair forces are antisymmetric."""
    P = _colliding_disks(mu=0.5, rd=0.8, Gc=50.0)
    P.init_accel()
    m = P.prm[O.P_RHO] * P.V
    p0 = (m[:, None] * P.v).sum(axis=0)
    saw_contact = False
    for _ in range(30):
        P.run(100)
        d = P.diagnostics()
        saw_contact |= np.any(P.v[: P.grain_start[1], 1] < -1e-3)
    p1 = (m[:, None] * P.v).sum(axis=0)
    scale = (m * np.abs(P.v).sum(axis=1)).sum()
    assert saw_contact
    assert np.abs(p1 - p0).max() < 1e-12 * scale


def test_energy_is_conserved_in_undamped_elastic_impact():
    """Sec. 4.3 (r_d = 0, mu = 0, no breaking): KE + bond + contact energy is
    conserved up to the O(dt^2) error of velocity Verlet."""
    P = _colliding_disks(mu=0.0, rd=0.0, Gc=1e9)
    P.init_accel()
    d0 = P.diagnostics()
    E0 = d0["KE"] + d0["E_bond"] + d0["E_contact"]
    worst = 0.0
    max_contact = 0.0
    for _ in range(40):
        P.run(50)
        d = P.diagnostics()
        max_contact = max(max_contact, d["E_contact"])
        worst = max(worst, abs(d["KE"] + d["E_bond"] + d["E_contact"] - E0) / E0)
    assert max_contact > 1e-3 * E0
    assert worst < 2e-3


def test_many_grain_collision_keeps_momentum_angular_momentum_and_energy():
    """Six grains (three hexagons, three disks, random orientations) driven
    together at 5 m/s in free space: no walls within reach, no gravity,
    friction, damping or breaking.  Every bond force acts along its deformed
    bond (eq:pmb) and every contact force along the line of centres (Sec. 4.1),
    so all forces are central pair forces.  Velocity Verlet then keeps the total
    linear momentum and the total angular momentum sum m (x cross v) to rounding
    (each half step leaves x cross v unchanged for central forces), and
    KE + bond + contact energy to its O(dt^2) error (Sec. 4.3).  A bond force
    along the reference direction, or a contact force off the line of centres,
    would make the angular momentum drift.  Every grain takes part in the
    collisions."""
    w = I.free_grains(shapes=("hexagon", "disk"), n_per_shape=3, R=1e-3, h_ratio=8, dt=2e-8)
    w.params.update(friction=0.0, damping_ratio=0.0, Gc=1e9, k_bulk=5.0e5, wall_lo=(-1.0, -1.0),
                    wall_hi=(1.0, 1.0))
    c = w.grain_geom[:, :2].copy()
    d = c.mean(axis=0) - c
    w.grain_geom[:, 4:6] = 5.0 * d / np.linalg.norm(d, axis=1)[:, None]
    P = O.OracleProblem.from_workload(w).init_accel()
    m = P.prm[O.P_RHO] * P.V

    def invariants():
        x = P.X + P.u
        mom = (m[:, None] * P.v).sum(axis=0)
        ang = (m * (x[:, 0] * P.v[:, 1] - x[:, 1] * P.v[:, 0])).sum()
        dg = P.diagnostics()
        return mom, ang, dg["KE"] + dg["E_bond"] + dg["E_contact"], dg["E_contact"]

    mom0, ang0, E0, _ = invariants()
    x0 = P.X + P.u
    mom_scale = (m * np.abs(P.v).sum(axis=1)).sum()
    ang_scale = (m * np.hypot(x0[:, 0], x0[:, 1]) * np.hypot(P.v[:, 0], P.v[:, 1])).sum()
    grain_v0 = np.array([P.v[P.grain == g].mean(axis=0) for g in range(w.n_grains)])
    d_mom = d_ang = d_E = max_contact = 0.0
    for _ in range(160):
        P.run(100)
        mom, ang, En, Ec = invariants()
        d_mom = max(d_mom, np.abs(mom - mom0).max() / mom_scale)
        d_ang = max(d_ang, abs(ang - ang0) / ang_scale)
        d_E = max(d_E, abs(En - E0) / E0)
        max_contact = max(max_contact, Ec / E0)
    grain_v = np.array([P.v[P.grain == g].mean(axis=0) for g in range(w.n_grains)])
    assert np.all(np.linalg.norm(grain_v - grain_v0, axis=1) > 0.3 * 5.0)
    assert max_contact > 5e-3
    assert not P.broken.any()
    assert d_mom < 1e-12
    assert d_ang < 1e-12
    assert d_E < 1e-3


def test_grid_search_matches_brute_force():
    """The oracle's cell grid returns the same S^nbr as the O(N^2) definition."""
    P = _colliding_disks(mu=0.5, rd=0.8, Gc=50.0)
    P.init_accel()
    P.run(2000)
    Q = O.OracleProblem(P.X, P.V, P.grain, P.row_ptr, P.col, P.g_cw, P.g_s0, P.g_eps, P.prm.copy(), P.v)
    Q.prm[O.P_SEARCH] = 0.0
    Q.u[:] = P.u
    Q.broken[:] = P.broken
    F1, parts1 = P.forces()
    F2, parts2 = Q.forces()
    assert np.abs(parts1[2]).max() > 0
    assert np.array_equal(F1, F2)


def test_damage_is_monotone_in_fracturing_impact():
    P = _colliding_disks(mu=0.5, rd=0.0, Gc=0.5, v=8.0)
    P.init_accel()
    prev = P.damage()
    grew = False
    for _ in range(40):
        P.run(25)
        dmg = P.damage()
        assert np.all(dmg >= prev)
        grew |= bool(np.any(dmg > prev))
        prev = dmg
    assert grew


# ---------------------------------------------------------------------------
# materials (Sec. 4.1 harmonic-mean bulk modulus; material table of Sec. 5)


def _two_material_nodes(Rc, h, gap, v_rel, mats, rd=0.0):
    """Two single-node grains of materials mats = [(rho1, k1), (rho2, k2)],
    approaching head-on; K_n from the harmonic mean of k1, k2 and eps_c = 3h."""
    V = h * h
    (r1, k1), (r2, k2) = mats
    keff = 2 * k1 * k2 / (k1 + k2) if k1 != k2 else k1
    Kn = O.contact_stiffness(keff, 3 * h)
    mu_red = r1 * r2 * V / (r1 + r2)
    omega = math.sqrt(Kn * V * V / mu_red)
    dt = 0.002 / omega
    prm = _prm(1.0, Rc, rho=1.0, dt=dt, rd=rd)          # the table replaces rho and K_n
    eps = 3 * h
    prm[O.P_PE5] = math.pi * eps * eps * eps * eps * eps
    X = np.array([[0.0, 0.0], [Rc + gap, 0.0]])
    # equal and opposite momenta: the centre of mass is at rest
    v0 = np.array([[v_rel * r2 / (r1 + r2), 0.0], [-v_rel * r1 / (r1 + r2), 0.0]])
    P = O.OracleProblem(X, [V, V], [0, 1], [0, 0, 0], [], [1.0, 1.0], [1.0, 1.0], [1.0, 1.0], prm, v0,
                        g_mat=[[r1, k1], [r2, k2]])
    return P, omega, dt, V


def test_two_materials_contact_is_spring_on_reduced_mass():
    """Grains of densities rho1, rho2 and bulk moduli k1, k2: eq. (law-repulsive)
    with K_n = 18 k / (pi eps^5), k = 2 k1 k2 / (k1 + k2) (Sec. 4.1), is a
    linear spring K_n V^2 on the reduced mass m1 m2 / (m1 + m2): the contact
    lasts pi / omega, momentum is conserved and the relative speed reverses."""
    h, Rc = 1e-4, 0.95e-4
    mats = [(1200.0, 1e6), (4800.0, 3e6)]
    P, omega, dt, V = _two_material_nodes(Rc, h, 1e-9, 0.1, mats)
    m = np.array([mats[0][0] * V, mats[1][0] * V])
    steps = _collide(P, Rc, max_steps=400000)
    assert steps * dt == pytest.approx(math.pi / omega, rel=0.01)
    assert abs(m @ P.v[:, 0]) <= 1e-12 * m[0] * 0.1
    assert P.v[0, 0] - P.v[1, 0] == pytest.approx(-0.1, rel=1e-4)


def test_two_materials_damping_restitution_independent_of_densities():
    """The damping reading (beta_d with the harmonic mean of the two densities)
    keeps the pair's damping ratio at sqrt(2) r_d for any two materials, so the
    restitution is exp(-pi zeta / sqrt(1 - zeta^2)) as for one material."""
    h, Rc, rd = 1e-4, 0.95e-4, 0.1
    P, omega, dt, V = _two_material_nodes(Rc, h, 1e-9, 0.1, [(1200.0, 1e6), (4800.0, 3e6)], rd=rd)
    _collide(P, Rc, max_steps=400000)
    zeta = math.sqrt(2.0) * rd
    e = math.exp(-math.pi * zeta / math.sqrt(1 - zeta ** 2))
    assert -(P.v[0, 0] - P.v[1, 0]) / 0.1 == pytest.approx(e, rel=0.01)


def test_one_material_table_equals_single_material_run():
    """A material table whose every grain has the parameter vector's rho and k
    gives bit-identical forces and trajectories: the harmonic mean of equal
    moduli is the modulus and K_n is formed in the same operation order."""
    w = I.two_disks()
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_geom[0, 1] = 1e-3 + rc * 0.25
    w.grain_geom[1, 1] = w.grain_geom[0, 1] + 16 * h + 1.05 * rc
    w.grain_geom[1, 5] = -1.0
    a = O.OracleProblem.from_workload(w).init_accel()
    p = w.params
    w.materials = (np.array([[p["E"], p["k_bulk"], p["rho"], p["Gc"]]]), np.zeros(w.n_grains, dtype=np.int64))
    b = O.OracleProblem.from_workload(w).init_accel()
    assert b.g_mat is not None
    a.run(200)
    b.run(200)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.v, b.v)
    Fa, _ = a.forces()
    Fb, _ = b.forces()
    assert np.array_equal(Fa, Fb)


# ---------------------------------------------------------------------------
# potential energies of the contact laws (Secs. 4.1, 4.4, 4.5)


@pytest.mark.parametrize("frac", [0.0, 0.2, 0.5, 0.5403, 0.55, 0.9, 0.99, 0.9999])
def test_wall_potential_is_the_integral_of_the_wall_repulsion(frac):
    """W(d) = int_d^{R_c} |S_l(s)| (R_c - |c_l(s) - p|) ds per unit K_n V_x: the
    potential whose derivative is the repulsion of eq. (wall-repulsive), by
    quadrature of the (separately pinned) segment area and centroid."""
    Rc = 1.0e-4
    d = frac * Rc

    def force(s):
        A, c = O.wall_segment(s, Rc)
        return A * (Rc - c)

    val, _ = quad(force, d, Rc, epsabs=0.0, epsrel=1e-13, limit=200)
    assert O.wall_segment_energy(d, Rc) == pytest.approx(val, rel=1e-9)


@pytest.mark.parametrize("theta", [1e-3, 0.05, 0.3, 0.9, 0.999, 1.001, 1.3, math.pi / 2])
def test_wall_potential_matches_50_digit_closed_form(theta):
    """J(theta) = sin th - th cos th - sin^3 th / 3 - th / 4 + sin 2th / 6 - sin 4th / 48
    evaluated with 50 digits at the angle of the rounded d (R_c = 1): the series
    below theta = 1 and the closed form above it both keep full precision,
    including theta -> 0 where J ~ theta^7 / 35 and every closed-form term cancels."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    d = math.cos(theta)
    th = mp.acos(mp.mpf(d))
    J = mp.sin(th) - th * mp.cos(th) - mp.sin(th) ** 3 / 3 - th / 4 + mp.sin(2 * th) / 6 - mp.sin(4 * th) / 48
    assert O.wall_segment_energy(d, 1.0) == pytest.approx(float(J), rel=1e-12)
    if theta == math.pi / 2:
        assert O.wall_segment_energy(0.0, 1.0) == pytest.approx(2.0 / 3.0 - math.pi / 8.0, rel=1e-15)


def test_self_contact_energy_falls_by_the_work_of_the_self_contact_force():
    """E_self of a compressed unbonded same-grain pair (both branches) changes by
    minus the work of the self-contact force along a small separation step."""
    h, Rc = 1e-4, 0.95e-4
    Kn = O.contact_stiffness(1e6, 3 * h)
    for xi, d in ((0.5 * Rc, 0.3 * Rc), (2.0 * Rc, 0.6 * Rc)):
        P, _ = _self_pair(xi, Rc, Kn, d)
        e0 = P.energies()["E_self"]
        F, _ = P.forces()
        delta = 1e-6 * Rc
        P.u[1, 0] += delta                      # node 1 moves away along +x
        e1 = P.energies()["E_self"]
        work = F[1, 0] * delta                  # force on node 1 along the move
        assert e0 > 0 and (e0 - e1) == pytest.approx(work, rel=1e-5)


def test_energy_is_conserved_for_a_grain_bouncing_on_the_floor():
    """Sec. 4.3 energy identity with the wall (r_d = 0, mu = 0, no breaking): a
    disk dropped on the floor under gravity conserves kinetic + bond + wall +
    gravitational energy to the O(dt^2) error of velocity Verlet, and the wall
    energy really takes part (it peaks at a sizeable share)."""
    w = I.two_disks(gy=-5000.0, friction=0.0, damping_ratio=0.0, Gc=1e9, dt=2e-8)
    h = 1e-3 / 8
    rc = w.params["rc_ratio"] * h
    w.grain_shape = w.grain_shape[:1]
    w.grain_geom = w.grain_geom[:1].copy()
    low = O.OracleProblem.from_workload(w).positions[:, 1].min()
    w.grain_geom[0, 1] += 1.02 * rc - low          # lowest nodes 1.02 R_c above the floor
    w.grain_geom[0, 5] = -1.0
    P = O.OracleProblem.from_workload(w)
    P.init_accel()
    m = P.prm[O.P_RHO] * P.V

    def total():
        d = P.diagnostics()
        e = P.energies()
        grav = -np.sum(m * (P.prm[O.P_GX] * P.positions[:, 0] + P.prm[O.P_GY] * P.positions[:, 1]))
        return d["KE"] + d["E_bond"] + e["E_wall"] + e["E_self"] + grav, e["E_wall"]

    E0, _ = total()
    ke0 = P.diagnostics()["KE"]
    worst, peak = 0.0, 0.0
    for _ in range(40):
        P.run(100)
        Et, ew = total()
        peak = max(peak, ew)
        worst = max(worst, abs(Et - E0) / ke0)
    assert peak > 0.05 * ke0
    assert worst < 1e-4
    assert P.v[:, 1].mean() > 0.9                  # it bounced back up


def test_all_core_build_is_bitwise_the_single_threaded_one():
    """The OpenMP build of the oracle splits the node loop over host threads and
    changes no arithmetic: a fracturing, contacting run is bitwise identical."""
    a = _colliding_disks(mu=0.5, rd=0.8, Gc=0.5, v=6.0)
    b = _colliding_disks(mu=0.5, rd=0.8, Gc=0.5, v=6.0)
    b.omp = True
    a.init_accel()
    b.init_accel()
    Fa, pa = a.run(1500, want_parts=True)
    Fb, pb = b.run(1500, want_parts=True)
    assert a.broken.sum() > 0
    assert np.array_equal(a.u, b.u) and np.array_equal(a.v, b.v) and np.array_equal(Fa, Fb)
    assert np.array_equal(pa, pb) and np.array_equal(a.broken, b.broken)
    assert np.array_equal(a.status, b.status)

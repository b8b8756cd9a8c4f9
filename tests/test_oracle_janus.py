"""Pins of the oracle's Janus wettability (CPU only).

The paper's colloid benchmarks (Sec. 5.1; App. A, the MD room's
wettability-angle directive; App. D input) give each particle a wettability
that depends on the polar angle theta between a surface node and the
particle's first body axis x*, switched smoothly from -1 to 1 over a width
around theta0 (108 and 10 degrees there).  The oracle's reading: the switch
s(theta) multiplies zeta^A and -zeta^B in Eq. 20.  Pinned here against what
holds independently of the oracle's code:
  * switch saturated (theta0 far outside [0, 180]): the run is the plain run
    with wetting constants (-zeta^A, zeta^B) or (zeta^A, -zeta^B), bit for
    bit (the component sign rule);
  * the virtual densities of the frontier nodes against the body axis taken
    from scipy's rotation of the quaternion (the frame convention of
    Eq. 31): wetting -zeta on the cap around x*, +zeta on the far cap,
    monotone across the switch, and -s zeta^B with s zeta^A on every node;
  * a 90 degree lattice rotation of the whole system, quaternion included,
    maps the particle force and torque onto themselves;
  * at a flat A/B interface the wetting torque turns the axis toward the
    phase its cap prefers, and vanishes when the axis is aligned.
"""
import math

import numpy as np
import pytest

from oracle import Oracle, lattice

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def quat_wxyz(rot):
    x, y, z, w = rot.as_quat()
    return np.array([w, x, y, z])


def janus_run(shape, zeta, theta0, width, quat, pos, steps, dens=None, vel=None, omega=None, G=0.6, janus=1):
    o = Oracle(*shape, 2)
    o.set_params(G=G, tau=(1.0, 1.0), zeta=zeta, janus=janus, janus_theta0=theta0, janus_width=width,
                 hertz_K=10.0, hertz_sigma=8.0, hertz_rcap=7.0)
    N = int(np.prod(shape))
    if dens is None:
        rng = np.random.default_rng(11)
        a = 0.5 + 0.02 * rng.standard_normal(N)
        dens = (a, 1.0 - a)
    o.init_fields(*dens)
    o.add_colloids(pos, [3.4] * len(pos), [400.0] * len(pos), vel=vel, omega=omega, quat=quat)
    o.step(steps)
    return o


def test_saturated_switch_is_the_plain_rule_with_component_signs():
    """theta0 beyond 180 + width/2: s = -1 on every node, the wetting
    constants become (-zeta^A, +zeta^B); theta0 below -width/2: s = +1, they
    become (zeta^A, -zeta^B).  Two moving, rotating particles, 12 steps."""
    shape = (18, 16, 14)
    pos = [[5.3, 6.2, 6.9], [12.6, 9.1, 7.4]]
    q = [quat_wxyz(Rotation.from_rotvec([0.3, -0.5, 0.8])), quat_wxyz(Rotation.from_rotvec([-1.1, 0.2, 0.4]))]
    kw = dict(vel=[[0.02, -0.01, 0.0], [-0.01, 0.02, 0.01]], omega=[[0.0, 0.02, 0.01], [0.03, 0.0, -0.01]])
    za, zb = 0.12, 0.07
    for theta0, plain in ((400.0, (-za, zb)), (-300.0, (za, -zb))):
        j = janus_run(shape, (za, zb), theta0, 10.0, q, pos, 12, **kw)
        p = janus_run(shape, plain, 0.0, 0.0, q, pos, 12, janus=0, **kw)
        for k in (0, 1):
            assert np.array_equal(j.populations(k), p.populations(k))
        cj, cp = j.get_colloids(), p.get_colloids()
        for key in ("pos", "vel", "omega", "quat"):
            assert np.array_equal(cj[key], cp[key]), key


def test_frontier_wetting_follows_the_body_axis():
    """Eq. 20 with the switch: on every frontier node psi^k / rhobar^k - 1 is
    the node's wetting constant; against the angle to the body axis
    R(q) e_x computed by scipy: -zeta^A below theta0 - w/2, +zeta^A above
    theta0 + w/2, nondecreasing in theta in between, and the B constant is
    minus the A constant times zeta^B / zeta^A on every node."""
    shape = (20, 20, 20)
    c, w, _ = lattice()
    rot = Rotation.from_rotvec([0.4, 1.1, -0.7])
    r_p = np.array([9.6, 10.3, 9.8])
    za, zb, theta0, width = 0.2, 0.1, 108.0, 10.0
    o = janus_run(shape, (za, zb), theta0, width, [quat_wxyz(rot)], [r_p], 0)
    ra, rb, _ = o.get_fields()  # evaluates the forces on the current map
    owner = o.owner()
    psi = [o.psi(0), o.psi(1)]
    nx, ny, nz = shape
    axis = rot.apply([1.0, 0.0, 0.0])
    found = []
    for s in np.nonzero(owner == 0)[0]:
        x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
        num = np.zeros(2)
        den = 0.0
        for i in range(1, 19):
            n = ((x + c[i, 0]) % nx) + nx * (((y + c[i, 1]) % ny) + ny * ((z + c[i, 2]) % nz))
            if owner[n] < 0:
                num += w[i] * np.array([ra[n], rb[n]])
                den += w[i]
        if den == 0.0:
            continue
        zeff = np.array([psi[0][s], psi[1][s]]) / (num / den) - 1.0
        d = np.array([x, y, z], dtype=float) - r_p
        theta = math.degrees(math.acos(np.clip(axis @ d / np.linalg.norm(d), -1.0, 1.0)))
        found.append((theta, zeff[0] / za, zeff[1] / zb))
    found.sort()
    th = np.array([f[0] for f in found])
    sa = np.array([f[1] for f in found])
    sb = np.array([f[2] for f in found])
    assert len(found) > 100 and th.min() < theta0 - width and th.max() > theta0 + width
    lo, hi = th < theta0 - width / 2, th > theta0 + width / 2
    assert np.allclose(sa[lo], -1.0, atol=1e-12) and np.allclose(sa[hi], 1.0, atol=1e-12)
    mid = ~lo & ~hi
    assert mid.sum() >= 5 and np.all(np.abs(sa[mid]) < 1.0)
    assert np.all(np.diff(sa) >= -1e-12)
    assert np.allclose(sb, -sa, atol=1e-12)


def test_lattice_rotation_maps_the_janus_run_onto_itself():
    """Rotate the box, the fields, the particle and its orientation by 90
    degrees about z (x -> y, y -> -x): the particle's force and torque after
    8 steps rotate with it (to roundoff)."""
    n = 16
    shape = (n, n, n)
    N = n ** 3
    rng = np.random.default_rng(5)
    a = (0.5 + 0.03 * rng.standard_normal(N)).reshape(n, n, n)  # [z][y][x]
    b = 1.0 - a
    rot = Rotation.from_rotvec([0.5, -0.3, 0.9])
    r_p = np.array([7.3, 8.1, 7.6])
    R90 = Rotation.from_rotvec([0.0, 0.0, math.pi / 2])

    def run(dA, dB, r, q):
        o = Oracle(*shape, 1)
        o.set_params(G=0.6, tau=(1.0, 1.0), zeta=(0.15, 0.1), janus=1, janus_theta0=100.0, janus_width=20.0)
        o.init_fields(dA.ravel(), dB.ravel())
        o.add_colloids([r], [3.6], [math.inf], quat=[q])
        o.step(8)
        return o.term("F_s")[0], o.term("T_s")[0], o.term("F_liq")[0], o.term("T_liq")[0]

    base = run(a, b, r_p, quat_wxyz(rot))
    # new[z][y'][x'] = old[z][y][x] with x' = n - y, y' = x (mod n): the site
    # (x, y) goes to (-y, x), a rotation by +90 degrees about z with the
    # lattice origin fixed
    def rot_field(f):
        g = np.empty_like(f)
        for y in range(n):
            for x in range(n):
                g[:, x, (-y) % n] = f[:, y, x]
        return g

    r_new = np.array([(-r_p[1]) % n, r_p[0], r_p[2]])
    turned = run(rot_field(a), rot_field(b), r_new, quat_wxyz(R90 * rot))
    for u, v in zip(base, turned):
        expect = R90.apply(u)
        assert np.abs(v - expect).max() <= 1e-10 * max(np.abs(u).max(), 1e-12), (u, v, expect)
    assert np.abs(base[1]).max() > 1e-6  # the wetting torque is not trivially zero


def test_wetting_torque_turns_the_axis_toward_its_phase():
    """An immobile half-and-half particle (theta0 = 90, width 10) centred on
    a flat A/B interface normal to z, A-rich below: the cap around x* wets B
    (its constants are -zeta^A, +zeta^B with zeta = (0.1, 0.1)), so the
    wetting torque turns x* toward +z: for a tilt alpha of x* from +z in the
    x-z plane, T_y < 0 (rotating x* back toward z), and the torque vanishes
    (to roundoff against the tilted case) at alpha = 0."""
    shape = (20, 20, 32)
    nx, ny, nz = shape
    zc = np.repeat(np.arange(nz), nx * ny).astype(float)
    # B-rich between the interfaces at z = 15.5 and 31.5 (periodic), A-rich
    # elsewhere, between the coexistence densities of the demixing mixture
    # (rho0 = 1 per component, G = 0.65)
    prof = 0.5 * (np.tanh((zc - 15.5) / 2.0) - np.tanh((zc - 31.5) / 2.0))
    rich, poor = 1.8, 0.25
    rb = poor + (rich - poor) * prof
    ra = rich + poor - rb

    def torque(alpha_deg):
        # x* = (sin a, 0, cos a): rotate e_x onto it
        ax = np.array([math.sin(math.radians(alpha_deg)), 0.0, math.cos(math.radians(alpha_deg))])
        rot, _ = Rotation.align_vectors([ax], [[1.0, 0.0, 0.0]])
        o = Oracle(*shape, 1)
        o.set_params(G=0.65, tau=(1.0, 1.0), rho0=(1.0, 1.0), zeta=(0.1, 0.1), janus=1, janus_theta0=90.0,
                     janus_width=10.0)
        o.init_fields(ra, rb)
        o.add_colloids([[10.0, 10.0, 15.5]], [4.5], [math.inf], quat=[quat_wxyz(rot)])
        o.step(60)
        return o.term("T_s")[0] + o.term("T_liq")[0]

    t30, t0 = torque(30.0), torque(0.0)
    assert t30[1] < 0.0
    assert abs(t30[1]) > 10 * max(abs(t30[0]), abs(t30[2]))
    assert np.abs(t0).max() < 1e-6 * abs(t30[1])

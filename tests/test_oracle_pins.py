"""Pins of the FP64 oracle against what the paper and lattice-Boltzmann theory
fix, independently of the oracle's own code (CPU only).

Each test names the passage it pins.  A plausible slip in the oracle (a
dropped term, a flipped sign, a wrong index or weight) fails at least one:
  * lattice isotropy and equilibrium moments pin the D3Q19 table and Eq. 5;
  * mass / momentum conservation pin Eqs. 3, 6-7, 11 (sign), 13-16;
  * shear-wave decay pins the viscosity of Eq. 4;
  * Couette pins the moving-wall bounce-back of Eq. 9;
  * Poiseuille pins the forcing (Eqs. 15-16) with the halfway bounce-back;
  * the composition-mode threshold pins the Shan-Chen coupling (Eqs. 11-12);
  * the particle momentum budget pins Eqs. 17-19, 22, 24, 25, 35;
  * closed forms pin the integrator (Eqs. 32-34) and the Hertz force (Eq. 26);
  * exact symmetries pin the wetting and component bookkeeping (Eqs. 20-21).
"""
import math

import numpy as np
import pytest

from oracle import Oracle, feq, integrate_one, lattice, pair_force

CS2 = 1.0 / 3.0


def make(shape, max_colloids=4, **params):
    o = Oracle(*shape, max_colloids)
    o.set_params(**params)
    return o


def zcoord(shape):
    nx, ny, nz = shape
    return np.repeat(np.arange(nz), nx * ny)


# --------------------------------------------------------------- lattice
def test_d3q19_isotropy():
    """Sec. 2.1: D3Q19 with w0=1/3, w1-6=1/18, w7-18=1/36 and cs^2=1/3 has the
    isotropic moments up to fourth order that the 2nd-order equilibrium needs."""
    c, w, opp = lattice()
    c = c.astype(float)
    sq = (c * c).sum(1)
    assert sorted(sq.tolist()) == [0] + [1] * 6 + [2] * 12
    for s, wt in ((0, 1 / 3), (1, 1 / 18), (2, 1 / 36)):
        assert np.all(np.abs(w[sq == s] - wt) < 1e-16)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ c, 0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, CS2 * np.eye(3), atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(M3, 0, atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(M4, iso, atol=1e-15)
    for i in range(19):
        assert np.all(c[opp[i]] == -c[i])


def test_equilibrium_moments():
    """Eq. 5 reproduces rho (Eq. 6), rho u (Eq. 7) and the Euler stress
    rho (cs^2 I + u u) exactly; its third moment is rho cs^2 (u d + ...)
    minus the missing u^3 term that D3Q19 cannot carry."""
    c, w, _ = lattice()
    c = c.astype(float)
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho = rng.uniform(0.1, 3.0)
        u = rng.uniform(-0.1, 0.1, 3)
        f = feq(rho, u)
        assert abs(f.sum() - rho) < 1e-14 * rho
        assert np.allclose(f @ c, rho * u, rtol=0, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.allclose(P, rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-15)
        # the diagonal third moment sum_i f c_a^3 = rho cs^2 * 3 u_a... D3Q19 has
        # c_a^3 = c_a, so sum f c_a^3 = rho u_a exactly
        assert np.allclose(np.einsum("i,ia->a", f, c ** 3), rho * u, atol=1e-15)


# --------------------------------------------------------- conservation
def test_mass_conserved_periodic_and_walls():
    """Eqs. 3, 8, 9, 16: collision, streaming and (moving) halfway bounce-back
    conserve each component's mass to roundoff."""
    shape = (12, 10, 9)
    N = int(np.prod(shape))
    rng = np.random.default_rng(1)
    a = 0.5 * (1 + 0.01 * rng.uniform(-1, 1, N))
    b = 1.0 - a
    for kw in (dict(), dict(bc=(1, 1, 0), wall_u_lo=(-0.03, 0.01, 0), wall_u_hi=(0.05, -0.02, 0),
                            body_force=(1e-5, 0, 0))):
        o = make(shape, G=0.65, tau=(0.8, 1.3), **kw)
        o.init_fields(a, b)
        m0 = o.totals()[:2]
        o.step(40)
        m1 = o.totals()[:2]
        assert np.all(np.abs(m1 - m0) / m0 < 1e-13), (kw, m1 - m0)


def test_momentum_conserved_with_shan_chen():
    """Eq. 11 with the repulsive sign is a pairwise force: summed over a
    periodic box it cancels, so with equal tau the EDM collision (Eq. 16)
    conserves the total momentum to roundoff."""
    shape = (10, 9, 8)
    N = int(np.prod(shape))
    rng = np.random.default_rng(2)
    a = 0.5 * (1 + 0.05 * rng.uniform(-1, 1, N))
    b = 0.5 * (1 - 0.05 * rng.uniform(-1, 1, N))
    u = np.zeros((3, N))
    u[0] = 0.01 + 0.002 * rng.uniform(-1, 1, N)
    u[2] = -0.005
    o = make(shape, G=0.9, tau=(0.8, 0.8))
    o.init_fields(a, b, u)
    p0 = o.totals()[2:5]
    o.step(40)
    t = o.totals()
    assert np.all(np.abs(t[2:5] - p0) < 1e-13 * np.abs(p0).max()), t[2:5] - p0
    # the half-force corrected momentum carries the same total
    assert np.all(np.abs(t[5:8] - p0) < 1e-13 * np.abs(p0).max())


# ----------------------------------------------------------- viscosity
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_shear_wave_viscosity(tau):
    """Eq. 4: a transverse wave u_x = U sin(kz) decays at rate nu k^2 with
    nu = cs^2 (tau - 1/2); the lattice error is O(k^2) (O(k^4) at tau = 1)."""
    errs = []
    for L in (16, 32):
        shape = (4, 4, L)
        N = 16 * L
        z = zcoord(shape)
        k = 2 * math.pi / L
        u = np.zeros((3, N))
        u[0] = 1e-4 * np.sin(k * z)
        o = make(shape, tau=(tau, tau))
        o.init_fields(np.full(N, 0.5), np.full(N, 0.5), u)
        nu = CS2 * (tau - 0.5)
        T = int(0.5 / (nu * k * k))
        o.step(20)
        A1 = 2 * np.mean(o.get_fields()[2][0] * np.sin(k * z))
        o.step(T)
        A2 = 2 * np.mean(o.get_fields()[2][0] * np.sin(k * z))
        errs.append(-math.log(A2 / A1) / T / (nu * k * k) - 1)
    assert abs(errs[1]) < 0.011
    assert abs(errs[1]) < abs(errs[0]) / 3.5  # second-order convergence


# ---------------------------------------------------------------- walls
@pytest.mark.parametrize("tau", [0.8, 1.7])
def test_couette_linear_profile(tau):
    """Eq. 9: walls at z=-1/2 and z=H-1/2 moving at -U and +U give the exact
    linear profile u_x = U (2 (z+1/2)/H - 1) at steady state (BGK reproduces
    linear shear without lattice error)."""
    H, U = 12, 0.01
    shape = (4, 4, H)
    N = 16 * H
    z = zcoord(shape)
    o = make(shape, tau=(tau, tau), bc=(1, 1, 0), wall_u_lo=(-U, 0, 0), wall_u_hi=(U, 0, 0), G=0.3)
    o.init_fields(np.full(N, 0.5), np.full(N, 0.5))
    nu = CS2 * (tau - 0.5)
    o.step(int(32 / (nu * (math.pi / H) ** 2)))
    a, b, u = o.get_fields()
    assert np.max(np.abs(u[0] - U * (2 * (z + 0.5) / H - 1))) < 1e-12 * U
    assert np.max(np.abs(u[1:])) < 1e-13
    assert np.max(np.abs(a - 0.5)) < 1e-12


def test_poiseuille_profile():
    """Eqs. 8, 15-16 with a body force g: at tau = 1/2 + sqrt(3/16) halfway
    bounce-back gives the analytic parabola u = g/(2 nu) (z+1/2)(H-1/2-z)
    exactly; at tau = 1 the error is O(H^-2)."""
    g = 1e-6
    out = {}
    for tau in (0.5 + math.sqrt(3.0 / 16.0), 1.0):
        for H in (8, 16):
            shape = (4, 4, H)
            N = 16 * H
            z = zcoord(shape)
            o = make(shape, tau=(tau, tau), bc=(1, 1, 0), body_force=(g, 0, 0))
            o.init_fields(np.full(N, 0.5), np.full(N, 0.5))
            nu = CS2 * (tau - 0.5)
            o.step(int(34 / (nu * (math.pi / H) ** 2)))
            ex = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
            out[(tau, H)] = np.max(np.abs(o.get_fields()[2][0] - ex)) / ex.max()
    tm = 0.5 + math.sqrt(3.0 / 16.0)
    assert out[(tm, 8)] < 1e-10 and out[(tm, 16)] < 1e-10
    assert 1e-3 < out[(1.0, 8)] < 1e-2
    assert 3.5 < out[(1.0, 8)] / out[(1.0, 16)] < 4.5


# ------------------------------------------------------------ Shan-Chen
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_composition_mode_threshold(tau):
    """Eqs. 11-12 with the EDM source: a long composition wave of a 50/50
    mixture relaxes with D = cs^2 [(tau - 1/2) - tau G rho / 2] (second-order
    expansion of streaming plus the force entering the post-collision flux),
    so demixing starts at G rho = 2 - 1/tau; at tau = 1 this is the paper's
    G_crit = 1/(rho^k + rho^kbar) (Sec. 2.3)."""
    Gc = 2.0 - 1.0 / tau
    L = 32
    shape = (L, 4, 4)
    x = np.tile(np.arange(L), 16)
    c = np.cos(2 * np.pi * x / L)
    rates = []
    for f in (0.9, 1.1):
        o = make(shape, G=f * Gc, tau=(tau, tau))
        o.init_fields(0.5 * (1 + 1e-4 * c), 0.5 * (1 - 1e-4 * c))
        o.step(30)
        a, b, _ = o.get_fields()
        A1 = np.mean((a - b) * c)
        o.step(200)
        a, b, _ = o.get_fields()
        rates.append(math.log(np.mean((a - b) * c) / A1) / 200)
    assert rates[0] < 0 < rates[1]
    # growth rate for G = 0 is the ideal mutual diffusion cs^2 (tau - 1/2) k^2
    k2 = (2 * np.pi / L) ** 2
    predicted = [CS2 * ((tau - 0.5) - tau * f * Gc / 2) * k2 for f in (0.9, 1.1)]
    for r, p in zip(rates, predicted):
        assert abs(-r - p) < 0.2 * abs(p)  # leading order in k; O(k^4) terms remain


def test_uniform_state_is_fixed_point():
    """A uniform mixture at rest with a neutrally wetting sphere centred on a
    lattice-symmetric point feels no Shan-Chen force (Eqs. 11, 20, 21 with
    zeta = 0 and cubic symmetry): nothing moves."""
    shape = (16, 16, 16)
    N = 16 ** 3
    o = make(shape, G=0.65, hertz_K=20, hertz_sigma=10, hertz_rcap=9)
    o.init_fields(np.full(N, 0.4), np.full(N, 0.6))
    o.add_colloids([[8.0, 8.0, 8.0]], 4.5, 400.0)
    o.step(10)
    a, b, u = o.get_fields()
    fl = o.owner() < 0
    assert np.max(np.abs(a[fl] - 0.4)) < 1e-14 and np.max(np.abs(b[fl] - 0.6)) < 1e-14
    assert np.max(np.abs(u)) < 1e-15
    col = o.get_colloids()
    assert np.max(np.abs(col["vel"])) < 1e-15 and np.max(np.abs(col["omega"])) < 1e-15


# ------------------------------------------------------------ particles
def _moving_particle_run(G, zeta=(0.0, 0.0), steps=60):
    shape = (16, 14, 15)
    N = int(np.prod(shape))
    rng = np.random.default_rng(5)
    a = 0.5 * (1 + 0.01 * rng.uniform(-1, 1, N))
    b = 1.0 - a
    o = make(shape, G=G, zeta=zeta, tau=(1.0, 1.0))
    o.init_fields(a, b)
    o.add_colloids([[7.3, 6.8, 7.1]], 3.6, 60.0, vel=[[0.03, -0.02, 0.025]], omega=[[0.0, 0.01, -0.02]])
    return o, steps


def test_particle_momentum_budget():
    """Eqs. 17-19, 22, 24, 25, 35 together: bounce-back hands the particle
    exactly what the fluid loses, covered nodes hand over their momentum and
    refilled nodes take theirs from the particle, so with G = 0
    Pi(t) = P_fluid(t) + m v(t-1/2) + F_liq(t-1/2)/2 is conserved to roundoff
    while the particle crosses many nodes."""
    o, steps = _moving_particle_run(G=0.0)
    m = 60.0
    pis = []
    events = 0
    for t in range(steps):
        o.step(1)
        col = o.get_colloids()
        pf = o.totals()[2:5]
        fl = o.term("F_liq")[0]
        pis.append(pf + m * col["vel"][0] + 0.5 * fl)
        events += np.any(o.term("F_d") != 0) + np.any(o.term("F_c") != 0)
    pis = np.array(pis)
    assert events > 10  # the particle really moved across nodes
    assert np.max(np.abs(pis - pis[0])) < 1e-13 * m * 0.03


def test_particle_mass_change_matches_bounce_back():
    """Eq. 17 with a moving particle changes the fluid mass only through the
    -2 w_i rho (u_w.c_i)/cs^2 term and node events; with the particle at rest
    the mass is conserved to roundoff (the rule reduces to Eq. 8)."""
    shape = (14, 14, 14)
    N = 14 ** 3
    rng = np.random.default_rng(6)
    a = 0.5 * (1 + 0.01 * rng.uniform(-1, 1, N))
    o = make(shape, G=0.65, tau=(1.0, 1.0))
    o.init_fields(a, 1 - a)
    o.add_colloids([[6.5, 7.0, 7.2]], 4.0, math.inf)  # infinite mass: never moves
    m0 = o.totals()[:2]
    o.step(30)
    m1 = o.totals()[:2]
    assert np.all(np.abs(m1 - m0) / m0 < 1e-13)


def test_exact_symmetries():
    """Component exchange A<->B with zeta -> swapped, and an integer periodic
    translation, map a particle-laden run onto itself (Eqs. 11, 14, 20, 21 treat
    the components and the lattice sites alike)."""
    shape = (14, 13, 12)
    N = int(np.prod(shape))
    rng = np.random.default_rng(7)
    a = 0.5 * (1 + 0.02 * rng.uniform(-1, 1, N))
    b = 0.5 * (1 - 0.02 * rng.uniform(-1, 1, N))
    pos = np.array([[6.2, 6.7, 5.9]])
    vel = np.array([[0.01, 0.02, -0.015]])
    base = dict(G=0.65, hertz_K=20, hertz_sigma=10, hertz_rcap=9)

    def run(ra, rb, zeta, p):
        o = make(shape, zeta=zeta, **base)
        o.init_fields(ra, rb)
        o.add_colloids(p, 4.0, 300.0, vel=vel)
        o.step(25)
        return o.get_fields(), o.get_colloids()

    (fa, fb, fu), c0 = run(a, b, (0.2, -0.2), pos)
    (ga, gb, gu), c1 = run(b, a, (-0.2, 0.2), pos)
    assert np.max(np.abs(ga - fb)) < 1e-14 and np.max(np.abs(gb - fa)) < 1e-14
    assert np.max(np.abs(gu - fu)) < 1e-14
    assert np.max(np.abs(c1["pos"] - c0["pos"])) < 1e-13
    # translate by (3, 5, 2) sites
    sh = (3, 5, 2)
    A = a.reshape(shape[::-1])
    B = b.reshape(shape[::-1])
    At = np.roll(A, (sh[2], sh[1], sh[0]), axis=(0, 1, 2)).ravel()
    Bt = np.roll(B, (sh[2], sh[1], sh[0]), axis=(0, 1, 2)).ravel()
    (ha, hb, hu), c2 = run(At, Bt, (0.2, -0.2), pos + np.array(sh))
    back = lambda v: np.roll(v.reshape(shape[::-1]), (-sh[2], -sh[1], -sh[0]), axis=(0, 1, 2)).ravel()
    assert np.max(np.abs(back(ha) - fa)) < 1e-13
    assert np.max(np.abs(back(hu[0]) - fu[0])) < 1e-13
    assert np.max(np.abs(c2["pos"] - np.array(sh) - c0["pos"])) < 1e-12
    # the wetting term matters: zeta != 0 changes the run
    (ka, kb, ku), c3 = run(a, b, (0.0, 0.0), pos)
    assert np.max(np.abs(ka - fa)) > 1e-6


def test_wetting_prefers_component():
    """Eq. 20: zeta^A > 0 fills the particle frontier with extra A density,
    and by Eq. 11 (repulsive G) the surrounding fluid is enriched in A."""
    shape = (16, 16, 16)
    N = 16 ** 3
    o = make(shape, G=0.5, zeta=(0.3, -0.3))
    o.init_fields(np.full(N, 0.5), np.full(N, 0.5))
    o.add_colloids([[8.0, 8.0, 8.0]], 4.5, math.inf)
    o.step(40)
    a, b, _ = o.get_fields()
    s = np.arange(N)
    x, y, z = s % 16, (s // 16) % 16, s // 256
    r = np.sqrt((x - 8) ** 2 + (y - 8) ** 2 + (z - 8) ** 2)
    shell = (r >= 4.5) & (r < 6.0)
    far = r > 7.5
    assert (a[shell] - b[shell]).mean() > 1e-3
    assert (a[shell] - b[shell]).mean() > 5 * abs((a[far] - b[far]).mean())


# ---------------------------------------------------------- integrator
def test_leapfrog_translation_closed_form():
    """Eq. 32: with a constant force the leap-frog gives
    r(t) = r0 + t v0 + (F/m) t(t+1)/2 exactly (v0 = v(-1/2))."""
    r0 = np.array([3.0, 4.0, 5.0])
    v0 = np.array([0.01, -0.02, 0.005])
    F = np.array([0.3, -0.1, 0.2])
    m = 50.0
    r, v, w, q = r0, v0, np.zeros(3), np.array([1.0, 0, 0, 0])
    for t in range(1, 41):
        r, v, w, q = integrate_one(r, v, w, q, m, 3.0, F, np.zeros(3))
        assert np.allclose(r, r0 + t * v0 + F / m * t * (t + 1) / 2, rtol=0, atol=1e-12)
        assert np.allclose(v, v0 + t * F / m, atol=1e-15)


def test_svanberg_quaternion_closed_form():
    """Eqs. 33-34 with a constant angular velocity: the converged implicit
    mid-step is the Cayley map, q(t+1) = (1 + W/4)(1 - W/4)^-1 q(t) with
    W = (0, omega) acting from the left, i.e. a rotation by 4 atan(|omega|/4)
    per step about omega; q stays a unit quaternion."""
    rng = np.random.default_rng(11)
    q0 = rng.normal(size=4)
    q0 /= np.linalg.norm(q0)
    omega = np.array([0.03, -0.05, 0.02])
    wn = np.linalg.norm(omega)
    phi = 2 * math.atan(wn / 4)
    n = omega / wn

    def qmul(a, b):
        return np.array([a[0] * b[0] - a[1:] @ b[1:],
                         *(a[0] * b[1:] + b[0] * a[1:] + np.cross(a[1:], b[1:]))])

    r, v, w, q = np.zeros(3), np.zeros(3), omega.copy(), q0.copy()
    for t in range(1, 101):
        r, v, w, q = integrate_one(r, v, w, q, 10.0, 2.0, np.zeros(3), np.zeros(3))
        C = np.array([math.cos(t * phi), *(math.sin(t * phi) * n)])
        assert np.allclose(q, qmul(C, q0), atol=1e-12)
    # a constant torque changes omega linearly with I = 2/5 m R^2
    T = np.array([0.1, 0.0, -0.2])
    r, v, w, q = integrate_one(np.zeros(3), np.zeros(3), omega, q0, 10.0, 2.0, np.zeros(3), T)
    assert np.allclose(w, omega + T / (0.4 * 10.0 * 4.0), atol=1e-15)


def test_hertz_force_is_potential_gradient():
    """Eq. 26: the contact force is minus the gradient of K (sigma - r)^{5/2}
    (checked by a central difference of the potential), repulsive, zero beyond
    sigma and capped below r_cap."""
    K, sigma, rcap = 20.0, 12.0, 11.0
    pr = dict(hertz_K=K, hertz_sigma=sigma, hertz_rcap=rcap)
    U = lambda r: K * (sigma - r) ** 2.5
    d = np.array([0.6, -0.3, 0.74])
    d /= np.linalg.norm(d)
    for r in (11.2, 11.5, 11.9):
        F = pair_force(r * d, 5.5, 5.5, **pr)
        h = 1e-5
        dUdr = (U(r + h) - U(r - h)) / (2 * h)
        assert np.allclose(F, dUdr * d, rtol=1e-8)  # F on i = +dU/dr * r_ij/r: away from j
        assert F @ d < 0
    assert np.all(pair_force(12.5 * d, 5.5, 5.5, **pr) == 0)
    assert np.allclose(pair_force(10.0 * d, 5.5, 5.5, **pr), pair_force(11.0 * d, 5.5, 5.5, **pr))


def test_moving_particle_mass_budget_exact():
    """Eqs. 17, 24, 25 with reading c10: while two rotating particles move
    through a demixing-capable mixture, destroying and creating nodes, the
    fluid mass of each component changes per step by exactly
        - sum over destroyed nodes of rho^k (their fluid is removed, Eq. 24)
        + sum over created nodes of rhobar^k (Eq. 25: f = f^eq(rhobar, u_w),
          rhobar the w_i-weighted mean over neighbours fluid before and
          after the remap, rho0^k if there is none)
        - sum over bounce-back links (x, i) of 6 w_i rho^k(x) c_i . u_w (Eq. 17),
    u_w = v_p + omega_p x (x + c_i/2 - r_p) the rigid-body velocity of Eq. 18
    (reading c6) at v(t-1/2), omega(t-1/2); streaming and the collision
    (Eqs. 3, 13-16) conserve it.  The right-hand side is formed here from the
    observable state alone (fields, node maps and particle state before and
    after each step), so a slip in the refill weights, the destroy set, the
    wall-velocity term or its rotation sign breaks the identity."""
    shape = (20, 18, 16)
    nx, ny, nz = shape
    N = nx * ny * nz
    rng = np.random.default_rng(5)
    a = 0.5 * (1 + 0.05 * rng.uniform(-1, 1, N))
    b = 0.5 * (1 - 0.05 * rng.uniform(-1, 1, N))
    params = dict(G=0.5, zeta=(0.1, -0.1), hertz_K=20, hertz_sigma=9.0, hertz_rcap=8.0, rho0=(0.5, 0.5))
    o = make(shape, 2, **params)
    o.init_fields(a, b)
    o.add_colloids([[6.3, 7.7, 5.2], [14.6, 11.1, 10.4]], [3.6, 3.2], [400.0, 300.0],
                   vel=[[0.08, -0.05, 0.03], [-0.06, 0.04, 0.05]],
                   omega=[[0.01, 0.02, -0.015], [-0.02, 0.0, 0.03]])
    c, w, _ = lattice()
    s = np.arange(N)
    X, Y, Z = s % nx, (s // nx) % ny, s // (nx * ny)
    NB = [((X + c[i, 0]) % nx) + nx * (((Y + c[i, 1]) % ny) + ny * ((Z + c[i, 2]) % nz)) for i in range(19)]
    xyz = np.stack([X, Y, Z], 1).astype(float)
    box = np.array(shape, float)
    events = 0
    for _ in range(40):
        ra, rb, _ = o.get_fields()
        own0, col, m0 = o.owner(), o.get_colloids(), o.totals()[:2]
        o.step(1)
        own1, m1 = o.owner(), o.totals()[:2]
        destroyed = (own0 == -1) & (own1 >= 0)
        created = (own0 >= 0) & (own1 == -1)
        events += int(destroyed.sum() + created.sum())
        expect = np.zeros(2)
        rho_b = []
        for k, rho in enumerate((ra, rb)):
            num, den = np.zeros(N), np.zeros(N)
            for i in range(1, 19):
                ok = (own0[NB[i]] == -1) & (own1[NB[i]] == -1)
                num += np.where(ok, w[i] * rho[NB[i]], 0.0)
                den += np.where(ok, w[i], 0.0)
            bar = np.where(den > 0, num / np.where(den > 0, den, 1.0), params["rho0"][k])
            expect[k] = bar[created].sum() - rho[destroyed].sum()
            rho_b.append(np.where(created, bar, rho))
        fluid = own1 == -1
        for i in range(1, 19):
            p = own1[NB[i]]
            m = fluid & (p >= 0)
            if not m.any():
                continue
            rw = xyz[m] + 0.5 * c[i] - col["pos"][p[m]]
            rw -= box * np.round(rw / box)
            cu = (col["vel"][p[m]] + np.cross(col["omega"][p[m]], rw)) @ c[i]
            for k in range(2):
                expect[k] -= (6.0 * w[i] * rho_b[k][m] * cu).sum()
        assert np.all(np.abs((m1 - m0) - expect) < 1e-13 * m0), ((m1 - m0), expect)
    assert events > 10


def test_lubrication_magnitude_leading_order():
    """Eq. 27 (reading c13) against the leading-order lubrication force
    between two spheres approaching along their line of centres (Reynolds
    lubrication of the gap; e.g. Jeffrey and Onishi 1984, Kim and Karrila
    1991): F h -> 6 pi mu (a_i a_j / (a_i + a_j))^2 v as h -> 0, mu = rho nu
    with rho = 1 and the mixture's nu = cs^2 (tau - 1/2) averaged over the two
    components; the prefactor s scales it, the cut-off 1/h_n subtracts a
    constant, the floor h_min clamps it, and a relative velocity
    perpendicular to the line of centres gives no squeeze force."""
    tau = (1.3, 0.9)
    nu = 0.5 * ((tau[0] - 0.5) + (tau[1] - 0.5)) / 3.0
    for Ri, Rj, s in ((5.5, 5.5, 1.0), (4.0, 6.0, 0.3)):
        astar = Ri * Rj / (Ri + Rj)
        pr = dict(lub_on=1, lub_hn=50.0, lub_hmin=1e-6, lub_scale=s, tau=tau)
        d = np.array([0.48, -0.6, 0.64])
        vn = 0.013
        for h in (1e-3, 1e-4):
            F = pair_force((Ri + Rj + h) * d, Ri, Rj, vi=vn * d, vj=(0, 0, 0), **pr)
            leading = 6.0 * math.pi * nu * s * astar ** 2 * vn
            assert abs((-F @ d) * h / leading - 1.0) < 1e-4 + h / 50.0
            assert np.allclose(F, (F @ d) * d, atol=1e-12 * abs(F @ d))
        # below the floor the force stays at its value at h_min
        pr_floor = dict(pr, lub_hmin=0.05)
        F1 = pair_force((Ri + Rj + 0.01) * d, Ri, Rj, vi=vn * d, **pr_floor)
        F2 = pair_force((Ri + Rj + 0.05) * d, Ri, Rj, vi=vn * d, **pr_floor)
        assert np.allclose(F1, F2, rtol=1e-14)
        # sliding past each other: no squeeze force (to the rounding of
        # v . r_hat, relative to the squeeze force at the same gap and speed)
        t = np.cross(d, [0.0, 0.0, 1.0])
        t /= np.linalg.norm(t)
        Ft = pair_force((Ri + Rj + 0.01) * d, Ri, Rj, vi=vn * t, **pr)
        Fn = pair_force((Ri + Rj + 0.01) * d, Ri, Rj, vi=vn * d, **pr)
        assert np.abs(Ft).max() < 1e-12 * np.abs(Fn).max()


def test_lubrication_opposes_approach():
    """Eq. 27: inside h_n the lubrication force on i opposes the relative
    approach velocity along the line of centres and diverges like 1/h."""
    pr = dict(lub_on=1, lub_hn=0.67, lub_hmin=0.1, lub_scale=1.0, tau=(1.0, 1.0))
    d = np.array([1.0, 0, 0])
    F1 = pair_force(11.4 * d, 5.5, 5.5, vi=(0.01, 0, 0), vj=(0, 0, 0), **pr)
    F2 = pair_force(11.2 * d, 5.5, 5.5, vi=(0.01, 0, 0), vj=(0, 0, 0), **pr)
    assert F1[0] < 0 and F2[0] < F1[0]
    # the force reverses with the relative velocity and vanishes without it
    F3 = pair_force(11.4 * d, 5.5, 5.5, vi=(-0.01, 0, 0), vj=(0, 0, 0), **pr)
    assert np.allclose(F3, -F1)
    assert np.all(pair_force(11.4 * d, 5.5, 5.5, vi=(0, 0.01, 0), **pr) == 0)
    assert np.all(pair_force(12.0 * d, 5.5, 5.5, vi=(0.01, 0, 0), **pr) == 0)


def test_thread_count_gives_the_same_bits():
    """The site loops shared out over OpenMP threads: one thread and all
    threads give bit-identical populations and particle states, with moving
    particles, walls, wetting and a body force (each site's arithmetic is
    independent of the others, and the per-particle sums stay in site order)."""
    from oracle import set_threads

    def run(threads):
        set_threads(threads)
        o = Oracle(18, 15, 13, 2)
        o.set_params(G=0.7, tau=(0.8, 1.3), zeta=(0.2, -0.1), bc=(1, 1, 0), wall_u_lo=(0.01, 0, 0),
                     wall_u_hi=(-0.02, 0.01, 0), body_force=(2e-5, 0, 0), hertz_K=10, hertz_sigma=7.0,
                     hertz_rcap=6.0)
        rng = np.random.default_rng(4)
        o.init_fields(0.5 + 0.05 * rng.standard_normal(o.N), 0.5 + 0.05 * rng.standard_normal(o.N))
        o.add_colloids([[5.2, 6.1, 6.3], [12.4, 8.5, 6.6]], [2.7, 3.1], [300.0, 400.0],
                       vel=[[0.03, -0.01, 0.0], [-0.02, 0.02, 0.01]], omega=[[0, 0.02, 0.01], [0.01, 0, 0]])
        o.step(15)
        return o.populations(0), o.populations(1), o.get_colloids()

    try:
        one = run(1)
        many = run(0)
    finally:
        set_threads(0)
    assert np.array_equal(one[0], many[0]) and np.array_equal(one[1], many[1])
    for key in ("pos", "vel", "omega", "quat", "force", "torque"):
        assert np.array_equal(one[2][key], many[2][key]), key
    # and without particles, where the streaming loop is threaded as well
    set_threads(1)
    a = Oracle(20, 9, 11)
    a.set_params(G=0.9, tau=(0.7, 1.1))
    rng = np.random.default_rng(5)
    ra, rb = 0.5 + 0.1 * rng.random(a.N), 0.5 + 0.1 * rng.random(a.N)
    a.init_fields(ra, rb)
    a.step(10)
    set_threads(0)
    b = Oracle(20, 9, 11)
    b.set_params(G=0.9, tau=(0.7, 1.1))
    b.init_fields(ra, rb)
    b.step(10)
    assert np.array_equal(a.populations(0), b.populations(0))
    assert np.array_equal(a.populations(1), b.populations(1))


# ---------------------------------------------------------- one component
def test_one_component_reduction():
    """The single-component fluid of the paper's first benchmark (Sec. 5.1,
    App. D test 1) is the mixture with rho^B = 0: Eq. 14 gives u = j^A/rho^A,
    Eq. 11 gives no force on A (psi^B = 0) and the mixture viscosity is
    component A's.  Pinned here by (a) the exact Poiseuille parabola of the
    halfway bounce-back at tau = 1/2 + sqrt(3/16) with a body force, for
    component A alone; (b) component B's populations staying exactly zero;
    (c) G having no effect on the bits."""
    g, H = 1e-6, 8
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    shape = (4, 4, H)
    N = 16 * H
    z = zcoord(shape)
    runs = []
    for G in (0.0, 0.9):
        o = make(shape, tau=(tau, tau), bc=(1, 1, 0), body_force=(g, 0, 0), G=G)
        o.init_fields(np.full(N, 0.7), np.zeros(N))
        nu = CS2 * (tau - 0.5)
        o.step(int(34 / (nu * (math.pi / H) ** 2)))
        a, b, u = o.get_fields()
        ex = g / (2 * nu) * (z + 0.5) * (H - 0.5 - z)
        assert np.max(np.abs(u[0] - ex)) / ex.max() < 1e-10
        assert np.all(b == 0.0) and np.all(o.populations(1) == 0.0)
        runs.append(o.populations(0))
    assert np.array_equal(runs[0], runs[1])

"""Pins of the oracle's open z faces (Sec. 2.2; App. A, the LB room's open
boundary directives: 1 pressure / Dirichlet by anti-bounce-back, Eq. 10;
2 velocity / Neumann, Eq. 9; 3 equilibrium), against what the lattice
Boltzmann equations fix (CPU only):
  * uniform plug flow f^eq(rho0, u0) between an equilibrium inlet
    (rho0, u0) and a pressure outlet (rho0) is an exact fixed point: it pins
    the signs of Eq. 10 and the reversed link of the equilibrium face;
  * a fluid between two pressure faces of density rho_w relaxes to rho_w
    (the face fixes the density) with a uniform velocity (nothing brakes a
    plug flow between two pressure faces);
  * a density drop between the faces drives fluid out of the dense face and
    into the light one, and leaves the sites beyond the reach of the
    populations exactly at rest;
  * a velocity face is the moving wall of Eq. 9: bit for bit the wall run;
  * the first-order face extrapolation of Sec. 2.2 is exact for a linear
    profile: after one step the populations a velocity face sends in carry
    the density of a linear rho(z) at the face z = -1/2, and those of a
    pressure face the velocity of a linear u(z) there; walls and
    equilibrium faces ignore it (bit for bit).
"""
import numpy as np
import pytest

from oracle import Oracle, feq, lattice


def plug(shape, tau, G, rho0, u0, steps):
    nx, ny, nz = shape
    N = nx * ny * nz
    o = Oracle(*shape)
    o.set_params(tau=tau, G=G, rho0=rho0, bc=(1, 1, 0), open=(3, 1), wall_u_lo=u0,
                 open_rho=(rho0[0], rho0[1], rho0[0], rho0[1]))
    u = np.zeros((3, N))
    u[:] = np.asarray(u0)[:, None]
    o.init_fields(np.full(N, rho0[0]), np.full(N, rho0[1]), u)
    f0 = [o.populations(k) for k in range(2)]
    o.step(steps)
    return o, f0


@pytest.mark.parametrize("tau,G", [((1.0, 1.0), 0.0), ((0.8, 1.3), 0.4)])
def test_plug_flow_is_a_fixed_point(tau, G):
    o, f0 = plug((6, 5, 12), tau, G, (0.7, 0.45), (0.01, -0.02, 0.05), 25)
    for k in range(2):
        assert np.abs(o.populations(k) - f0[k]).max() < 1e-14


def test_pressure_faces_fix_the_density():
    shape = (4, 4, 16)
    N = 4 * 4 * 16
    o = Oracle(*shape)
    o.set_params(tau=(1.0, 1.0), bc=(1, 1, 0), open=(1, 1), open_rho=(0.6, 0.4, 0.6, 0.4))
    rng = np.random.default_rng(2)
    o.init_fields(0.5 + 0.05 * rng.random(N), 0.3 + 0.05 * rng.random(N))
    o.step(5000)
    ra, rb, u = o.get_fields()
    assert np.abs(ra - 0.6).max() < 1e-12 and np.abs(rb - 0.4).max() < 1e-12
    # without walls nothing brakes the flow: the net momentum left by the
    # relaxation stays as a uniform drift (plug flow at rho_w is a fixed point)
    for d in range(3):
        assert np.ptp(u[d]) < 1e-12


def test_density_drop_drives_flow_downhill():
    """Faces at rho 1.04 (z = 0) and 0.96 (z = nz - 1) over a fluid at 1.0 at
    rest: after 10 steps fluid flows out of the dense face and into the light
    one (u_z > 0 next to both), the face planes sit at the face densities,
    and the planes more than 10 links from either face have not been reached
    (a population moves one link per step): they are exactly at rest."""
    shape = (4, 4, 24)
    nx, ny, nz = shape
    N = nx * ny * nz
    o = Oracle(*shape)
    o.set_params(tau=(1.0, 1.0), bc=(1, 1, 0), open=(1, 1), open_rho=(0.52, 0.52, 0.48, 0.48))
    o.init_fields(np.full(N, 0.5), np.full(N, 0.5))
    o.step(10)
    ra, rb, u = o.get_fields()
    rho = (ra + rb).reshape(nz, ny, nx).mean(axis=(1, 2))
    uz = u[2].reshape(nz, ny, nx).mean(axis=(1, 2))
    assert np.all(uz[:3] > 0.01) and np.all(uz[-3:] > 0.01)
    assert np.abs(u.reshape(3, nz, ny, nx)[:, 11:13]).max() == 0.0
    assert abs(rho[0] - 1.04) < 1e-3 and abs(rho[-1] - 0.96) < 1e-3
    assert np.abs(rho[11:13] - 1.0).max() < 1e-14


def test_velocity_face_is_the_moving_wall():
    shape = (5, 4, 9)
    N = 5 * 4 * 9
    rng = np.random.default_rng(3)
    a, b = 0.5 + 0.02 * rng.random(N), 0.5 + 0.02 * rng.random(N)
    runs = []
    for face in (0, 2):
        o = Oracle(*shape)
        o.set_params(tau=(0.9, 1.1), G=0.5, bc=(1, 1, 0), open=(face, face), wall_u_lo=(0.02, 0, 0),
                     wall_u_hi=(-0.01, 0.01, 0))
        o.init_fields(a, b)
        o.step(30)
        runs.append([o.populations(k) for k in range(2)])
    for k in range(2):
        assert np.array_equal(runs[0][k], runs[1][k])


def _lattice():
    """Directions in the oracle's numbering; the weights from |c|^2 (1/3,
    1/18, 1/36 of D3Q19), not from the oracle."""
    c, _w, opp = lattice()
    w = np.array([{0: 1 / 3, 1: 1 / 18, 2: 1 / 36}[int(n)] for n in (c * c).sum(axis=1)])
    return c, w, opp


def _feq(i, c, w, rho, u):
    cu = c[i] @ u
    return w[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (u @ u))


def test_velocity_face_extrapolates_a_linear_density():
    """rho^A(z) = a + b z, rho^B constant, at rest, tau = 1, G = 0: one step
    later the population a velocity face (u_w) sends into a node of z = 0 is
    f*_i - 6 w_i rho_w c_i.u_w with f*_i = w_i rho(0) and rho_w = a - b/2,
    the profile's value at the face; without the extrapolation rho_w = a."""
    shape = nx, ny, nz = (4, 3, 8)
    N = nx * ny * nz
    a_, b_, rb = 0.55, -0.015, 0.45
    z = np.repeat(np.arange(nz), nx * ny)
    uw = np.array([0.03, -0.02, 0.01])
    c, w, opp = _lattice()
    got = {}
    for ex in (0, 1):
        o = Oracle(*shape)
        o.set_params(tau=(1.0, 1.0), bc=(1, 1, 0), open=(2, 0), wall_u_lo=tuple(uw), open_extrap=ex)
        o.init_fields(a_ + b_ * z, np.full(N, rb))
        o.step(1)
        got[ex] = [o.populations(k) for k in range(2)]
    face = z == 0
    for i in np.nonzero(c[:, 2] == -1)[0]:
        for ex, rw in ((1, a_ - b_ / 2), (0, a_)):
            fa = got[ex][0][opp[i], face]
            assert np.abs(fa - (w[i] * a_ - 6 * w[i] * rw * (c[i] @ uw))).max() < 1e-15
            fb = got[ex][1][opp[i], face]
            assert np.abs(fb - (w[i] * rb - 6 * w[i] * rb * (c[i] @ uw))).max() < 1e-15
    # everything away from the face's incoming links is the same
    keep = np.ones((19, N), dtype=bool)
    keep[np.ix_(opp[c[:, 2] == -1], np.nonzero(face)[0])] = False
    assert np.array_equal(got[0][0][keep], got[1][0][keep])


def test_pressure_face_extrapolates_a_linear_velocity():
    """u(z) = u0 + g z (a shear with a linear profile), uniform densities,
    tau = 1, G = 0: one step later a pressure face sends into the nodes of
    z = 0 the anti-bounce-back of Eq. 10, -f^eq_i(rho, u(0)) + 2 w_i rho_w
    (1 + 9/2 (c_i.u_w)^2 - 3/2 u_w^2), with u_w = u0 - g/2 the profile's
    velocity at the face; without the extrapolation u_w = u0."""
    shape = nx, ny, nz = (4, 3, 8)
    N = nx * ny * nz
    z = np.repeat(np.arange(nz), nx * ny)
    u0, g = np.array([0.02, -0.01, 0.015]), np.array([0.004, 0.003, -0.002])
    u = u0[:, None] + g[:, None] * z[None, :]
    rho = (0.5, 0.4)
    rw = (0.6, 0.35)
    c, w, opp = _lattice()
    for ex, uw in ((1, u0 - g / 2), (0, u0)):
        o = Oracle(*shape)
        o.set_params(tau=(1.0, 1.0), bc=(1, 1, 0), open=(1, 0), open_rho=(rw[0], rw[1], 1.0, 1.0),
                     open_extrap=ex)
        o.init_fields(np.full(N, rho[0]), np.full(N, rho[1]), u)
        o.step(1)
        for k in range(2):
            f = o.populations(k)
            for i in np.nonzero(c[:, 2] == -1)[0]:
                cu = c[i] @ uw
                want = -_feq(i, c, w, rho[k], u0) + 2 * w[i] * rw[k] * (1 + 4.5 * cu * cu - 1.5 * (uw @ uw))
                assert np.abs(f[opp[i], z == 0] - want).max() < 1e-15


def test_extrapolation_leaves_walls_and_equilibrium_faces():
    shape = (5, 4, 9)
    N = 5 * 4 * 9
    rng = np.random.default_rng(4)
    a, b = 0.5 + 0.02 * rng.random(N), 0.5 + 0.02 * rng.random(N)
    runs = []
    for ex in (0, 1):
        o = Oracle(*shape)
        o.set_params(tau=(0.9, 1.1), G=0.5, bc=(1, 1, 0), open=(0, 3), wall_u_lo=(0.02, 0, 0),
                     wall_u_hi=(-0.01, 0.01, 0.02), open_rho=(1.0, 1.0, 0.52, 0.49), open_extrap=ex)
        o.init_fields(a, b)
        o.step(20)
        runs.append([o.populations(k) for k in range(2)])
    for k in range(2):
        assert np.array_equal(runs[0][k], runs[1][k])


def test_extrapolation_flag_is_checked():
    o = Oracle(4, 4, 6)
    with pytest.raises(RuntimeError):
        o.set_params(bc=(1, 1, 0), open=(2, 0), open_extrap=2)
    o.set_params(bc=(1, 1, 0), open=(2, 0), open_extrap=1)


def test_extrapolation_falls_back_under_a_particle():
    """Where the next interior node b + 1 is a particle node the velocity
    face takes the density of the boundary node itself: the populations the
    face sends into that column are those of the run without extrapolation,
    while a column with fluid at b + 1 differs by -3 w_i (rho_b - rho_{b+1})
    c_i.u_w, half the density step in the wall term of Eq. 9."""
    shape = nx, ny, nz = (8, 8, 8)
    N = nx * ny * nz
    a_, b_ = 0.55, -0.02
    z = np.repeat(np.arange(nz), nx * ny)
    uw = np.array([0.03, -0.02, 0.01])
    c, w, opp = _lattice()
    got = {}
    for ex in (0, 1):
        o = Oracle(*shape, 1)
        o.set_params(tau=(1.0, 1.0), bc=(1, 1, 0), open=(2, 0), wall_u_lo=tuple(uw), open_extrap=ex)
        o.init_fields(a_ + b_ * z, np.full(N, 0.45))
        o.add_colloids([[2.0, 2.0, 2.2]], [1.5], [1e30])
        own = o.owner()
        o.step(1)
        got[ex] = o.populations(0)
    site = lambda x, y, zz: x + nx * (y + ny * zz)
    assert own[site(2, 2, 1)] == 0 and own[site(2, 2, 0)] < 0 and own[site(0, 0, 1)] < 0
    for i in np.nonzero(c[:, 2] == -1)[0]:
        under, free = site(2, 2, 0), site(0, 0, 0)
        assert got[1][opp[i], under] == got[0][opp[i], under]
        d = got[1][opp[i], free] - got[0][opp[i], free]
        assert abs(d - 3 * w[i] * b_ * (c[i] @ uw)) < 1e-15


def test_pressure_face_extrapolates_the_weighted_mixture_velocity():
    """Unequal tau, G = 0: component k starts at f^eq(rho^k, u^k(z)) with
    linear u^k(z).  The boundary velocity of Eq. 10 is the mixture velocity
    of Eq. 14, u = sum_k omega_k rho^k u^k / sum_k omega_k rho^k, so the
    face sends in -f*_i + 2 w_i rho_w (1 + 9/2 (c_i.u_w)^2 - 3/2 u_w^2)
    with f*_i = (1 - omega) f^eq(rho^k, u^k(0)) + omega f^eq(rho^k, u(0)),
    omega the mixture frequency of Eq. 13 (1/omega = 3 nubar + 1/2,
    1/nubar = sum_k (rho^k / rho) / nu_k), and u_w = u(0) + (u(0) - u(1))/2;
    an unweighted mixture velocity fails this."""
    shape = nx, ny, nz = (4, 3, 8)
    N = nx * ny * nz
    z = np.repeat(np.arange(nz), nx * ny)
    tau = (0.7, 1.4)
    om = [1 / t for t in tau]
    rho = (0.6, 0.3)
    ua0, ga = np.array([0.02, 0.0, 0.01]), np.array([0.003, 0.001, -0.002])
    ub0, gb = np.array([-0.01, 0.015, 0.0]), np.array([-0.002, 0.002, 0.001])
    c, w, opp = _lattice()
    mix = lambda ua, ub: (om[0] * rho[0] * ua + om[1] * rho[1] * ub) / (om[0] * rho[0] + om[1] * rho[1])
    u0, u1 = mix(ua0, ub0), mix(ua0 + ga, ub0 + gb)
    nu = [(t - 0.5) / 3 for t in tau]
    nubar = 1 / sum(r / sum(rho) / n for r, n in zip(rho, nu))
    omega = 1 / (3 * nubar + 0.5)
    uw = u0 + 0.5 * (u0 - u1)
    rw = (0.62, 0.28)
    o = Oracle(*shape)
    o.set_params(tau=tau, bc=(1, 1, 0), open=(1, 0), open_rho=(rw[0], rw[1], 1.0, 1.0), open_extrap=1)
    o.init_fields(np.full(N, rho[0]), np.full(N, rho[1]))
    for k, (u_0, g_) in enumerate(((ua0, ga), (ub0, gb))):
        f = np.empty((19, N))
        for s in range(N):
            u = u_0 + g_ * z[s]
            f[:, s] = [_feq(i, c, w, rho[k], u) for i in range(19)]
        o.set_populations(k, f)
    o.step(1)
    for k, u_k in enumerate((ua0, ub0)):
        f = o.populations(k)
        for i in np.nonzero(c[:, 2] == -1)[0]:
            fs = (1 - omega) * _feq(i, c, w, rho[k], u_k) + omega * _feq(i, c, w, rho[k], u0)
            cu = c[i] @ uw
            want = -fs + 2 * w[i] * rw[k] * (1 + 4.5 * cu * cu - 1.5 * (uw @ uw))
            assert np.abs(f[opp[i], z == 0] - want).max() < 1e-15

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every quantity is compared on its natural lattice scale, at the bound that
the storage form states: 1e-12 for FP64, 1e-5 for FP32, 1e-3 for FP16
deviation storage.
  * densities: relative to max |rho| (rho is O(1));
  * fluid velocity: relative to max(|u|_max, c = 1 lattice speed); in the
    bijel workloads the mixture relaxes to |u| ~ 1e-8, where a comparison
    relative to |u| itself only measures rounding of j = sum_i f_i c_i
    (sum_i |f_i| / |j| ~ 1e7), so the lattice speed is the scale there; the
    sheared-wall cases (|u| ~ 0.05) test the velocity relative to itself;
  * particle position (lattice spacing), velocity and angular velocity
    (lattice speed), orientation (unit quaternion) and force / torque terms
    (lattice momentum per step): absolute in those units.
Boxes span several thread blocks with ragged tails (nx a multiple of 4, odd
ny and nz).
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2004_04080_gb300.workloads import mixture_densities, workload

pytestmark = pytest.mark.gpu


def _lattice(shape, prec, maxc):
    from paper_2004_04080_gb300.lbgb import LBLattice

    return LBLattice(shape, prec, max_colloids=maxc)


def run_both(shape, params, steps, prec="fp64", colloids=None, dens=None, u=None):
    a, b = dens if dens is not None else mixture_densities(shape, seed=7)
    maxc = 0 if colloids is None else len(colloids["pos"])
    g = _lattice(shape, prec, maxc)
    g.set_params(**params)
    g.init_fields(a, b, u)
    o = Oracle(*shape, maxc)
    o.set_params(**params)
    o.init_fields(a, b, u)
    if colloids is not None:
        g.add_colloids(**colloids)
        o.add_colloids(**colloids)
        o.radius = np.asarray(colloids["radius"], dtype=np.float64)
    g.step(steps)
    o.step(steps)
    return g, o


def rel(x, y, floor=0.0):
    den = max(np.abs(y).max(), floor, 1e-300)
    return np.abs(x - y).max() / den


def compare_fields(g, o, tol, u_scale=1.0):
    ga, gb, gu = g.get_fields()
    ra, rb, ru = o.get_fields()
    assert np.array_equal(g.owner(), o.owner())
    ea, eb, eu = rel(ga, ra), rel(gb, rb), rel(gu, ru, floor=u_scale)
    assert ea < tol and eb < tol, (ea, eb)
    assert eu < tol, eu
    return ea, eb, eu


def compare_colloids(g, o, tol, term_tol=None, event_mom=0.0):
    """Particle state absolute; the force and torque terms absolute, or with
    ``term_tol`` relative to each term's largest value, floored at one
    lattice momentum unit for a force and at R_max such units for a torque
    (the lever arm of the link forces).  ``event_mom`` is the momentum of one
    node refill (Eq. 25) that the terms holding the refills (F_c and the
    totals) may differ by in addition: a refill is a discrete event, and a
    state that carries the error of a reduced-precision form can create a node
    one step earlier or later than the oracle, which moves that node's whole
    momentum from one step's F_c to the next one's."""
    gc, rc = g.get_colloids(), o.get_colloids()
    for key in ("pos", "vel", "omega", "quat"):
        err = np.abs(gc[key] - rc[key]).max()
        assert err < tol, (key, err)
    rmax = float(np.max(o.radius)) if getattr(o, "radius", None) is not None else 1.0
    for term in ("F_liq", "T_liq", "F_s", "T_s", "F_d", "F_c", "F_pair", "F_total", "T_total"):
        ref = o.term(term)
        err = np.abs(g.term(term) - ref).max()
        if term_tol is None:
            assert err < tol, (term, err)
        else:
            floor = rmax if term.startswith("T") else 1.0
            event = 0.0
            if term in ("F_c", "F_total"):
                event = event_mom
            elif term == "T_total":
                event = rmax * event_mom
            assert (err - event) / max(np.abs(ref).max(), floor) < term_tol, (term, err, event)


def refill_momentum(o):
    """Momentum of one created node (Eq. 25), bounded from the oracle's state:
    the largest total density of the lattice times the fastest surface speed
    |v_p| + |omega_p| R_p of a particle."""
    ra, rb, _ = o.get_fields()
    c = o.get_colloids()
    speed = np.linalg.norm(c["vel"], axis=1) + np.linalg.norm(c["omega"], axis=1) * np.asarray(o.radius)
    return float((ra + rb).max() * speed.max())


def test_fp64_small_workload_100_steps():
    """Two-component SC, tau=1, G=0.65, 50/50 +-1 %, four R=4.5 neutral
    spheres, 32^3 periodic, 100 steps: fields and particle state to 1e-12."""
    w = workload("small_fp64")
    g, o = run_both(w.shape, w.params, w.steps, "fp64", w.colloids(), w.densities())
    compare_fields(g, o, 1e-12)
    compare_colloids(g, o, 1e-12)


def test_fp64_ragged_walls_moving_particle():
    """Odd-sized box, sheared walls, body force, unequal tau, wetting and two
    fast particles that collide and cross many nodes (destroy/create events in
    most steps), 40 steps compared step by step."""
    shape = (20, 13, 11)
    params = dict(G=0.6, tau=(0.8, 1.2), zeta=(0.15, -0.15), bc=(1, 1, 0), wall_u_lo=(-0.02, 0.01, 0),
                  wall_u_hi=(0.03, 0, 0), body_force=(1e-5, 0, -2e-6), hertz_K=20, hertz_sigma=8.0,
                  hertz_rcap=7.0, side_wall_k=0.5, side_wall_d=4.0)
    col = dict(pos=[[7.2, 6.1, 5.3], [15.5, 6.5, 5.0]], radius=[3.2, 3.0], mass=[1500.0, 1200.0],
               vel=[[0.05, 0.03, -0.01], [-0.04, 0.0, 0.02]], omega=[[0.01, 0.0, 0.02], [0, -0.02, 0]])
    g, o = run_both(shape, params, 0, "fp64", col)
    events = 0
    for t in range(40):
        g.step(1)
        o.step(1)
        events += np.any(o.term("F_c") != 0) + np.any(o.term("F_d") != 0)
        if t % 10 == 9:
            compare_colloids(g, o, 1e-11)
    assert events > 20
    compare_fields(g, o, 1e-12)
    compare_colloids(g, o, 1e-11)


def pickering_like(shape):
    """Two B-rich droplets in the A-rich matrix of the demixing mixture (the
    calibrated coexistence densities and Delta(77 deg) of the Pickering
    workload), six mobile R = 4 particles, some across the interfaces."""
    import json
    import os

    from paper_2004_04080_gb300.workloads import droplet_densities

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "pickering_calibration.json")) as f:
        cal = json.load(f)
    dl = cal["delta_77"]
    params = dict(G=0.65, tau=(1.0, 1.0), rho0=(1.0, 1.0), zeta=(dl, -dl), hertz_K=20.0, hertz_sigma=9.0,
                  hertz_rcap=8.0)
    dens = droplet_densities(shape, [[12.3, 11.6, 10.2], [31.7, 25.4, 22.8]], 8.0, cal["rho_rich"],
                             cal["rho_poor"])
    col = dict(pos=[[12.1, 11.8, 19.6], [21.4, 11.2, 10.7], [31.2, 25.9, 13.3], [5.5, 30.2, 24.9],
                    [38.6, 6.4, 5.1], [24.0, 20.0, 29.5]],
               radius=[4.0] * 6, mass=[4.0 / 3.0 * math.pi * 64.0] * 6,
               vel=[[0.01, -0.005, 0.02], [0, 0, 0], [-0.01, 0.01, 0], [0, 0.02, 0], [0, 0, 0], [0.005, 0, 0]])
    return params, dens, col


def test_fp64_cell_list_with_lubrication():
    """80 mobile R = 3 particles in a 48^3 box (more than 64: the pair forces
    search a cell grid of 6^3 cells instead of all pairs), soft Hertz contact
    (Eq. 26, K = 2) and lubrication (Eq. 27) on, centres placed at least 6.3
    apart (9 pairs start inside the lubrication range h < 0.67, 18 inside the
    contact range) with random velocities; compared while the pair forces act
    (step 4) and after 20 steps."""
    from paper_2004_04080_gb300.workloads import place_colloids

    shape = (48, 48, 48)
    n, R = 80, 3.0
    params = dict(G=0.5, tau=(1.0, 1.0), zeta=(0.05, -0.05), hertz_K=2.0, hertz_sigma=2 * R + 1, hertz_rcap=2 * R,
                  lub_on=1, lub_hn=0.67, lub_hmin=0.1, lub_scale=1.0)
    pos = place_colloids(shape, n, R, seed=11, min_dist=2 * R + 0.3)
    rng = np.random.default_rng(12)
    col = dict(pos=pos, radius=[R] * n, mass=[4.0 / 3.0 * math.pi * R ** 3] * n,
               vel=0.01 * rng.standard_normal((n, 3)))
    g, o = run_both(shape, params, 4, "fp64", col)
    assert np.count_nonzero(np.abs(o.term("F_pair")).sum(axis=1)) >= 10
    compare_colloids(g, o, 1e-11)
    g.step(16)
    o.step(16)
    compare_fields(g, o, 1e-12)
    compare_colloids(g, o, 1e-11)


def test_fp64_demixing_droplets_wetting_particles():
    """The Pickering physics at a size the oracle runs in seconds: the
    demixing mixture (G rho_tot = 1.3), sharp droplet interfaces, wetting
    particles (Eq. 20, 21) crossing them; ragged 44 x 38 x 34 box, 60 steps."""
    shape = (44, 38, 34)
    params, dens, col = pickering_like(shape)
    g, o = run_both(shape, params, 60, "fp64", col, dens=dens)
    compare_fields(g, o, 1e-12)
    compare_colloids(g, o, 1e-11)


@pytest.mark.parametrize("prec,tol,term_tol", [("fp32", 1e-5, None), ("fp16", 1e-3, 1e-2)])
def test_reduced_precision_demixing_droplets(prec, tol, term_tol):
    """The same case in the reduced-precision forms against the oracle.  The
    link-force sums reach |F_liq| ~ 3 here (capillary and wetting forces,
    nearly balanced by F_s); in FP16 storage they are sums over the ~300
    links of a particle of terms of the fields, which carry the 1e-3 error of
    the form, and are compared relative to their scale at 1e-2 (measured: 1e-3
    for F_liq, 4e-3 for T_liq with the lever-arm floor).  In FP16 the refill
    term F_c at the compared step differs from the oracle's by one node's
    momentum in about half of the rounding seeds (measured 8.9e-3 against
    3e-5 otherwise): a node created one step apart; that event is allowed
    on F_c and the totals (refill_momentum)."""
    shape = (44, 38, 34)
    params, dens, col = pickering_like(shape)
    g, o = run_both(shape, params, 60, prec, col, dens=dens)
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol, term_tol, event_mom=refill_momentum(o) if prec == "fp16" else 0.0)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 1e-3)])
@pytest.mark.parametrize("nx", [20, 24])
def test_reduced_precision_ragged_walls_moving_particles(prec, tol, nx):
    """The ragged-tile case in the reduced-precision forms: tiles 20 or 24
    sites wide and 5 rows high at the lattice edges (FP16 with nx = 20 takes
    the plain-load fused kernel, every other case the copy-pipelined one),
    sheared walls, unequal tau, moving particles, 40 steps."""
    shape = (nx, 13, 11)
    params = dict(G=0.6, tau=(0.8, 1.2), zeta=(0.15, -0.15), bc=(1, 1, 0), wall_u_lo=(-0.02, 0.01, 0),
                  wall_u_hi=(0.03, 0, 0), body_force=(1e-5, 0, -2e-6), hertz_K=20, hertz_sigma=8.0,
                  hertz_rcap=7.0, side_wall_k=0.5, side_wall_d=4.0)
    col = dict(pos=[[7.2, 6.1, 5.3], [15.5, 6.5, 5.0]], radius=[3.2, 3.0], mass=[1500.0, 1200.0],
               vel=[[0.05, 0.03, -0.01], [-0.04, 0.0, 0.02]], omega=[[0.01, 0.0, 0.02], [0, -0.02, 0]])
    g, o = run_both(shape, params, 40, prec, col)
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol)


@pytest.mark.parametrize("tau", [(0.7, 0.9), (1.0, 1.0)])
def test_fp64_fluid_only_populations_exact(tau):
    """No particles (the plain fused kernel, and the lean kernel at tau = 1):
    every population matches the oracle to 1e-13."""
    shape = (16, 9, 7)
    g, o = run_both(shape, dict(G=0.9, tau=tau), 25, "fp64")
    assert g.fused_kernel() == ("k_lean" if tau == (1.0, 1.0) else "k_fused")
    for k in (0, 1):
        assert rel(g.populations(k), o.populations(k)) < 1e-13


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_reduced_precision_small_workload(prec, tol):
    """FP32 storage, and FP16 deviation storage with FP32 arithmetic, vs the
    FP64 oracle on the 32^3 bijel workload after 100 steps."""
    w = workload("small_fp64")
    g, o = run_both(w.shape, w.params, w.steps, prec, w.colloids(), w.densities())
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol)


@pytest.mark.parametrize("prec,tol,tol_u", [("fp64", 1e-12, 1e-12), ("fp32", 1e-5, 1e-5), ("fp16", 1e-3, 2e-3)])
@pytest.mark.parametrize("nx", [32, 36])
def test_sheared_walls_with_particles(prec, tol, tol_u, nx):
    """Walls at z = -1/2, nz - 1/2 moving at -/+0.05 (the confined shear
    workload's boundary), four particles, 100 steps: velocities are O(0.05)
    here and are compared relative to themselves.  At tau = 1 the momentum
    kernel runs; nx = 36 leaves a ragged last tile of 4 columns.  FP16
    deviation storage rounds each population to 11 significant bits of
    f_i - w_i rho0; next to the sheared walls (|u| = 0.05) this leaves a
    velocity error of about 1.1e-3 of max |u| after 100 steps (5e-5 of the
    lattice speed), so the FP16 velocity bound here is 2e-3 relative to max |u|."""
    shape = (nx, 21, 23)
    w = workload("shear512")
    params = dict(w.params, side_wall_d=6.5)
    col = dict(pos=[[8.2, 5.3, 7.7], [22.6, 14.1, 11.4], [9.9, 16.2, 15.8], [25.1, 4.4, 16.0]],
               radius=5.5, mass=700.0)
    g, o = run_both(shape, params, 100, prec, col)
    assert g.fused_kernel() == "k_lean"
    ga, gb, gu = g.get_fields()
    ra, rb, ru = o.get_fields()
    assert np.abs(ru).max() > 0.02
    keep = np.ones(ga.shape, dtype=bool)
    if prec == "fp16":
        keep = event_mask(g, o, shape, [5.5] * 4)
    else:
        assert np.array_equal(g.owner(), o.owner())
    assert rel(ga[keep], ra[keep]) < tol and rel(gb[keep], rb[keep]) < tol
    assert rel(gu[:, keep], ru[:, keep]) < tol_u, rel(gu[:, keep], ru[:, keep])
    # FP16: the force and torque terms at 1e-2 of their scale, as in the
    # droplet case (a node created a step apart changes the links of its
    # particle: 3e-3 of F_liq measured in such a run)
    compare_colloids(g, o, tol, 1e-2 if prec == "fp16" else None)


def event_mask(g, o, shape, radius):
    """Sites to compare the fields on, for a reduced-precision run against
    the oracle.  The particle positions carry the error of the form (about
    2e-5 here in FP16), so a node whose distance to a centre lies that close
    to R can be created or destroyed (Eqs. 24-25) a step apart from the
    oracle, and then holds a density of order one in one run and none in the
    other.  At most two such nodes are allowed, each within 0.1 of a
    particle's surface; the sites within two links of them (where the
    different bounce-back surface has reached by the compared step) are left
    out, and the owner map must agree everywhere else."""
    go, oo = g.owner(), o.owner()
    diff = np.flatnonzero(go != oo)
    assert len(diff) <= 2, len(diff)
    nx, ny, nz = shape
    pos = o.get_colloids()["pos"]
    keep = np.ones(go.shape, dtype=bool)
    for s in diff:
        x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
        d = np.array([x, y, z], dtype=float) - pos
        for a, n in enumerate(shape):
            d[:, a] -= n * np.round(d[:, a] / n)
        gap = np.abs(np.linalg.norm(d, axis=1) - np.asarray(radius)).min()
        assert gap < 0.1, (s, gap)
        for dz in range(-2, 3):
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    keep[(x + dx) % nx + nx * ((y + dy) % ny + ny * ((z + dz) % nz))] = False
    return keep


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_momentum_kernel_runs_the_particle_workloads(prec):
    """Every tau = 1 lattice (the particle workloads: bijel, Pickering,
    confined shear; and the fluid alone) takes the lean kernel after the full
    density pass; other tau the two-pass kernel with particles, the plain
    fused kernel without."""
    w = workload("small_fp64")
    g = _lattice(w.shape, prec, w.n_colloids)
    g.set_params(**w.params)
    a, b = w.densities()
    g.init_fields(a, b)
    assert g.fused_kernel() == "k_lean"
    g.set_params(**dict(w.params, tau=(0.8, 1.2)))
    assert g.fused_kernel() == "k_fused"
    g.set_params(**w.params)
    c = w.colloids()
    g.add_colloids(c["pos"], c["radius"], c["mass"])
    assert g.fused_kernel() == "k_lean"
    g.set_params(**dict(w.params, tau=(0.8, 1.2)))
    assert g.fused_kernel() == "k_fused_async"


def test_mass_conservation_gpu_fp64():
    shape = (12, 11, 9)
    a, b = mixture_densities(shape, seed=9, amp=0.05)
    g = _lattice(shape, "fp64", 0)
    g.set_params(G=0.8, tau=(1.0, 1.0), bc=(1, 1, 0), wall_u_lo=(0.01, 0, 0), wall_u_hi=(-0.01, 0, 0))
    g.init_fields(a, b)
    m0 = g.totals()[:2]
    g.step(50)
    m1 = g.totals()[:2]
    assert np.all(np.abs(m1 - m0) / m0 < 1e-13)


def test_error_paths_are_reported():
    """Out-of-order calls, overlapping particles and non-finite densities are
    reported as status codes (host-side injections only)."""
    from paper_2004_04080_gb300 import lbgb

    shape = (12, 12, 12)
    g = _lattice(shape, "fp32", 2)
    with pytest.raises(lbgb.LBError) as e:
        g.step(1)
    assert e.value.code == lbgb.LB_ERR_STATE
    g.set_params(G=0.5)
    a = np.full(12 ** 3, 0.5)
    g.init_fields(a, a)
    with pytest.raises(lbgb.LBError) as e:
        g.add_colloids([[2.0, 2.0, 2.0], [2.5, 2.0, 2.0]], 1.5, 10.0)
    assert e.value.code == lbgb.LB_ERR_OVERLAP
    bad = a.copy()
    bad[17] = math.nan
    g.init_fields(bad, a)
    with pytest.raises(lbgb.LBError) as e:
        g.step(2)
    assert e.value.code == lbgb.LB_ERR_NONFINITE
    with pytest.raises(lbgb.LBError) as e:
        g.set_params(tau=(0.4, 1.0))
    assert e.value.code == lbgb.LB_ERR_ARG


def test_create_rejects_lattices_beyond_32bit_site_indices():
    """Sites are indexed in 32 bits inside the kernels: a lattice of 2^31 or
    more sites is refused before any allocation is used."""
    import torch

    from paper_2004_04080_gb300 import lbgb

    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbgb.LBError) as e:
        lbgb.lb_create(2048, 1024, 1024, lbgb.LB_FP32, 0, ws.data_ptr(), ws.numel(), 0)
    assert e.value.code == lbgb.LB_ERR_ARG


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("fp16", 1e-3)])
def test_janus_particles_rotating(prec, tol):
    """Janus wettability: the wetting of a particle node switches with its
    angle to the particle's body axis (smoothed over 20 degrees around 100),
    on two mobile particles that spin and drift across a demixing mixture,
    so that the switch moves over the surface as the orientation changes
    (Eqs. 20, 21, 31-34); 40 steps, ragged 36 x 27 x 23 box."""
    shape = (36, 27, 23)
    params = dict(G=0.9, tau=(1.0, 1.0), zeta=(0.2, 0.15), rho0=(0.5, 0.5), janus=1, janus_theta0=100.0,
                  janus_width=20.0, hertz_K=20.0, hertz_sigma=8.0, hertz_rcap=7.0)
    rs = math.sqrt(0.5)
    col = dict(pos=[[9.3, 12.2, 10.6], [25.7, 14.1, 12.3]], radius=[4.2, 3.8], mass=[300.0, 250.0],
               vel=[[0.03, -0.01, 0.02], [-0.02, 0.02, -0.01]],
               omega=[[0.0, 0.03, 0.02], [0.04, -0.01, 0.0]],
               quat=[[rs, 0.0, rs, 0.0], [0.5, 0.5, -0.5, 0.5]])
    dens = mixture_densities(shape, seed=19, amp=0.05)
    g, o = run_both(shape, params, 40, prec, col, dens=dens)
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol, 1e-2 if prec == "fp16" else None)
    # the wetting of the two caps differs: the particle force from Eq. 21
    # is not that of a uniformly wetting particle
    p = dict(params, janus=0)
    _, o2 = run_both(shape, p, 40, "fp64", col, dens=dens)
    assert np.abs(o.term("T_s") - o2.term("T_s")).max() > 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_particle_sums_repeat_bit_for_bit(prec):
    """The per-particle sums that many threads add to (link forces and
    torques of Eqs. 19, 22-23, the wetting force of Eq. 21, the remap momenta
    of Eqs. 24-25) are fixed-point sums, so two runs of the same input give
    the same bits in every term and in the particle trajectories, whatever
    the order in which the threads added (60 steps, 8 moving particles
    crossing nodes, sheared walls, momentum kernel)."""
    from paper_2004_04080_gb300.lbgb import LBLattice

    shape = (48, 37, 29)
    w = workload("shear512")
    params = dict(w.params, side_wall_d=6.5)
    rng = np.random.default_rng(3)
    pos = [[6.0 + 12.0 * (i % 4) + rng.uniform(0, 2), 8.0 + 18.0 * (i // 4) + rng.uniform(0, 2),
            14.0 + rng.uniform(-2, 2)] for i in range(8)]
    col = dict(pos=pos, radius=4.5, mass=350.0, vel=rng.uniform(-0.03, 0.03, (8, 3)),
               omega=rng.uniform(-0.02, 0.02, (8, 3)))
    a, b = mixture_densities(shape, seed=29, amp=0.05)

    def run():
        g = LBLattice(shape, prec, max_colloids=8)
        g.set_params(**params)
        g.init_fields(a, b)
        g.add_colloids(**col)
        g.step(60)
        return g

    g1, g2 = run(), run()
    for term in ("F_liq", "T_liq", "F_s", "T_s", "F_d", "T_d", "F_c", "T_c", "F_total", "T_total"):
        assert np.array_equal(g1.term(term), g2.term(term)), term
    c1, c2 = g1.get_colloids(), g2.get_colloids()
    for key in ("pos", "vel", "omega", "quat"):
        assert np.array_equal(c1[key], c2[key]), key
    assert np.array_equal(g1.populations(0), g2.populations(0))
    assert np.abs(g1.term("F_liq")).max() > 1e-4 and np.abs(g1.term("F_d")).max() > 0.0


def test_pair_list_skin_keeps_the_forces_and_rebuilds_rarely():
    """The particle pair list with a skin (App. A rcut, delr): lubrication
    (Eq. 27) and Hertz contacts (Eq. 26) between 10 particles driven into
    each other, 120 steps.  With delr = 1 the list is rebuilt only after a
    particle has moved 1/2, yet the run is bit for bit the run that rebuilds
    every step (delr = 0), and it matches the FP64 oracle, which evaluates
    every pair."""
    from paper_2004_04080_gb300.lbgb import LBLattice

    shape = (56, 45, 39)
    params = dict(G=0.3, tau=(0.9, 1.1), hertz_K=20.0, hertz_sigma=10.0, hertz_rcap=9.0, lub_on=1,
                  lub_scale=0.1, lub_hn=0.67, lub_hmin=0.5, rcut=10.5)
    rng = np.random.default_rng(8)
    pos = [[8.0 + 11.5 * (i % 4) + rng.uniform(-1, 1), 10.0 + 24.0 * (i // 4 % 2) + rng.uniform(-1, 1),
            10.0 + 18.0 * (i // 8) + rng.uniform(-1, 1)] for i in range(10)]
    # pairs of neighbours along x driven towards each other
    vel = [[0.03 if i % 2 == 0 else -0.03, rng.uniform(-0.01, 0.01), rng.uniform(-0.01, 0.01)] for i in range(10)]
    # heavy enough that the fluid's drag leaves them moving for the whole run
    col = dict(pos=pos, radius=4.5, mass=3000.0, vel=vel)
    a, b = mixture_densities(shape, seed=31, amp=0.05)
    steps = 120

    def run(delr):
        g = LBLattice(shape, "fp64", max_colloids=10)
        g.set_params(**dict(params, delr=delr))
        g.init_fields(a, b)
        g.add_colloids(**col)
        fmax = 0.0
        for _ in range(steps // 10):
            g.step(10)
            fmax = max(fmax, np.abs(g.term("F_pair")).max())
        return g, fmax

    (g1, fmax), (g0, _) = run(1.0), run(0.0)
    assert g0.pair_list_builds() == steps
    assert 2 <= g1.pair_list_builds() <= steps // 6, g1.pair_list_builds()
    for term in ("F_pair", "F_total", "T_total"):
        assert np.array_equal(g1.term(term), g0.term(term)), term
    c1, c0 = g1.get_colloids(), g0.get_colloids()
    for key in ("pos", "vel", "omega", "quat"):
        assert np.array_equal(c1[key], c0[key]), key
    assert fmax > 1e-2  # contacts acted during the run
    o = Oracle(*shape, 10)
    o.set_params(**dict(params, delr=1.0))
    o.init_fields(a, b)
    o.add_colloids(**col)
    o.radius = np.full(10, 4.5)
    o.step(steps)
    compare_fields(g1, o, 1e-12)
    compare_colloids(g1, o, 1e-11)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_janus_lubrication_benchmark_physics(prec, tol):
    """The colloid benchmark's physics (Sec. 5.1 with the App. D input):
    demixing mixture, R = 5.5 Janus particles (108 +- 5 degrees, wetting
    0.1 / 0.1) of mass 472 at random orientations, lubrication, Hertz
    (20, 12, 11) and the pair list with rcut 12, delr 1, at phi = 0.10 in a
    48 x 44 x 40 box (12 particles), 60 steps against the oracle."""
    w = workload("janus_lub256", scale=(48, 44, 40))
    c = w.colloids()
    assert w.n_colloids == 12 and "quat" in c
    g, o = run_both(w.shape, w.params, 60, prec, c, w.densities())
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("fp16", 1e-3)])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.2)])
def test_open_faces(prec, tol, tau):
    """Open z faces (Sec. 2.2): an equilibrium inlet (rho_w, u_w) at z = -1/2
    and a pressure outlet (Eq. 10) at z = nz - 1/2 on the demixing-capable
    mixture, without particles (the lean kernel at tau = 1, the plain fused
    kernel otherwise), 40 steps."""
    shape = (24, 13, 17)
    params = dict(G=0.6, tau=tau, bc=(1, 1, 0), open=(3, 1), wall_u_lo=(0.01, 0.0, 0.03),
                  open_rho=(0.56, 0.46, 0.5, 0.5))
    g, o = run_both(shape, params, 40, prec, dens=mixture_densities(shape, seed=41, amp=0.05))
    compare_fields(g, o, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.2)])
def test_open_faces_with_particles(prec, tol, tau):
    """Open z faces with moving particles (the momentum kernel at tau = 1, the
    copy-pipelined one otherwise): a pressure face below, a velocity face
    (Eq. 9) above, 40 steps."""
    shape = (32, 21, 23)
    params = dict(G=0.5, tau=tau, bc=(1, 1, 0), open=(1, 2), wall_u_hi=(0.02, 0.0, 0.0),
                  open_rho=(0.52, 0.5, 0.5, 0.5), hertz_K=20, hertz_sigma=8.0, hertz_rcap=7.0,
                  side_wall_k=0.5, side_wall_d=4.0)
    col = dict(pos=[[8.2, 5.3, 7.7], [22.6, 14.1, 12.4]], radius=[3.5, 3.2], mass=[400.0, 350.0],
               vel=[[0.02, 0.01, -0.01], [-0.01, 0.0, 0.02]], omega=[[0.0, 0.01, 0.0], [0.01, 0.0, 0.0]])
    g, o = run_both(shape, params, 40, prec, col, mixture_densities(shape, seed=43, amp=0.05))
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol)


def _away_from(g, o_plain, tol):
    """The run differs from the oracle's run without extrapolation by more
    than the tolerance: the extrapolated face values reached the result."""
    ga, _, gu = g.get_fields()
    ra, _, ru = o_plain.get_fields()
    assert max(rel(ga, ra), rel(gu, ru, floor=1.0)) > 10 * tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("fp16", 1e-3)])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.2)])
def test_open_faces_extrapolated(prec, tol, tau):
    """Open z faces with the first-order extrapolation of Sec. 2.2: a
    velocity face (Eq. 9 with rho_w extrapolated) below, a pressure face
    (Eq. 10 with u_w extrapolated) above, without particles (the lean kernel
    at tau = 1, the plain fused kernel otherwise), 40 steps."""
    shape = (24, 13, 17)
    params = dict(G=0.6, tau=tau, bc=(1, 1, 0), open=(2, 1), wall_u_lo=(0.01, -0.02, 0.03),
                  open_rho=(0.5, 0.5, 0.47, 0.5), open_extrap=1)
    dens = mixture_densities(shape, seed=45, amp=0.05)
    g, o = run_both(shape, params, 40, prec, dens=dens)
    assert g.fused_kernel() == ("k_lean" if tau == (1.0, 1.0) else "k_fused")
    compare_fields(g, o, tol)
    if prec != "fp16":
        o0 = Oracle(*shape)
        o0.set_params(**dict(params, open_extrap=0))
        o0.init_fields(*dens)
        o0.step(40)
        _away_from(g, o0, tol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("tau", [(1.0, 1.0), (0.8, 1.2)])
def test_open_faces_extrapolated_with_particles(prec, tol, tau):
    """The extrapolated faces with particles (the lean kernel and its wall
    kernel at tau = 1, the copy-pipelined kernel otherwise): a pressure face
    below, a velocity face above; the first particle covers nodes of the
    plane next to the lower face, where the face values fall back to those
    of the boundary node, 40 steps."""
    shape = (32, 21, 23)
    params = dict(G=0.5, tau=tau, bc=(1, 1, 0), open=(1, 2), wall_u_hi=(0.02, 0.0, -0.01),
                  open_rho=(0.52, 0.5, 0.5, 0.5), hertz_K=20, hertz_sigma=8.0, hertz_rcap=7.0,
                  open_extrap=1)
    col = dict(pos=[[8.2, 5.3, 3.2], [22.6, 14.1, 12.4]], radius=[2.6, 3.2], mass=[400.0, 350.0],
               vel=[[0.01, 0.01, 0.0], [-0.01, 0.0, 0.02]], omega=[[0.0, 0.01, 0.0], [0.01, 0.0, 0.0]])
    g, o = run_both(shape, params, 40, prec, col, mixture_densities(shape, seed=47, amp=0.05))
    assert g.fused_kernel() == ("k_lean" if tau == (1.0, 1.0) else "k_fused_async")
    own = o.owner().reshape(shape[2], shape[1], shape[0])
    assert (own[1] == 0).any() and (own[0] < 0).all()
    compare_fields(g, o, tol)
    compare_colloids(g, o, tol)

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 storage 1e-12 relative (max-norm over the field, the state
after 100 steps); FP32 1e-5; FP16 deviation storage 1e-3.  Boxes are chosen to
span several thread blocks and ragged tails (nx a multiple of 4, odd ny, nz).
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
    g.step(steps)
    o.step(steps)
    return g, o


def rel(x, y):
    den = max(np.abs(y).max(), 1e-300)
    return np.abs(x - y).max() / den


def compare_fields(g, o, tol, tol_u=None):
    ga, gb, gu = g.get_fields()
    ra, rb, ru = o.get_fields()
    assert np.array_equal(g.owner(), o.owner())
    ea, eb, eu = rel(ga, ra), rel(gb, rb), rel(gu, ru)
    assert ea < tol and eb < tol, (ea, eb)
    assert eu < (tol_u or tol), eu
    return ea, eb, eu


def compare_colloids(g, o, tol):
    gc, rc = g.get_colloids(), o.get_colloids()
    for key in ("pos", "vel", "omega", "quat"):
        scale = {"pos": 1.0}.get(key, max(np.abs(rc[key]).max(), 1e-300))
        err = np.abs(gc[key] - rc[key]).max() / scale
        assert err < tol, (key, err)
    for term in ("F_liq", "T_liq", "F_s", "F_d", "F_c", "F_pair", "F_total"):
        gt, rt = g.term(term), o.term(term)
        scale = max(np.abs(rt).max(), 1e-12)
        assert np.abs(gt - rt).max() / scale < max(tol, 1e-10), term


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


def test_fp64_fluid_only_populations_exact():
    """No particles: every population matches the oracle to 1e-13."""
    shape = (16, 9, 7)
    g, o = run_both(shape, dict(G=0.9, tau=(0.7, 0.9)), 25, "fp64")
    for k in (0, 1):
        assert rel(g.populations(k), o.populations(k)) < 1e-13


def test_fp32_small_workload():
    """FP32 storage and arithmetic vs the FP64 oracle: 1e-5 on rho and u
    after 100 steps."""
    w = workload("small_fp64")
    g, o = run_both(w.shape, w.params, w.steps, "fp32", w.colloids(), w.densities())
    ga, gb, gu = g.get_fields()
    ra, rb, ru = o.get_fields()
    assert rel(ga, ra) < 1e-5 and rel(gb, rb) < 1e-5
    # velocities are ~1e-4 of the density scale: compare on the density scale
    assert np.abs(gu - ru).max() < 1e-5 * np.abs(ra).max()
    assert np.abs(g.get_colloids()["pos"] - o.get_colloids()["pos"]).max() < 1e-5


def test_fp16_storage_small_workload():
    """FP16 deviation storage (FP32 arithmetic) vs the FP64 oracle: 1e-3 on
    the fields after 100 steps."""
    w = workload("small_fp64")
    g, o = run_both(w.shape, w.params, w.steps, "fp16", w.colloids(), w.densities())
    ga, gb, gu = g.get_fields()
    ra, rb, ru = o.get_fields()
    assert rel(ga, ra) < 1e-3 and rel(gb, rb) < 1e-3
    assert np.abs(gu - ru).max() < 1e-3 * np.abs(ra).max()


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

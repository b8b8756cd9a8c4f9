"""The reduced-precision forms on a long demixing run: the bijel with
rho0 = 1 per component (G rho_tot = 1.3, supercritical), 96^3, R = 5
spheres at volume fraction 0.20.  After the first hundred steps the
spinodal pattern is chaotic, so individual fields of two runs part; the
observables of the morphology (interface measure A, interface link
crossings, domain size L of Eq. 40, structure-factor peak) are compared
against the FP64 run instead.

FP32 and FP16 deviation storage with stochastic rounding (the FP16 default)
must meet the stated bounds: fields within 1e-5 / 1e-3 at 100 steps, every
morphology observable within 1 % and the same S(k) peak up to 5000 steps.
FP16 rounded to nearest is recorded beside them: on a GB300 (seed 1) it
kept L within 0.7 % and the peak, but A drifted to 1.8 % and the link
crossings to 1.4 % at 5000 steps (A is dominated by the bulk phases,
1 - phi^2 = 0.4 per site at the coexistence densities 1.81 / 0.23, and
rounding the minor-phase populations, about 0.8 w_i below the shift, the same
way every step is a bias of about 0.3 % per population)."""
import numpy as np
import pytest

from paper_2004_04080_gb300 import analysis as an
from paper_2004_04080_gb300.workloads import workload

pytestmark = pytest.mark.gpu

CHECKS = (100, 2000, 5000)


def observables(prec, w, a, b, c, nearest=False):
    from paper_2004_04080_gb300.lbgb import LB_ROUND_NEAREST, LBLattice

    g = LBLattice(w.shape, prec, max_colloids=w.n_colloids)
    g.set_params(**w.params)
    g.init_fields(a, b)
    g.add_colloids(c["pos"], c["radius"], c["mass"])
    if nearest:
        g.set_rounding(LB_ROUND_NEAREST)
    out, done = {}, 0
    for s in CHECKS:
        g.step(s - done)
        done = s
        ra, rb, _ = g.get_fields()
        own = g.owner()
        phi = an.order_parameter(ra, rb, own)
        k, S = an.structure_factor(phi, w.shape)
        out[s] = dict(A=an.interface_measure(ra, rb, own), L=an.domain_size(k, S),
                      X=an.interface_crossings(ra, rb, w.shape, own),
                      kp=an.peak_wavenumber(k, S), rho=(ra, rb))
    return out


@pytest.fixture(scope="module")
def runs():
    w = workload("bijel_demix", (96, 96, 96))
    a, b = w.densities()
    c = w.colloids()
    r = {p: observables(p, w, a, b, c) for p in ("fp64", "fp32", "fp16")}
    r["fp16rn"] = observables("fp16", w, a, b, c, nearest=True)
    print("morphology", {p: {s: (v[s]["A"], v[s]["X"], v[s]["L"], v[s]["kp"]) for s in CHECKS} for p, v in r.items()})
    return r


def rel(x, y):
    return abs(x - y) / abs(y)


def test_the_mixture_demixes_and_coarsens(runs):
    r = runs["fp64"]
    assert r[5000]["A"] < 0.6 * r[100]["A"]
    assert r[5000]["L"] > 4 * r[100]["L"]


def test_fp32_morphology_tracks_fp64(runs):
    for s in CHECKS:
        assert rel(runs["fp32"][s]["A"], runs["fp64"][s]["A"]) < 1e-3, s
        assert rel(runs["fp32"][s]["L"], runs["fp64"][s]["L"]) < 2e-3, s
        assert runs["fp32"][s]["kp"] == runs["fp64"][s]["kp"]


def test_fp16_fields_then_morphology(runs):
    """FP16 storage with stochastic rounding (the default): the fields at 100
    steps within 1e-3 and, up to 5000 steps, every observable of the
    morphology within the 1 % target and the same S(k) peak."""
    r16, r64 = runs["fp16"], runs["fp64"]
    ra, rb = r16[100]["rho"]
    qa, qb = r64[100]["rho"]
    assert max(np.abs(ra - qa).max(), np.abs(rb - qb).max()) / max(qa.max(), qb.max()) < 1e-3
    print("interface crossings", {p: {s: runs[p][s]["X"] for s in CHECKS} for p in runs})
    for s in CHECKS:
        assert r16[s]["kp"] == r64[s]["kp"], s
    for s in CHECKS[1:]:
        assert rel(r16[s]["L"], r64[s]["L"]) < 1e-2, s
        assert rel(r16[s]["A"], r64[s]["A"]) < 1e-2, s
        assert rel(r16[s]["X"], r64[s]["X"]) < 1e-2, s
    assert rel(runs["fp32"][5000]["X"], r64[5000]["X"]) < 5e-3


def test_fp16_round_to_nearest_recorded(runs):
    """FP16 rounded to nearest, recorded beside the default: within 1e-3 on
    the fields at 100 steps and 1 % on A and L at 2000 steps, the same peak,
    and at 5000 steps L within 1 %, but the bulk-dominated A (measured 1.8 %)
    and the link crossings (1.4 %) beyond the 1 % target."""
    r16, r64 = runs["fp16rn"], runs["fp64"]
    ra, rb = r16[100]["rho"]
    qa, qb = r64[100]["rho"]
    assert max(np.abs(ra - qa).max(), np.abs(rb - qb).max()) / max(qa.max(), qb.max()) < 1e-3
    assert rel(r16[2000]["A"], r64[2000]["A"]) < 1e-2
    assert rel(r16[2000]["L"], r64[2000]["L"]) < 1e-2
    for s in CHECKS:
        assert r16[s]["kp"] == r64[s]["kp"], s
    assert rel(r16[5000]["L"], r64[5000]["L"]) < 1e-2
    assert rel(r16[5000]["X"], r64[5000]["X"]) < 2e-2
    assert rel(r16[5000]["A"], r64[5000]["A"]) < 3e-2

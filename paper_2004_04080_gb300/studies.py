"""Long runs of the paper's colloid studies, driven through the library's
public API, with the observables of ``analysis``:

* ``bijel_arrest``: the demixing mixture with R = 5.5 particles at volume
  fraction 0.20 (Sec. 5.1, the L(t) study of the 256^3 and 512^3 boxes):
  the domain size L(t) of Eq. 40 grows while the mixture demixes and is
  arrested once the particles jam the interfaces; without particles it keeps
  growing.
* ``sheared_bijel``: a bijel confined between two walls moving in opposite
  directions (Sec. 5.3, confined bijels under shear): after an equilibration
  at rest the walls move at +-U, and for large enough U the coarsening
  revives.  The paper's walls are normal to x and move along z, with no-slip
  walls normal to y; here the moving walls are normal to z and move along x
  (the library's walls), and y is periodic.

Each returns a dict with the time series (steps, L, the S(k) peak
wavenumber, the interface crossings and A) and the run's description.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import analysis
from .lbgb import LBLattice
from .workloads import n_for_fraction, workload


def _observe(lat, shape):
    a, b, _ = lat.get_fields()
    owner = lat.owner()
    phi = analysis.order_parameter(a, b, owner)
    k, Sk = analysis.structure_factor(phi, shape)
    return {"L": analysis.domain_size(k, Sk), "k_peak": analysis.peak_wavenumber(k, Sk),
            "crossings": analysis.interface_crossings(a, b, shape, owner),
            "A": analysis.interface_measure(a, b, owner)}


def _run(lat, shape, steps, every, t0=0, log=None):
    series = []
    t = t0
    while t < t0 + steps:
        n = min(every, t0 + steps - t)
        lat.step(n)
        t += n
        o = _observe(lat, shape)
        o["step"] = t
        series.append(o)
        if log:
            log("step %d: L %.2f, k_peak %.4f, crossings %d" % (t, o["L"], o["k_peak"], o["crossings"]))
    return series


def bijel_arrest(n=256, phi=0.20, steps=30000, every=1000, particles=True, prec="fp32", device="cuda",
                 log=None):
    """The colloid benchmark's physics (workload janus_lub256: Janus particles,
    lubrication, Hertz, pair list) in an n^3 box at volume fraction phi,
    or the same mixture without particles."""
    shape = (n, n, n)
    w = workload("janus_lub256", scale=shape)
    w = dataclasses.replace(w, n_colloids=n_for_fraction(shape, w.radius, phi) if particles else 0)
    c = w.colloids()
    lat = LBLattice(shape, prec, max_colloids=max(w.n_colloids, 1), device=device)
    lat.set_params(**w.params)
    a, b = w.densities()
    lat.init_fields(a, b)
    if c is not None:
        lat.add_colloids(c["pos"], c["radius"], c["mass"], quat=c.get("quat"))
    t0 = time.perf_counter()
    series = _run(lat, shape, steps, every, log=log)
    return {"study": "bijel arrest", "box": list(shape), "particles": w.n_colloids, "phi": phi if particles else 0.0,
            "prec": prec, "steps": steps, "seconds": round(time.perf_counter() - t0, 1),
            "pair_list_builds": lat.pair_list_builds() if particles else 0, "series": series}


def sheared_bijel(shape=(1024, 128, 128), phi=0.15, wall_speed=0.005, equil=30000, shear=40000, every=2000,
                  prec="fp32", device="cuda", log=None):
    """Demixing mixture (1.0 + 1.0, standard deviation 0.004, G = 0.65) with
    neutral R = 5.5 particles at volume fraction phi between walls normal to
    z, at rest for ``equil`` steps, then moving at -+wall_speed along x for
    ``shear`` steps.  The soft particle-wall spring is 20 (the paper gives
    none for this study): with the shear workload's 1 the capillary forces of
    the demixing interfaces (up to about 28 per particle) push particles
    through it into the wall within a thousand steps."""
    base = workload("shear512", scale=shape)
    R = base.radius
    params = dict(base.params, rho0=(1.0, 1.0), wall_u_lo=(0.0, 0.0, 0.0), wall_u_hi=(0.0, 0.0, 0.0),
                  side_wall_k=20.0)
    w = dataclasses.replace(base, params=params, n_colloids=n_for_fraction(shape, R, phi), mean=1.0,
                            amp=0.004 * np.sqrt(3.0))
    c = w.colloids()
    lat = LBLattice(shape, prec, max_colloids=w.n_colloids, device=device)
    lat.set_params(**params)
    a, b = w.densities()
    lat.init_fields(a, b)
    lat.add_colloids(c["pos"], c["radius"], c["mass"])
    t0 = time.perf_counter()
    series = _run(lat, shape, equil, every, log=log)
    lat.set_params(**dict(params, wall_u_lo=(-wall_speed, 0.0, 0.0), wall_u_hi=(wall_speed, 0.0, 0.0)))
    series += _run(lat, shape, shear, every, t0=equil, log=log)
    return {"study": "confined bijel under shear", "box": list(shape), "particles": w.n_colloids, "phi": phi,
            "wall_speed": wall_speed, "equil": equil, "shear": shear, "prec": prec,
            "seconds": round(time.perf_counter() - t0, 1), "series": series}

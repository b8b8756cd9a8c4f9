"""Inputs of the Pickering-emulsion workload, computed with the FP64 oracle.

Test infrastructure (it runs the oracle only); from the repository root:

    python tests/golden/calibrate_pickering.py

writes tests/golden/pickering_calibration.json with

1. the coexistence densities of the demixing mixture (G = 0.65, rho0 = 1 per
   component, tau = 1; G rho_tot = 1.3 exceeds the threshold 2 - 1/tau = 1):
   a flat slab of A-rich fluid between B-rich fluid relaxed to equilibrium,
   the bulk densities read at the middle of each phase;
2. the wetting parameter Delta (zeta_A = +Delta, zeta_B = -Delta, Eq. 20) for
   a contact angle of 77 degrees measured through the A phase.  The paper
   gives no relation between Delta and the angle; it is measured: one free
   sphere of radius R = 5 set on a flat A|B interface settles with its centre
   a depth d = R cos(theta) on the A side of the far-field interface plane
   (theta = 90 degrees, d = 0, for Delta = 0).  d is measured for a few Delta
   and Delta(77) is interpolated linearly between the two bracketing values.
"""
from __future__ import annotations

import json
import math
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "pickering_calibration.json")

G = 0.65
RHO0 = (1.0, 1.0)
R = 5.0
THETA = 77.0
DELTAS = (0.0, 0.01, 0.02, 0.03, 0.035, 0.04, 0.05, 0.08)
CA_SHAPE = (32, 32, 48)
CA_STEPS = 4000
CA_EVERY = 100
CA_TAIL = 1000  # steps averaged at the end


def _oracle(shape, maxc):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from oracle import Oracle

    return Oracle(*shape, maxc)


def tanh_profile(z, z0, width=2.0):
    """1 below the plane z0, 0 above, tanh of the given width."""
    return 0.5 * (1.0 - np.tanh((z - z0) / width))


def coexistence(steps=6000):
    """Bulk (rho_A, rho_B) of the A-rich and B-rich phases of a relaxed slab."""
    shape = (4, 4, 64)
    nz = shape[2]
    N = int(np.prod(shape))
    z = np.arange(N) // (shape[0] * shape[1])
    inA = tanh_profile(np.abs(z - 31.5), 16.0)  # A-rich for |z - 31.5| < 16
    hi, lo = 1.8, 0.2
    a = lo + (hi - lo) * inA
    b = lo + (hi - lo) * (1.0 - inA)
    o = _oracle(shape, 0)
    o.set_params(tau=(1.0, 1.0), G=G, rho0=RHO0)
    o.init_fields(a, b)
    hist = []
    for _ in range(steps // 1000):
        o.step(1000)
        ra, rb, _ = o.get_fields()
        ra = ra.reshape(nz, -1).mean(axis=1)
        rb = rb.reshape(nz, -1).mean(axis=1)
        midA = slice(28, 36)
        midB = np.r_[0:4, 60:64]
        hist.append((ra[midA].mean(), rb[midA].mean(), ra[midB].mean(), rb[midB].mean()))
    last, prev = np.array(hist[-1]), np.array(hist[-2])
    return dict(A_rich=[last[0], last[1]], B_rich=[last[2], last[3]],
                change_last_1000_steps=float(np.abs(last - prev).max()), steps=steps)


def settle(args):
    """Depth of a free sphere's centre below the far-field interface (on the
    A side), for one Delta: time series and the mean over the last steps."""
    delta, rich, poor = args
    shape = CA_SHAPE
    nx, ny, nz = shape
    N = nx * ny * nz
    s = np.arange(N)
    x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
    z_int0 = nz / 2 - 0.5
    # A for 0 <= z < nz/2, B above; the second interface is the periodic seam
    dz = np.mod(z - (nz / 4 - 0.5) + nz / 2, nz) - nz / 2
    inA = tanh_profile(np.abs(dz), nz / 4)
    a = poor + (rich - poor) * inA
    b = poor + (rich - poor) * (1.0 - inA)
    o = _oracle(shape, 1)
    o.set_params(tau=(1.0, 1.0), G=G, rho0=RHO0, zeta=(delta, -delta))
    o.init_fields(a, b)
    c = (nx / 2, ny / 2, z_int0)
    o.add_colloids([list(c)], R, 4.0 / 3.0 * math.pi * R ** 3)
    far = ((x - c[0]) ** 2 + (y - c[1]) ** 2) >= 12.0 ** 2
    series = []
    for t in range(CA_STEPS // CA_EVERY):
        o.step(CA_EVERY)
        ra, rb, _ = o.get_fields()
        own = o.owner()
        fl = far & (own < 0)
        phi = np.where(fl, (ra - rb) / np.maximum(ra + rb, 1e-300), 0.0)
        prof = np.bincount(z, weights=phi, minlength=nz) / np.maximum(np.bincount(z, weights=fl, minlength=nz), 1)
        # A (phi > 0) below, B above: the crossing near the middle of the box
        k = int(np.argmax((prof[:-1] > 0) & (prof[1:] <= 0) & (np.arange(nz - 1) >= nz // 4)))
        z_int = k + prof[k] / (prof[k] - prof[k + 1])
        pos = o.get_colloids()["pos"][0]
        series.append(((t + 1) * CA_EVERY, float(z_int - pos[2]), float(pos[2]), float(z_int)))
    tail = [d for (t, d, _, _) in series if t > CA_STEPS - CA_TAIL]
    return dict(delta=delta, depth=float(np.mean(tail)), depth_spread=float(np.ptp(tail)), series=series)


def main():
    co = coexistence()
    rich = 0.5 * (co["A_rich"][0] + co["B_rich"][1])
    poor = 0.5 * (co["A_rich"][1] + co["B_rich"][0])
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(DELTAS), os.cpu_count() or 1)) as pool:
        runs = pool.map(settle, [(d, rich, poor) for d in DELTAS])
    target = R * math.cos(math.radians(THETA))
    depths = [r["depth"] for r in runs]
    delta77 = None
    for i in range(len(DELTAS) - 1):
        if (depths[i] - target) * (depths[i + 1] - target) <= 0 and depths[i + 1] != depths[i]:
            f = (target - depths[i]) / (depths[i + 1] - depths[i])
            delta77 = DELTAS[i] + f * (DELTAS[i + 1] - DELTAS[i])
            break
    out = dict(
        what="Pickering workload inputs from the FP64 oracle (tests/golden/calibrate_pickering.py)",
        G=G, rho0=list(RHO0), tau=[1.0, 1.0],
        coexistence=co, rho_rich=rich, rho_poor=poor,
        contact_angle=dict(theta_deg=THETA, radius=R, target_depth=target, shape=list(CA_SHAPE),
                           steps=CA_STEPS, averaged_last=CA_TAIL,
                           runs=[dict(delta=r["delta"], depth=r["depth"], depth_spread=r["depth_spread"])
                                 for r in runs],
                           series={str(r["delta"]): r["series"] for r in runs}),
        delta_77=delta77,
    )
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(dict(coexistence=co, runs=out["contact_angle"]["runs"], delta_77=delta77), indent=1))


if __name__ == "__main__":
    main()

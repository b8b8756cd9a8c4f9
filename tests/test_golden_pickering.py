"""The Pickering inputs measured with the oracle (tests/golden/
calibrate_pickering.py -> pickering_calibration.json), checked against what
the model's symmetry fixes, and the coexistence slab re-run."""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def calib():
    with open(os.path.join(HERE, "golden", "pickering_calibration.json")) as f:
        return json.load(f)


def test_coexistence_is_symmetric_and_converged():
    """With equal tau and rho0 the model is symmetric under A <-> B, so the
    A-rich and B-rich bulk phases are mirror images; the slab had settled."""
    c = calib()
    co = c["coexistence"]
    assert abs(co["A_rich"][0] - co["B_rich"][1]) < 1e-12
    assert abs(co["A_rich"][1] - co["B_rich"][0]) < 1e-12
    assert co["change_last_1000_steps"] < 1e-3
    rich, poor = c["rho_rich"], c["rho_poor"]
    assert rich > 1.5 and 0.0 < poor < 0.5  # demixed: G rho_tot = 1.3 > 2 - 1/tau = 1


def test_contact_angle_sweep():
    """Neutral wetting (Delta = 0) leaves the sphere centred on the interface
    (90 degrees, by the A <-> B symmetry); the depth on the A side does not
    decrease with Delta; Delta(77 deg) interpolates the bracketing runs."""
    c = calib()
    ca = c["contact_angle"]
    runs = sorted(ca["runs"], key=lambda r: r["delta"])
    assert runs[0]["delta"] == 0.0 and abs(runs[0]["depth"]) < 1e-10
    d = [r["depth"] for r in runs]
    assert all(b >= a - 1e-3 for a, b in zip(d, d[1:]))
    target = ca["radius"] * math.cos(math.radians(ca["theta_deg"]))
    assert abs(target - ca["target_depth"]) < 1e-12
    i = next(k for k in range(len(runs) - 1) if d[k] <= target <= d[k + 1])
    f = (target - d[i]) / (d[i + 1] - d[i])
    assert abs(c["delta_77"] - (runs[i]["delta"] + f * (runs[i + 1]["delta"] - runs[i]["delta"]))) < 1e-12
    for r in runs[:-1]:
        assert r["depth_spread"] < 0.05  # settled over the averaged steps


def test_coexistence_slab_reproduces():
    """The slab of the calibration, re-run with the oracle (regression of the
    stored values)."""
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import calibrate_pickering as cp

    co = cp.coexistence(steps=6000)
    stored = calib()["coexistence"]
    assert np.allclose(co["A_rich"], stored["A_rich"], rtol=0, atol=1e-12)
    assert np.allclose(co["B_rich"], stored["B_rich"], rtol=0, atol=1e-12)

"""The observables of the analysis module against closed forms (CPU)."""
import math

import numpy as np
import pytest

from paper_2004_04080_gb300 import analysis as an


def test_structure_factor_of_a_plane_wave_peaks_at_its_wavenumber():
    shape = (32, 16, 16)
    x = np.arange(32)
    phi = np.tile(0.3 * np.cos(2 * math.pi * 4 * x / 32), 16 * 16)
    k, S = an.structure_factor(phi, shape)
    assert abs(an.peak_wavenumber(k, S) - 2 * math.pi * 4 / 32) < 1e-12
    # a single shell holds the power: sum_k S(k) counts (0.3/2)^2 N per +-k mode over its shell
    assert np.count_nonzero(S > 1e-9 * S.max()) == 1
    # Eq. 40 for one wavenumber: L = 2 pi / k
    assert abs(an.domain_size(k, S) - 32 / 4) < 1e-9


def test_interface_measure_counts_mixed_sites_only():
    a = np.array([1.0, 0.0, 0.5, 0.3, 0.0])
    b = np.array([0.0, 2.0, 0.5, 0.3, 0.0])
    owner = np.array([-1, -1, -1, -1, 3])
    # pure sites contribute 0, mixed sites 1, the particle node nothing
    assert an.interface_measure(a, b, owner) == 2.0
    phi = an.order_parameter(a, b, owner)
    assert phi[0] == 1.0 and phi[1] == -1.0 and phi[4] == 0.0


def _crossings_by_loops(phi, fluid, shape):
    """the link count written out site by site"""
    nx, ny, nz = shape
    n = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                s = x + nx * (y + ny * z)
                for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    t = (x + d[0]) % nx + nx * (((y + d[1]) % ny) + ny * ((z + d[2]) % nz))
                    if fluid[s] and fluid[t] and phi[s] * phi[t] < 0:
                        n += 1
    return n


def test_interface_crossings_of_flat_slabs_and_a_random_field():
    shape = (6, 5, 8)
    nx, ny, nz = shape
    z = np.arange(nx * ny * nz) // (nx * ny)
    # a slab 2 <= z < 5 of B in A: two flat interfaces of nx * ny sites each,
    # whatever the bulk densities
    for rich, poor in ((1.0, 0.0), (1.81, 0.23)):
        inB = (z >= 2) & (z < 5)
        a = np.where(inB, poor, rich)
        b = np.where(inB, rich, poor)
        assert an.interface_crossings(a, b, shape) == 2 * nx * ny
    # random fields with particle nodes: the vectorised count equals the loops
    rng = np.random.default_rng(3)
    a, b = rng.random(nx * ny * nz), rng.random(nx * ny * nz)
    owner = np.where(rng.random(nx * ny * nz) < 0.2, 1, -1)
    phi = an.order_parameter(a, b, owner)
    assert an.interface_crossings(a, b, shape, owner) == _crossings_by_loops(phi, owner < 0, shape)


@pytest.mark.gpu
def test_study_drivers_run_small():
    """The long-run study drivers on small boxes: the bijel's domain size grows
    from the mixed start, and the sheared run switches the walls on."""
    from paper_2004_04080_gb300 import studies

    r = studies.bijel_arrest(n=48, steps=400, every=200)
    Ls = [o["L"] for o in r["series"]]
    assert r["particles"] > 0 and len(Ls) == 2 and Ls[1] > Ls[0] > 0
    s = studies.sheared_bijel(shape=(96, 32, 32), equil=200, shear=200, every=100, wall_speed=0.01)
    assert [o["step"] for o in s["series"]] == [100, 200, 300, 400]
    assert all(o["L"] > 0 for o in s["series"])

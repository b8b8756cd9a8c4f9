"""The observables of the analysis module against closed forms (CPU)."""
import math

import numpy as np

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

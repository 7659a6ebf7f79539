"""Pins of the oracle's particle summation (Sec. 5.1, Eq. sum), CPU only.

With equal weights 4 pi a^2 / N on N nearly uniform points of a sphere, the direct sum is a quadrature of the
single- and double-layer potentials of a uniform density, whose exterior values follow from the addition
theorem G = (ik/4pi) sum (2n+1) j_n(k|y|) h_n(k|x|) P_n:
  single layer  int_S G(x, y) dS_y            = a sin(ka) e^{ikr} / (k r)
  double layer  int_S dG/dn_y(x, y) dS_y      = i k^2 a^2 j_0'(ka) h_0(kr)      (outward normals)
"""
import math

import numpy as np

from oracle import oracle as O
from paper_1311_5202_gb300 import inputs


def _layers(N=20000, a=1.0, k=3.0):
    x, n = inputs.sphere_points(N, a)
    q = np.full(N, 4.0 * math.pi * a * a / N, dtype=complex)
    t = np.array([[0.0, 0.0, 2.0], [1.5, 0.3, -1.0], [-2.5, 1.0, 0.5]])
    r = np.linalg.norm(t, axis=1)
    pS = O.particle_field(x, n, k, q, t, alpha=0.0)
    pSD = O.particle_field(x, n, k, q, t, alpha=1.0)
    z = k * a
    j0p = (z * math.cos(z) - math.sin(z)) / (z * z)
    refS = a * math.sin(z) * np.exp(1j * k * r) / (k * r)
    refD = 1j * k * k * a * a * j0p * np.exp(1j * k * r) / (1j * k * r)
    return pS, pSD - pS, refS, refD


def test_particle_field_matches_sphere_layer_potentials():
    pS, pD, refS, refD = _layers()
    assert np.max(np.abs(pS - refS) / np.abs(refS)) < 2e-5
    assert np.max(np.abs(pD - refD) / np.abs(refD)) < 2e-5


def test_particle_rows_equal_field_at_the_sources_minus_self():
    """The row sum at a source point equals the field sum over all other sources (the self term dropped)."""
    N, k = 3000, 7.0
    x, n = inputs.sphere_points(N, 1.0)
    q = inputs.complex_gaussian(N, 3)
    rows = np.array([0, 17, 2999])
    pr = O.particle_rows(x, n, k, q, rows)
    for r, i in enumerate(rows):
        keep = np.arange(N) != i
        pf = O.particle_field(x[keep], n[keep], k, q[keep], x[i])
        assert abs(pr[r] - pf[0]) <= 1e-12 * abs(pf[0])


def test_table1_points_per_wavelength():
    """The synthetic Table-1 workloads: ~20 points per wavelength on the unit sphere (k = 8 pi at 73,728)."""
    for N, k in inputs.TABLE1:
        kk = inputs.table1_k(N)
        assert abs(kk / k - 1.0) < 0.06, (N, k, kk)

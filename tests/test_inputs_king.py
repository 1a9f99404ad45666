"""The King sphere of the isolated test (Sec. 3.5): the lowered-isothermal
profile the seeded input builder integrates, pinned to values that do not
come from this code.

* The concentration c = log10(r_t / r_0) of King's models is a tabulated
  function of the central depth W0 (King 1966; Binney & Tremaine 2008,
  Sec. 4.3.3c): about 0.67, 1.03, 1.25, 1.53 and 2.12 for W0 = 3, 5, 6, 7, 9.
  A dropped factor in the ODE (the 9 of r_0^2 = 9 sigma^2 / (4 pi G rho_0))
  or in the density law rho(W) moves every one of them.
* For small W the density law is rho_1 (8 / (15 sqrt(pi))) W^(5/2) (1 + 2 W / 7
  + ...): the series of e^W erf(sqrt W) cancels the subtracted terms up to
  W^(3/2).  Checked on small W.
* The central 1D dispersion falls below sigma and tends to sigma as W0 grows
  (the truncation of the Maxwellian matters less).
"""
import math

import numpy as np
import pytest

from paper_1206_6152_gb300 import inputs as I


@pytest.mark.parametrize("w0,c", [(3.0, 0.67), (5.0, 1.03), (6.0, 1.25), (7.0, 1.53), (9.0, 2.12)])
def test_king_concentration_matches_tabulated_values(w0, c):
    p = I.king_profile(w0)
    assert abs(math.log10(p.r_t) - c) < 0.01, (w0, p.r_t)
    # W decreases monotonically from W0 to 0 at the tidal radius
    assert p.W[0] == w0 and p.W[-1] == 0.0
    assert np.all(np.diff(p.W) <= 1e-12)


def test_king_density_law_small_w_series():
    W = np.array([1e-3, 3e-3, 1e-2])
    lead = 8.0 / (15.0 * math.sqrt(math.pi)) * W ** 2.5
    rel = I._king_density(W) / lead - 1.0
    assert np.all(np.abs(rel - 2.0 * W / 7.0) < W ** 2), rel


def test_king_central_dispersion_increases_towards_sigma():
    s = [I.king_profile(w0).sigma_c for w0 in (1.0, 3.0, 6.0, 9.0)]
    assert all(a < b for a, b in zip(s, s[1:])), s
    assert 0.95 < s[2] < 1.0 and 0.99 < s[3] < 1.0, s

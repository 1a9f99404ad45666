"""Pins of the oracle's 1D PFC update (Sec. 2.1) against what the paper and
the mathematics fix, independent of the oracle's own code path:

* integer Courant number -> exact shift (free streaming is a translation,
  Sec. 3.1);
* exactness for quadratic data when the slope corrector is inactive (the
  reconstruction is third order, Sec. 2.1);
* the update equals the cell average of the shifted reconstruction
  (Eq. conserve), computed here by direct integration of a test-side
  reconstruction, for every shift and both boundary rules;
* mass conservation, positivity and the maximum principle (Sec. 2.1);
* translation equivariance.
"""
import numpy as np
import pytest

from oracle import vp_oracle as O


def cell_avg_poly(coef, lo, hi):
    """Average of sum_k coef[k] x^k over [lo, hi]."""
    P = np.polynomial.polynomial.polyint(coef)
    return (np.polynomial.polynomial.polyval(hi, P)
            - np.polynomial.polynomial.polyval(lo, P)) / (hi - lo)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("s", [-7, -3, -1, 1, 2, 5, 12])
def test_integer_shift_is_exact(periodic, s):
    rng = np.random.default_rng(10 + s)
    n = 16
    f = rng.random(n) ** 3
    out = O.pfc_line(f, float(s), periodic)
    if periodic:
        expect = np.roll(f, s)
    else:
        expect = np.zeros(n)
        for i in range(n):
            if 0 <= i - s < n:
                expect[i] = f[i - s]
    # the conservative form f + Phi^- - Phi^+ sums whole cells, so the shift
    # is exact up to the rounding of those sums
    assert np.allclose(out, expect, rtol=0, atol=4e-16 * abs(s) * f.max())


@pytest.mark.parametrize("alpha", [0.1, 0.37, 0.5, 0.93, 1.25, 2.6, -0.2, -0.71, -1.4, -3.05])
def test_quadratic_exact_when_unlimited(alpha):
    # smooth increasing quadratic with a large offset: the corrector stays
    # inactive away from the line maximum and the outflow ends
    n, h = 40, 0.1
    coef = [50.0, 1.0, 0.3]
    x = (np.arange(n) + 0.5) * h
    f = np.array([cell_avg_poly(coef, xi - h / 2, xi + h / 2) for xi in x])
    out = O.pfc_line(f, alpha, False)
    shift = alpha * h
    margin = int(np.ceil(abs(alpha))) + 3
    for i in range(margin, n - margin):
        exact = cell_avg_poly(coef, x[i] - h / 2 - shift, x[i] + h / 2 - shift)
        assert abs(out[i] - exact) <= 1e-12 * exact, (i, out[i], exact)


def _limited_differences(g, j, finf):
    """E+ and E- of cell j for a line g with ghosts already applied
    (Filbet et al. 2001 corrector, clamp form)."""
    f0, fp, fm = g[j], g[j + 1], g[j - 1]
    ep = min(max(fp - f0, -2 * (finf - f0)), 2 * f0)
    em = min(max(f0 - fm, -2 * f0), 2 * (finf - f0))
    return ep, em


def _reconstruction_integral(f, periodic, lo, hi):
    """Integral over [lo, hi] (cell units, cell i = [i, i+1)) of the piecewise
    quadratic whose cell averages are f and whose one-sided differences are
    the corrected ones.  Ghost cells: periodic copies or zeros."""
    n = len(f)
    finf = max(f)
    pad = 40
    ext = np.zeros(n + 2 * pad + 2)
    for k in range(-pad - 1, n + pad + 1):
        if periodic:
            ext[k + pad + 1] = f[k % n]
        elif 0 <= k < n:
            ext[k + pad + 1] = f[k]
    total = 0.0
    j0, j1 = int(np.floor(lo)), int(np.ceil(hi))
    for j in range(j0, j1):
        a_, b_ = max(lo, j), min(hi, j + 1)
        if b_ <= a_:
            continue
        jj = j + pad + 1
        ep, em = _limited_differences(ext, jj, finf)
        b = 0.5 * (ep + em)
        c = 0.5 * (ep - em)
        a = ext[jj] - c / 12
        # local coordinate t = x - (j + 1/2)
        P = np.polynomial.polynomial.polyint([a, b, c])
        total += (np.polynomial.polynomial.polyval(b_ - j - 0.5, P)
                  - np.polynomial.polynomial.polyval(a_ - j - 0.5, P))
    return total


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.0, 0.25, 0.5, 0.999, 1.5, 3.3, -0.25, -0.8, -2.4])
def test_update_is_average_of_shifted_reconstruction(periodic, alpha):
    rng = np.random.default_rng(7)
    for trial in range(4):
        n = 9
        f = rng.random(n) * (rng.random(n) > 0.3)
        out = O.pfc_line(f, alpha, periodic)
        for i in range(n):
            expect = _reconstruction_integral(f, periodic, i - alpha, i + 1 - alpha)
            assert abs(out[i] - expect) <= 1e-13 * max(1.0, abs(expect)), (trial, i)


@pytest.mark.parametrize("alpha", [0.05, 0.45, 0.99, 1.7, -0.3, -2.2])
def test_mass_positivity_maximum_principle(alpha):
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(3, 40))
        f = rng.random(n) * (rng.random(n) > 0.5) * 10 ** rng.uniform(-5, 3)
        out = O.pfc_line(f, alpha, True)
        assert abs(out.sum() - f.sum()) <= 1e-13 * f.sum() + 1e-300
        assert out.min() >= 0.0
        assert out.max() <= f.max() * (1 + 1e-13)
        outf = O.pfc_line(f, alpha, False)
        assert outf.min() >= 0.0
        assert outf.sum() <= f.sum() * (1 + 1e-13)
        assert outf.max() <= f.max() * (1 + 1e-13)


def test_translation_equivariance():
    rng = np.random.default_rng(5)
    f = rng.random(23)
    for alpha in (0.3, -1.6, 2.2):
        a = O.pfc_line(np.roll(f, 5), alpha, True)
        b = np.roll(O.pfc_line(f, alpha, True), 5)
        assert np.allclose(a, b, rtol=0, atol=1e-14)


def test_outflow_removes_what_crosses_the_end():
    # a single full cell next to the right end leaves by the fraction the
    # reconstruction puts beyond the face (here beta of a flat-topped cell
    # is limited, so compare with the reconstruction integral)
    f = np.array([0.0, 0.0, 0.0, 1.0])
    out = O.pfc_line(f, 0.4, False)
    gone = f.sum() - out.sum()
    assert gone == pytest.approx(_reconstruction_integral(f, False, 3.6, 4.0), abs=1e-15)

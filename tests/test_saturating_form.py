"""The CUDA kernels evaluate the slope-corrected PFC flux (Sec. 2.1, with
the corrector of Filbet, Sonnendruecker & Bertrand 2001) in a saturating
form: with F = 2 f_inf, h_j = -f_j / F, r3 = 3 / F and sat(x) =
min(max(x, 0), 1),

    s1 = sat(r3 f_j + h_{j+1}),  s2 = sat(r3 f_j + h_{j-1}),
    phi_j = min(K0 f_j + A1 s1 + A2 s2, f_j),
    K0 = c0 + 2 (c1 - c2),  A1 = -c1 F,  A2 = c2 F     (u > 0; u < 0 mirrored),

which is an algebraic rewriting of the clamped differences
E+ = clamp(f_{j+1} - f_j, -(F - 2 f_j), 2 f_j), E- = clamp(f_j - f_{j-1},
-2 f_j, F - 2 f_j).  The oracle uses the corrector's ratio form.  This CPU
test restates the saturating form in numpy (FP64) and checks that it gives
the oracle's update to rounding, for sub-cell shifts of both signs, both
boundary rules, lines with zeros, plateaus at the maximum and steep
gradients (every arm of both clamps taken), and the all-zero line.

The generic kernels (any whole-cell shift) use the clamp form itself with
the update telescoped to f_{i-s} - phi_{i-s} + phi_{i-s-1} and an outflow
tally of the cells and partial flux that cross the end; that formulation is
checked against the oracle's sum of face fluxes the same way, and its tally
against the mass the line loses."""
import numpy as np
import pytest

from oracle import vp_oracle as O


def sat(x):
    # fmin/fmax as the kernels' saturation: NaN goes to 0
    return np.fmin(np.fmax(x, 0.0), 1.0)


def saturating_update(f, alpha, periodic):
    if alpha < 0:
        return saturating_update(f[::-1].copy(), -alpha, periodic)[::-1]
    # a line whose maximum is below 2^-968 is swept scaled by 2^968 (exact:
    # the update is positively homogeneous) and scaled back, as the FP64
    # kernels do, so that -1/F and the weights stay finite and normal
    fmax = max(f.max(), 0.0)
    if 0.0 < fmax < 2.0 ** -968:
        return saturating_update(f * 2.0 ** 968, alpha, periodic) * 2.0 ** -968
    b = alpha
    c0, c1, c2 = b, b * (1 - b) * (2 - b) / 6, b * (1 - b) * (1 + b) / 6
    F = 2.0 * fmax
    ninvF = -1.0 / F if F > 0 else 0.0
    h = f * ninvF
    r3 = -3.0 * ninvF
    if periodic:
        hp, hm = np.roll(h, -1), np.roll(h, 1)
    else:
        hp = np.append(h[1:], 0.0)
        hm = np.insert(h[:-1], 0, 0.0)
    s1, s2 = sat(r3 * f + hp), sat(r3 * f + hm)
    phi = np.minimum((c0 + 2 * (c1 - c2)) * f - c1 * F * s1 + c2 * F * s2, f)
    inflow = np.roll(phi, 1) if periodic else np.insert(phi[:-1], 0, 0.0)
    return f - phi + inflow


def lines(rng, n):
    yield rng.random(n) + 0.05                                  # smooth positive
    g = rng.random(n) ** 4                                      # steep, near-zero cells
    g[rng.integers(0, n, 3)] = 0.0
    yield g
    p = rng.random(n)
    p[3:7] = p.max()                                            # a plateau at the maximum
    yield p
    t = np.zeros(n)
    t[n // 3: n // 2] = 1.0                                     # a top hat
    yield t
    yield np.zeros(n)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.03, 0.25, 0.5, 0.77, 0.999, -0.11, -0.5, -0.93])
def test_saturating_form_is_the_corrector(periodic, alpha):
    rng = np.random.default_rng(int(1000 * abs(alpha)) + periodic)
    for f in lines(rng, 19):
        got = saturating_update(f, alpha, periodic)
        ref = O.pfc_line(f, alpha, periodic)
        scale = max(f.max(), 1e-300)
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-15 * scale)


def test_every_clamp_arm_is_taken():
    """The lines above reach both bounds of both clamps (so the comparison
    covers every arm, not only the unlimited one)."""
    rng = np.random.default_rng(0)
    seen = set()
    for f in lines(rng, 19):
        F = 2.0 * f.max()
        if F == 0:
            continue
        fp, fm = np.append(f[1:], 0.0), np.insert(f[:-1], 0, 0.0)
        for d, lo, hi, tag in ((fp - f, -(F - 2 * f), 2 * f, "E+"), (f - fm, -2 * f, F - 2 * f, "E-")):
            seen |= {tag + "lo" for x, a in zip(d, lo) if x < a}
            seen |= {tag + "hi" for x, a in zip(d, hi) if x > a}
            seen |= {tag + "in" for x, a, c in zip(d, lo, hi) if a < x < c}
    assert seen == {"E+lo", "E+hi", "E+in", "E-lo", "E-hi", "E-in"}, seen


def clamp_flux(fm, f0, fp, finf, c0, c1, c2):
    """The clamp form of the corrected partial flux (the generic kernels)."""
    a, b = 2 * f0, 2 * (finf - f0)
    ep = np.minimum(np.maximum(fp - f0, -b), a)
    em = np.minimum(np.maximum(f0 - fm, -a), b)
    return np.minimum(np.maximum(c0 * f0 + c1 * ep + c2 * em, 0.0), f0)


def shifted_update(f, alpha, periodic):
    """Any shift alpha = s + beta (u < 0 mirrored): the update telescoped to
    f_{i-s} - phi_{i-s}(beta) + phi_{i-s-1}(beta); with outflow the cells and
    partial fluxes that cross the end are returned as the outflow."""
    if alpha < 0:
        out, lost = shifted_update(f[::-1].copy(), -alpha, periodic)
        return out[::-1], lost
    s = int(np.floor(alpha))
    b = alpha - s
    c0, c1, c2 = b, b * (1 - b) * (2 - b) / 6, b * (1 - b) * (1 + b) / 6
    n = f.size
    finf = max(f.max(), 0.0)

    def cell(j):
        if periodic:
            return f[j % n]
        return f[j] if 0 <= j < n else 0.0

    def phi(j):
        if not periodic and not 0 <= j < n:
            return 0.0
        return float(clamp_flux(cell(j - 1), cell(j), cell(j + 1), finf, c0, c1, c2))

    out = np.array([cell(i - s) - phi(i - s) + phi(i - s - 1) for i in range(n)])
    lost = 0.0 if periodic else sum(f[max(n - s, 0):]) + (phi(n - 1 - s) if n - 1 - s >= 0 else 0.0)
    return out, lost


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.3, 0.81, -0.47])
@pytest.mark.parametrize("scale", [1e-310, 2.0 ** -1000, 5e-324 * 7, 1e-300])
def test_subnormal_line_maximum(periodic, alpha, scale):
    """Lines whose maximum is subnormal or barely normal: the rescaled
    saturating form gives the oracle's update to the line's own rounding
    (no reciprocal overflow, no loss of the corrector)."""
    rng = np.random.default_rng(int(1e3 * abs(alpha)) + periodic)
    for f in lines(rng, 19):
        g = f * scale
        got = saturating_update(g, alpha, periodic)
        ref = O.pfc_line(g, alpha, periodic)
        assert np.all(np.isfinite(got)) and got.min() >= 0.0
        # subnormal arithmetic rounds to multiples of 2^-1074 in both forms
        atol = 2e-15 * max(g.max(), 0.0) + 64 * 5e-324
        np.testing.assert_allclose(got, ref, rtol=0, atol=atol)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.4, 1.0, 1.3, 2.75, 7.5, -1.6, -3.25, -18.2])
def test_clamp_form_with_whole_cell_shifts_is_the_corrector(periodic, alpha):
    rng = np.random.default_rng(int(10 * abs(alpha)) + periodic)
    for f in lines(rng, 19):
        got, lost = shifted_update(f, alpha, periodic)
        ref = O.pfc_line(f, alpha, periodic)
        scale = max(f.max(), 1e-300)
        np.testing.assert_allclose(got, ref, rtol=0, atol=4e-15 * scale)
        # what left through the outflow end is the mass the line lost
        assert f.sum() - got.sum() == pytest.approx(lost, abs=1e-13 * scale)

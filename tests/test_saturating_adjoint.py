"""The cotangent formulas of the CUDA adjoint kernels, checked on the CPU.

For a sub-cell shift (|alpha| < 1, line in upwind order) the kernels write
the frozen-branch adjoint of the saturating flux form (phi_j = K0 f_j +
A1 s1_j + A2 s2_j, s = sat(u), u1 = r3 f_j + h_{j+1}, u2 = r3 f_j + h_{j-1},
h = -f / F, F = 2 f_inf) as, with mu_j = l_{j+1} - l_j and m = mu [s == u]:

    lambda_j = l_j + K0 mu_j - 3 c1 m1_j + 3 c2 m2_j + c1 m1_{j-1} - c2 m2_{j+1},
    lambda_F = sum_j mu_j (c2 g2_j - c1 g1_j),  g = s - [s == u] u,
    added as 2 lambda_F at the first maximum of the line, and
    d J / d beta = sum_j mu_j (kf f_j + Fd1 s1_j + Fd2 s2_j),
    kf = 1 + 2 (c1' - c2'), Fd1 = -F c1', Fd2 = F c2'  (c' = dc / dbeta).

This test restates those formulas in numpy (FP64) and compares them with
the oracle's adjoint of its own ratio-form update (Sec. 2.1 with Filbet's
corrector), which was derived separately: the two must agree to rounding
for both directions, both boundary rules and lines whose corrector takes
every arm."""
import numpy as np
import pytest

from oracle import vp_oracle as O


def kernel_formulas(f, lam_out, alpha, periodic, tie_tol=0.0):
    """tie_tol > 0: an argument u within tie_tol of a saturation bound counts
    as interior (the exact-arithmetic rule at a tie)."""
    if alpha < 0:
        li, d = kernel_formulas(f[::-1].copy(), lam_out[::-1].copy(), -alpha, periodic, tie_tol)
        return li[::-1], -d
    b = alpha
    c0, c1, c2 = b, b * (1 - b) * (2 - b) / 6, b * (1 - b) * (1 + b) / 6
    dc1, dc2 = (2 - 6 * b + 3 * b * b) / 6, (1 - 3 * b * b) / 6
    n = f.size
    F = 2.0 * max(f.max(), 0.0)
    ninvF = -1.0 / F if F > 0 else 0.0
    r3 = -3.0 * ninvF
    h = f * ninvF
    if periodic:
        hp, hm, lnext = np.roll(h, -1), np.roll(h, 1), np.roll(lam_out, -1)
    else:
        hp, hm = np.append(h[1:], 0.0), np.insert(h[:-1], 0, 0.0)
        lnext = np.append(lam_out[1:], 0.0)
    u1, u2 = r3 * f + hp, r3 * f + hm
    s1, s2 = np.clip(u1, 0, 1), np.clip(u2, 0, 1)
    I1, I2 = (s1 == u1).astype(float), (s2 == u2).astype(float)
    if tie_tol > 0:
        I1 = np.maximum(I1, (np.abs(u1 - s1) <= tie_tol).astype(float))
        I2 = np.maximum(I2, (np.abs(u2 - s2) <= tie_tol).astype(float))
    mu = lnext - lam_out
    m1, m2 = mu * I1, mu * I2
    K0 = c0 + 2 * (c1 - c2)
    lam = lam_out + K0 * mu - 3 * c1 * m1 + 3 * c2 * m2
    if periodic:
        lam += c1 * np.roll(m1, 1) - c2 * np.roll(m2, -1)
    else:
        lam += c1 * np.insert(m1[:-1], 0, 0.0) - c2 * np.append(m2[1:], 0.0)
    lamF = np.sum(mu * (c2 * (s2 - I2 * u2) - c1 * (s1 - I1 * u1)))
    lam[int(np.argmax(f))] += 2 * lamF
    kf, Fd1, Fd2 = 1 + 2 * (dc1 - dc2), -F * dc1, F * dc2
    return lam, float(np.sum(mu * (kf * f + Fd1 * s1 + Fd2 * s2)))


def lines(rng, n):
    yield rng.random(n) + 0.05
    g = rng.random(n) ** 4
    g[rng.integers(1, n - 1, 3)] = 0.0
    yield g
    p = rng.random(n) * 0.5 + 0.5
    p[4:7] = 0.6                       # a plateau below the maximum
    yield p
    t = np.full(n, 0.01)
    t[n // 3: n // 2] = 1.0
    t[n // 3 + 1] = 0.97               # a top hat with no cell tied at the maximum
    yield t


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.07, 0.31, 0.5, 0.86, -0.2, -0.64])
def test_kernel_cotangent_formulas_are_the_oracles_adjoint(periodic, alpha):
    rng = np.random.default_rng(int(100 * abs(alpha)) + 7 * periodic)
    for f in lines(rng, 17):
        w = rng.normal(size=f.size)
        lam, dbeta = kernel_formulas(f, w, alpha, periodic)
        ref, dref = O.pfc_line_adjoint(f, w, alpha, periodic)
        scale = np.abs(w).max()
        np.testing.assert_allclose(lam, ref, rtol=0, atol=1e-13 * scale)
        assert dbeta == pytest.approx(dref, rel=1e-12, abs=1e-13 * scale * f.max())


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("alpha", [0.31, -0.64])
def test_plateau_at_the_maximum_is_a_tie(periodic, alpha):
    """Cells of a plateau at the line maximum sit exactly on a saturation
    bound (u = 1 in exact arithmetic): the map has a kink there.  The kernel
    formulas classify the rounded u, which may land on either side; taking
    the exact-arithmetic rule at such ties (interior) they give the
    oracle's adjoint, so the tie rule is the only difference."""
    rng = np.random.default_rng(5)
    f = rng.random(17) * 0.9
    f[4:7] = 1.0
    w = rng.normal(size=f.size)
    ref, dref = O.pfc_line_adjoint(f, w, alpha, periodic)
    lam, dbeta = kernel_formulas(f, w, alpha, periodic, tie_tol=8 * np.finfo(float).eps)
    np.testing.assert_allclose(lam, ref, rtol=0, atol=1e-13 * np.abs(w).max())
    assert dbeta == pytest.approx(dref, rel=1e-12, abs=1e-13)

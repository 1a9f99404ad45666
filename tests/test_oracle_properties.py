"""Property-based pins of the oracle's line update (Sec. 2.1) over generated
lines and shifts (hypothesis; skipped where it is not installed):

* periodic lines keep their mass to rounding; outflow lines lose exactly
  what crosses the end, never gain;
* the update is non-negative and never exceeds the line maximum (the
  corrector's positivity and maximum principle);
* scaling the line scales the update (the map is positively homogeneous);
* the CUDA kernels' saturating form of the flux (restated in
  test_saturating_form) gives the same update."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402
from hypothesis.extra import numpy as hnp  # noqa: E402

from oracle import vp_oracle as O  # noqa: E402

from test_saturating_form import saturating_update, shifted_update  # noqa: E402

# subnormal values included: the FP64 kernels sweep a line whose maximum is
# below 2^-968 rescaled by a power of two (restated in saturating_update)
values = st.floats(min_value=0.0, max_value=1.0, allow_nan=False, allow_infinity=False)
lines = hnp.arrays(np.float64, st.integers(3, 24), elements=values)
shifts = st.floats(min_value=-6.0, max_value=6.0, allow_nan=False).filter(lambda a: abs(a) > 1e-6)


@settings(max_examples=300, deadline=None, derandomize=True, database=None)
@given(f=lines, alpha=shifts, periodic=st.booleans())
def test_mass_positivity_and_maximum(f, alpha, periodic):
    out = O.pfc_line(f, alpha, periodic)
    fmax = f.max()
    assert out.min() >= 0.0
    assert out.max() <= fmax * (1 + 1e-12) + 1e-300
    if periodic:
        assert abs(out.sum() - f.sum()) <= 1e-12 * max(f.sum(), 1e-300) * f.size
    else:
        _, lost = shifted_update(f, alpha, periodic)
        assert out.sum() <= f.sum() * (1 + 1e-12) + 1e-300
        assert abs((f.sum() - out.sum()) - lost) <= 1e-12 * max(f.sum(), 1e-300) * f.size


@settings(max_examples=200, deadline=None, derandomize=True, database=None)
@given(f=lines, alpha=shifts, periodic=st.booleans(),
       scale=st.floats(min_value=1e-3, max_value=1e3, allow_nan=False))
def test_positive_homogeneity(f, alpha, periodic, scale):
    a = O.pfc_line(scale * f, alpha, periodic)
    b = scale * O.pfc_line(f, alpha, periodic)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14 * scale * max(f.max(), 1e-300))


@settings(max_examples=400, deadline=None, derandomize=True, database=None)
@given(f=lines, alpha=shifts, periodic=st.booleans())
def test_kernel_formulations_agree_with_the_oracle(f, alpha, periodic):
    ref = O.pfc_line(f, alpha, periodic)
    tol = 4e-15 * max(f.max(), 1e-300)
    np.testing.assert_allclose(shifted_update(f, alpha, periodic)[0], ref, rtol=0, atol=tol)
    if abs(alpha) < 1:
        np.testing.assert_allclose(saturating_update(f, alpha, periodic), ref, rtol=0, atol=tol)

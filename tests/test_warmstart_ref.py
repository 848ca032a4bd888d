"""Pins of the FP64 projection reference (CPU): exact profiles are fixed points,
known shifts are recovered, and the target sum is met."""
import numpy as np
import pytest

from oracle import warmstart_ref as R

W = 4.0


def _layer(nx, ny, yc):
    y = np.arange(ny, dtype=np.float64)[:, None]
    return np.tanh((np.asarray(yc, dtype=np.float64)[None, :] - y) / (np.sqrt(2.0) * W))


def test_contour_heights_of_exact_profile():
    """A tanh profile about heights y_c(x): the sign change is found between the right
    nodes, and linear interpolation is within the profile's curvature error."""
    nx, ny = 16, 64
    yc = 30.3 + 2.0 * np.sin(2 * np.pi * np.arange(nx) / nx)
    got = R.contour_heights(_layer(nx, ny, yc))
    # |phi| <= tanh(0.5 / (sqrt 2 W)) at the bracketing nodes; the interpolation error of a
    # tanh over one cell is below 1e-3 cells for W = 4
    assert np.abs(got - yc).max() < 1e-3


@pytest.mark.parametrize("mode", ["contour", "atanh"])
def test_exact_profile_is_a_fixed_point(mode):
    nx, ny = 12, 48
    # contour heights on half-integers: the two bracketing nodes hold +-phi, so linear
    # interpolation finds the height exactly
    yc = 20.5 + np.round(1.5 * np.cos(2 * np.pi * np.arange(nx) / nx))
    phi = _layer(nx, ny, yc)
    out, s, got = R.project_phi(phi, W, phi.sum(), mode)
    assert abs(s) < 1e-9
    assert np.abs(out - phi).max() < 1e-9
    assert abs(got - phi.sum()) <= 1e-12 * phi.size


def test_known_shift_is_recovered():
    """Target the sum of the profile moved up by 0.75 cells: the contour mode returns
    exactly that profile, with s = 0.75 / (sqrt 2 W)."""
    nx, ny = 10, 40
    yc = np.full(nx, 17.5)
    phi = _layer(nx, ny, yc)
    target = _layer(nx, ny, yc + 0.75).sum()
    out, s, got = R.project_phi(phi, W, target, "contour")
    assert s == pytest.approx(0.75 / (np.sqrt(2.0) * W), abs=1e-10)
    assert np.abs(out - _layer(nx, ny, yc + 0.75)).max() < 1e-9


def test_noisy_prediction_is_rethresholded():
    """A prediction with a wrong bulk value and noise: the output is a clean tanh
    profile (bulk values -> +-1, width W) meeting the target sum."""
    rng = np.random.default_rng(0)
    nx, ny = 32, 64
    yc = 31.0 + np.sin(2 * np.pi * np.arange(nx) / nx)
    clean = _layer(nx, ny, yc)
    pred = 0.9 * clean + 0.01 * rng.standard_normal(clean.shape)
    target = clean.sum()
    out, s, got = R.project_phi(pred, W, target, "contour")
    assert abs(got - target) <= 1e-12 * out.size
    assert out[0].min() > 0.99 and out[-1].max() < -0.99
    assert np.abs(out - clean).max() < 0.05


def test_sum_is_monotone_in_offset():
    a = R.scaled_distance(_layer(8, 32, np.full(8, 15.0)), W, "contour")
    sums = [np.tanh(a + s).sum() for s in np.linspace(-2, 2, 41)]
    assert np.all(np.diff(sums) > 0)

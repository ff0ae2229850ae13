"""The high-contrast workload generator (synth.convdiff, Section 4's 2D
high-contrast experiments): a thresholded, Gaussian-smoothed uniform field.

Pins: the smoothing equals scipy's Gaussian filter with mirrored edges and a
kernel cut at four standard deviations; the field takes only rho and 1/rho,
about half each; rho = 1 reduces to the constant-coefficient matrix; the
matrix is an M-matrix with weakly dominant rows.
"""
import numpy as np
import pytest

from synth.convdiff import config_problem, convdiff, gaussian_smooth, high_contrast_field


def test_smoothing_matches_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    f = np.random.default_rng(1).uniform(size=(37, 29))
    np.testing.assert_allclose(gaussian_smooth(f, 1.0), ndimage.gaussian_filter(f, 1.0, mode="reflect", truncate=4.0),
                               rtol=0, atol=1e-14)
    np.testing.assert_allclose(gaussian_smooth(np.full((9, 7), 0.3)), 0.3, rtol=0, atol=1e-15)


@pytest.mark.parametrize("rho", [10.0, 100.0])
def test_field_values_and_balance(rho):
    a = high_contrast_field(np.random.Generator(np.random.PCG64(6000)), 128, rho)
    assert set(np.unique(a).tolist()) == {rho, 1.0 / rho}
    frac = np.mean(a == rho)
    assert 0.35 < frac < 0.65
    # the pattern does not depend on rho
    b = high_contrast_field(np.random.Generator(np.random.PCG64(6000)), 128, 7.0)
    np.testing.assert_array_equal(a == rho, b == 7.0)


def test_rho_one_is_constant_coefficient():
    p = config_problem("2d_high_contrast", n=20, rho=1.0)
    rp, ci, v = convdiff((20, 20), np.ones(400), np.tile([1.0, 1.0], (400, 1)))
    np.testing.assert_array_equal(p.rowptr, rp)
    np.testing.assert_array_equal(p.colind, ci)
    np.testing.assert_array_equal(p.val, v)


def test_m_matrix_and_contrast():
    p = config_problem("2d_high_contrast", n=40, rho=100.0)
    A = p.to_dense()
    off = A - np.diag(np.diag(A))
    assert (np.diag(A) > 0).all() and (off <= 0).all()
    assert (np.diag(A) + off.sum(axis=1) >= -1e-9 * np.diag(A)).all()
    # the coefficient spans rho^2 = 1e4: so does the diagonal
    d = np.diag(A)
    assert d.max() / d.min() > 1e3

"""Pins of the oracle's anti-aliasing Gaussian (Sec. 5.A):

* the spacing formula sigma = max(r/u - 1, 0)/3 at points where it has
  closed values;
* the whole filter equals scipy.ndimage.gaussian_filter with standard
  deviation sigma/sqrt(2) (the paper's kernel is exp(-x^2/sigma^2)), the same
  radii and constant extension by the fill value;
* sigma = 0 is the identity; a volume equal to the fill value is unchanged;
* an interior impulse spreads into the outer product of the 1-D weights and
  keeps its sum; a linear ramp is unchanged away from the boundary (the kernel
  is symmetric and normalised);
* sampled points equal the whole-volume result.
"""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import ref


def test_sigma_formula_closed_values():
    assert ref.antialias_sigma(3.0, 3.0) == 0.0
    assert ref.antialias_sigma(3.0, 5.0) == 0.0
    assert abs(ref.antialias_sigma(3.0, 1.0) - 2.0 / 3.0) < 1e-15
    assert abs(ref.antialias_sigma(3.0, 0.75) - 1.0) < 1e-15
    assert abs(ref.antialias_sigma(3.0, 0.7) - (3.0 / 0.7 - 1.0) / 3.0) < 1e-15
    assert ref.gauss_radius(0.0) == 0 and ref.gauss_radius(1.0) == 3
    assert ref.gauss_radius(1.0953) == 4


@pytest.mark.parametrize("sigma", [(1.0953, 1.0953, 1.0953), (0.5, 1.7, 0.0), (2.3, 0.0, 0.8)])
@pytest.mark.parametrize("dtype", [np.float32, np.int16])
def test_matches_scipy_gaussian_filter(sigma, dtype):
    rng = np.random.default_rng(1)
    img = (rng.standard_normal((13, 17, 21)) * 300).astype(dtype)
    fill = -1000.0
    out = ref.smooth(img, sigma, fill)
    sd = [s / math.sqrt(2.0) for s in sigma[::-1]]          # z, y, x
    rad = [ref.gauss_radius(s) for s in sigma[::-1]]
    exp = ndi.gaussian_filter(img.astype(np.float64), sigma=sd, mode="constant", cval=fill,
                              radius=rad, truncate=100.0)
    assert np.max(np.abs(out - exp)) < 1e-9 * np.max(np.abs(exp))


def test_identity_and_constant():
    rng = np.random.default_rng(2)
    img = (rng.standard_normal((6, 7, 8)) * 100).astype(np.float32)
    assert np.array_equal(ref.smooth(img, (0.0, 0.0, 0.0), -1000.0), img.astype(np.float64))
    const = np.full((9, 8, 7), -1000.0, np.float32)
    assert np.max(np.abs(ref.smooth(const, (1.3, 0.7, 2.1), -1000.0) + 1000.0)) < 1e-10


def test_impulse_is_outer_product_of_weights_and_keeps_its_sum():
    sigma = (1.2, 0.6, 0.9)
    img = np.zeros((15, 15, 15), np.float32)
    img[7, 7, 7] = 1.0
    out = ref.smooth(img, sigma, 0.0)
    wx, wy, wz = (ref.gauss_weights(s) for s in sigma)
    assert abs(out.sum() - 1.0) < 1e-14
    Rx, Ry, Rz = len(wx) // 2, len(wy) // 2, len(wz) // 2
    exp = np.zeros_like(out)
    exp[7 - Rz:7 + Rz + 1, 7 - Ry:7 + Ry + 1, 7 - Rx:7 + Rx + 1] = (
        wz[:, None, None] * wy[None, :, None] * wx[None, None, :])
    assert np.max(np.abs(out - exp)) < 1e-16
    # weights: symmetric, normalised, ratio exp(-1/sigma^2) between offsets 0 and 1
    assert abs(wx.sum() - 1.0) < 1e-15 and np.allclose(wx, wx[::-1], rtol=0, atol=0)
    assert abs(wx[Rx + 1] / wx[Rx] - math.exp(-1.0 / 1.2 ** 2)) < 1e-15


def test_linear_ramp_is_unchanged_in_the_interior():
    z, y, x = np.meshgrid(np.arange(20), np.arange(18), np.arange(22), indexing="ij")
    img = (3.0 * x - 2.0 * y + 0.5 * z + 7.0).astype(np.float32)
    sigma = (1.0953, 0.8, 1.4)
    out = ref.smooth(img, sigma, -1000.0)
    R = [ref.gauss_radius(s) for s in sigma]
    inner = (slice(R[2], 20 - R[2]), slice(R[1], 18 - R[1]), slice(R[0], 22 - R[0]))
    assert np.max(np.abs(out[inner] - img[inner])) < 1e-11


def test_points_equal_volume():
    rng = np.random.default_rng(3)
    img = rng.integers(-1024, 3071, (9, 10, 11)).astype(np.int16)
    sigma = (0.9, 1.1, 0.4)
    full = ref.smooth(img, sigma, -1000.0).reshape(-1)
    q = rng.integers(0, img.size, 50)
    assert np.array_equal(ref.smooth_points(img, sigma, -1000.0, q), full[q])

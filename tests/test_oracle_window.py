"""Pins of the oracle's occlusion and window/level steps (Sec. 4).

* Occlusion sets exactly the output slices z0 <= k <= z0 + dz to 0 (their
  number is a closed form) and leaves every other voxel unchanged; under the
  identity warp the untouched slices equal the input.
* Window/level equals numpy.clip of SciPy's affine_transform mapped through
  (I - lo)/(hi - lo); with noise every value lies in [0, 1].
* The adjoint of an occluded warp is the transpose of the operator whose
  occluded rows are zero (brute force on 8^3).
* The parameter draw gives every output slice the same chance of being
  occluded (the property Sec. 4 asks of the prism's start and height).
"""
import math

import numpy as np
import scipy.ndimage as ndi
import torch

from oracle import ref
from synth.params import AffineSpec, random_affine, random_window_occlusion
from synth.phantom import make_phantom
from synth.workloads import VolumeCase


def case(img, T, out_shape, **kw):
    base = dict(photo_a=np.float32(1.0), photo_b=np.float32(0.0), sigma=np.float32(0.0),
                fill_image=np.float32(-1000.0))
    base.update(kw)
    return VolumeCase(image=torch.as_tensor(img), label=None, out_shape=tuple(out_shape),
                      T=np.asarray(T, np.float32), **base)


def ident():
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = np.eye(3)
    return T


def test_occlusion_zeroes_exactly_the_slab():
    img, _ = make_phantom((16, 14, 40), seed=2)
    img = img.numpy()
    for z0, dz in [(3.0, 5.5), (-4.2, 6.0), (10.5, 0.0), (38.0, 10.0), (12.0, 0.49)]:
        v = case(img, ident(), (16, 14, 40), flags=2, occ_z0=np.float32(z0),
                 occ_dz=np.float32(dz))
        out, _, _, _ = ref.warp_fwd(v, 0)
        zero = np.all(out == 0.0, axis=(1, 2))
        lo, hi = max(0, math.ceil(z0)), min(39, math.floor(z0 + dz))
        expected = np.zeros(40, bool)
        if hi >= lo:
            expected[lo:hi + 1] = True
        assert np.array_equal(zero, expected), (z0, dz)
        assert np.array_equal(out[~expected], img[~expected].astype(np.float64))


def test_occlusion_skips_noise_and_window():
    img, _ = make_phantom((12, 10, 20), seed=3)
    v = case(img.numpy(), ident(), (12, 10, 20), flags=3, occ_z0=np.float32(5.0),
             occ_dz=np.float32(3.0), sigma=np.float32(0.3), photo_a=np.float32(1e-3),
             photo_b=np.float32(0.4))
    out, _, _, _ = ref.warp_fwd(v, 11)
    assert np.all(out[5:9] == 0.0)
    assert np.all((out >= 0.0) & (out <= 1.0))


def _scipy(img, T, out_shape, fill):
    M = np.asarray(T, np.float64)[::-1, :3][:, ::-1]
    off = np.asarray(T, np.float64)[::-1, 3]
    onx, ony, onz = out_shape
    return ndi.affine_transform(img.astype(np.float64), M, offset=off,
                                output_shape=(onz, ony, onx), order=1, mode="grid-constant",
                                cval=fill, prefilter=False)


def test_window_level_matches_clipped_scipy():
    rng = np.random.default_rng(4)
    img, _ = make_phantom((30, 26, 22), seed=4)
    img = img.numpy()
    T, _ = random_affine(rng, (30, 26, 22), (24, 20, 18), AffineSpec())
    for lo, hi in [(-150.0, 230.0), (-1000.0, 1500.0), (20.0, 60.0)]:
        a = np.float32(1.0 / (hi - lo))
        b = np.float32(-lo / (hi - lo))
        v = case(img, T, (24, 20, 18), flags=1, photo_a=a, photo_b=b)
        out, _, _, _ = ref.warp_fwd(v, 0)
        exp = np.clip(np.float64(a) * _scipy(img, T, (24, 20, 18), -1000.0) + np.float64(b),
                      0.0, 1.0)
        assert np.max(np.abs(out - exp)) < 1e-12
        assert (out == 0.0).any() or (out == 1.0).any() or lo == -1000.0


def test_window_with_noise_stays_in_unit_interval():
    img, _ = make_phantom((20, 20, 16), seed=5)
    rng = np.random.default_rng(5)
    a, b, s, z0, dz = random_window_occlusion(rng, 16)
    v = case(img.numpy(), ident(), (20, 20, 16), flags=1, photo_a=a, photo_b=b, sigma=s)
    out, _, _, _ = ref.warp_fwd(v, 3)
    assert np.all((out >= 0.0) & (out <= 1.0))
    assert 0.0 < np.mean((out > 0.0) & (out < 1.0)) < 1.0


def test_adjoint_of_occluded_warp_is_masked_transpose():
    n = 8
    rng = np.random.default_rng(6)
    T, _ = random_affine(rng, (n, n, n), (n, n, n), AffineSpec(max_rot_deg=30, max_shift_vox=1))
    occ = dict(flags=2, occ_z0=np.float32(2.3), occ_dz=np.float32(2.0))
    cols = []
    for m in range(n ** 3):
        e = np.zeros(n ** 3, np.float32)
        e[m] = 1.0
        o, _, _, _ = ref.warp_fwd(case(e.reshape(n, n, n), T, (n, n, n), fill_image=np.float32(0),
                                       **occ), 0)
        cols.append(o.reshape(-1))
    M = np.stack(cols, 1)
    masked = np.zeros((n, n, n), bool)
    masked[3:5] = True
    assert np.all(M[masked.reshape(-1)] == 0.0)
    g = rng.standard_normal(n ** 3).astype(np.float32)
    gi, _, _ = ref.warp_bwd(case(np.zeros((n, n, n), np.float32), T, (n, n, n), **occ),
                            g.reshape(n, n, n))
    assert np.max(np.abs(gi.reshape(-1) - M.T @ g.astype(np.float64))) < 1e-12


def test_occlusion_draw_covers_every_slice_equally():
    rng = np.random.default_rng(7)
    onz, draws = 40, 20000
    hits = np.zeros(onz)
    for _ in range(draws):
        _, _, _, z0, dz = random_window_occlusion(rng, onz)
        k = np.arange(onz)
        hits += (k >= z0) & (k <= z0 + dz)
    p = hits / draws
    # Every slice has the same probability; allow 6 binomial standard errors.
    se = np.sqrt(p.mean() * (1 - p.mean()) / draws)
    assert np.max(np.abs(p - p.mean())) < 6 * se + 1e-3

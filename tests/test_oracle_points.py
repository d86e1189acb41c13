"""Pins of the oracle's point-list entry points against its whole-grid ones.

The full-size GPU parity checks evaluate the oracle only at sampled output
voxels, through ``warp_fwd_points`` and ``noise``, which decode a flattened
output index q = (k * ony + j) * onx + i themselves.  Here both are pinned to
the whole-grid routine, whose loops run over (k, j, i) explicitly:

* ``warp_fwd_points(v, seed, q)`` equals ``warp_fwd(v, seed)`` at q, for the
  image value, the label and the tie flag, on output grids with three
  different extents (a swapped or mis-strided decoding reads another voxel);
* ``noise(seed, id, onx, ony, q)`` equals the image of a whole-grid warp with
  intensity slope 0, offset 0 and noise sigma 1, whose value at each voxel is
  exactly that voxel's normal (0 * v + 0 + 1 * n = n in IEEE arithmetic);
* the sampled indices include the grid's first and last voxel and the ends
  of rows and planes, where a wrong modulus or stride shows first.
"""
import numpy as np
import pytest
import torch

from oracle import ref
from synth.params import AffineSpec, random_affine
from synth.phantom import make_phantom
from synth.workloads import VolumeCase


def _case(in_xyz, out_xyz, seed, T=None, a=1.0, b=0.0, sigma=0.0, noise_id=3):
    img, lab = make_phantom(in_xyz, seed=seed)
    if T is None:
        T, _ = random_affine(np.random.default_rng(seed), in_xyz, out_xyz,
                             AffineSpec(max_rot_deg=25.0, max_shear=0.1))
    return VolumeCase(image=img, label=lab, out_shape=tuple(out_xyz),
                      T=np.asarray(T, np.float32), photo_a=np.float32(a),
                      photo_b=np.float32(b), sigma=np.float32(sigma), noise_id=noise_id)


def _indices(out_xyz, rng, n=4000):
    onx, ony, onz = out_xyz
    nvox = onx * ony * onz
    edges = [0, onx - 1, onx, onx * ony - 1, onx * ony, nvox - onx, nvox - 1,
             (onz // 2) * onx * ony + (ony // 2) * onx + onx // 2]
    return np.concatenate([np.asarray(edges, np.int64), rng.integers(0, nvox, n)])


@pytest.mark.parametrize("out_xyz", [(23, 17, 11), (9, 31, 14), (40, 6, 19)])
def test_points_equal_whole_grid(out_xyz):
    rng = np.random.default_rng(sum(out_xyz))
    v = _case((21, 18, 13), out_xyz, seed=out_xyz[0], a=1.07, b=-12.5, sigma=35.0)
    full, lab, tie, _ = ref.warp_fwd(v, seed=91)
    q = _indices(out_xyz, rng)
    vals, labs, ties = ref.warp_fwd_points(v, 91, q)
    assert np.array_equal(vals, full.reshape(-1)[q])
    assert np.array_equal(labs, lab.reshape(-1)[q])
    assert np.array_equal(ties, tie.reshape(-1)[q])


def test_points_equal_whole_grid_on_ties():
    # s_x = i / 2 + 0.25 j: every other column sits on a rounding tie in x, so the
    # tie flags are a dense, index-dependent pattern the decoding must follow.
    out_xyz = (26, 15, 7)
    T = np.zeros((3, 4), np.float32)
    T[0, 0], T[0, 1] = 0.5, 0.25
    T[1, 1], T[2, 2] = 1.0, 1.0
    T[:, 3] = (1.0, 2.0, 3.0)
    v = _case((24, 20, 12), out_xyz, seed=4, T=T)
    full, lab, tie, n_ties = ref.warp_fwd(v, seed=0)
    assert 0 < n_ties < tie.size
    q = _indices(out_xyz, np.random.default_rng(5), n=2000)
    vals, labs, ties = ref.warp_fwd_points(v, 0, q)
    assert np.array_equal(ties, tie.reshape(-1)[q])
    assert np.array_equal(labs, lab.reshape(-1)[q])
    assert np.array_equal(vals, full.reshape(-1)[q])


@pytest.mark.parametrize("out_xyz", [(23, 17, 11), (7, 29, 13)])
def test_noise_points_equal_whole_grid_noise(out_xyz):
    onx, ony, _ = out_xyz
    v = _case((12, 10, 9), out_xyz, seed=8, a=0.0, b=0.0, sigma=1.0, noise_id=5)
    full, _, _, _ = ref.warp_fwd(v, seed=1234, want_label=False)
    q = _indices(out_xyz, np.random.default_rng(onx))
    z = ref.noise(1234, 5, onx, ony, q)
    assert np.array_equal(z, full.reshape(-1)[q])
    # another noise_id draws other numbers at the same voxels
    assert not np.array_equal(ref.noise(1234, 6, onx, ony, q), z)

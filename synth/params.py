"""Seeded random augmentation parameters (drawn on the host, passed as inputs).

Affine convention: a 3x4 float32 matrix ``T`` in *voxel-index* units maps an
output index ``o = (i, j, k)`` (x, y, z) to an input coordinate
``s = A o + b`` with ``A = T[:, :3]`` and ``b = T[:, 3]`` (Sec. 4, the
coordinate map x' = Ax + b).

Sampling follows Sec. 4: ``A`` composes rotation, scaling and (optionally)
shear and per-axis reflection drawn from user ranges; a displacement ``d`` is
drawn and ``b = c_in + d - A c_out`` so that the output centre lands on the
input centre displaced by ``d`` (the paper's ``Ac + b = c + d`` with one
centre per grid when input and output sizes differ).  Centres are at
``(N - 1) / 2`` because voxel centres sit at integer indices.

Composition order (the paper leaves it open):
``A = Rz(gz) Ry(gy) Rx(gx) Sh diag(refl * s) diag(extra)``, where ``extra`` is
an optional fixed resampling factor (e.g. 3 mm / 0.7 mm for the
full-resolution workload).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class AffineSpec:
    max_rot_deg: float = 15.0
    scale_range: tuple = (0.9, 1.1)
    max_shift_vox: float = 10.0
    max_shear: float = 0.0
    reflect_prob: tuple = (0.0, 0.0, 0.0)
    extra_scale: tuple = (1.0, 1.0, 1.0)


def _rot(axis: int, ang: float) -> np.ndarray:
    c, s = np.cos(ang), np.sin(ang)
    m = np.eye(3)
    a, b = [(1, 2), (0, 2), (0, 1)][axis]
    m[a, a], m[a, b], m[b, a], m[b, b] = c, -s, s, c
    return m


def random_affine(rng: np.random.Generator, in_shape_xyz, out_shape_xyz,
                  spec: AffineSpec = AffineSpec()):
    """Draw one affine.  Returns ``(T, d)``: float32 ``[3, 4]`` and float64 ``d``."""
    rad = np.deg2rad(spec.max_rot_deg)
    gx, gy, gz = rng.uniform(-rad, rad, 3)
    s = rng.uniform(spec.scale_range[0], spec.scale_range[1], 3)
    refl = np.where(rng.uniform(0.0, 1.0, 3) < np.asarray(spec.reflect_prob), -1.0, 1.0)
    sh = np.eye(3)
    if spec.max_shear > 0.0:
        sh[0, 1], sh[0, 2], sh[1, 2] = rng.uniform(-spec.max_shear, spec.max_shear, 3)
    a = _rot(2, gz) @ _rot(1, gy) @ _rot(0, gx) @ sh @ np.diag(refl * s) @ np.diag(
        np.asarray(spec.extra_scale, dtype=np.float64))
    d = rng.uniform(-spec.max_shift_vox, spec.max_shift_vox, 3)
    c_in = (np.asarray(in_shape_xyz, dtype=np.float64) - 1.0) / 2.0
    c_out = (np.asarray(out_shape_xyz, dtype=np.float64) - 1.0) / 2.0
    b = c_in + d - a @ c_out
    t = np.concatenate([a, b[:, None]], axis=1).astype(np.float32)
    return t, d


def random_photometric(rng: np.random.Generator, a_range=(0.9, 1.1),
                       b_range=(-50.0, 50.0), sigma_range=(0.0, 50.0)):
    """Intensity affine ``a*v + b`` and noise standard deviation, float32."""
    a = np.float32(rng.uniform(*a_range))
    b = np.float32(rng.uniform(*b_range))
    sigma = np.float32(rng.uniform(*sigma_range))
    return a, b, sigma


def random_window_occlusion(rng: np.random.Generator, onz: int, lo_range=(-1000.0, -150.0),
                            hi_range=(230.0, 1500.0), sigma_range=(0.0, 50.0),
                            max_occ_frac=0.3):
    """Window/level and occlusion parameters of Sec. 4, as descriptor fields.

    Window [lo, hi] drawn from the given HU ranges; noise sigma in HU.  The
    window map clamp((I + n - lo)/(hi - lo), 0, 1) equals the intensity affine
    a = 1/(hi - lo), b = -lo/(hi - lo) with noise sigma * a, then a clamp.
    Occlusion: a z-slab of the output of height d ~ U[0, d_max] starting at
    z ~ U[-d_max, onz - 1], d_max = max_occ_frac * onz, so every slice is
    equally likely to be covered.  Returns (a, b, sigma, occ_z0, occ_dz), float32.
    """
    lo = rng.uniform(*lo_range)
    hi = rng.uniform(*hi_range)
    a = 1.0 / (hi - lo)
    b = -lo / (hi - lo)
    sigma = rng.uniform(*sigma_range) * a
    dmax = max_occ_frac * onz
    dz = rng.uniform(0.0, dmax)
    z0 = rng.uniform(-dmax, onz - 1)
    return (np.float32(a), np.float32(b), np.float32(sigma), np.float32(z0), np.float32(dz))

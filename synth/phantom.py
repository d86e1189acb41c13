"""CT-like phantom volumes with matching label maps (seeded).

Layout: arrays are ``[nz][ny][nx]`` with x fastest (C order), the same layout
the augmentation library reads.  Shapes are given as ``(nx, ny, nz)``.

Recipe (stands in for the paper's CT scans, Sec. 6.A; intensities in HU):

* background (air) at exactly -1000 HU, label 0;
* one ellipsoidal "body" at 40 HU, label 0, with i.i.d. Gaussian texture of
  standard deviation 20 HU added to every voxel inside the body;
* 3-6 ellipsoid "organs" inside the body at U[30, 80] HU, labels 1 + (i mod 4);
* 2-4 ellipsoid "bone" blobs inside the body at 700 HU, label 5.

Later shapes overwrite earlier ones.  Geometry is drawn relative to the grid
extent, so the same recipe at a finer grid (the 0.7 mm-like full-resolution
scans) gives the same anatomy with more voxels.  ``dtype="int16"`` rounds to
integers and clamps to the 12-bit CT range [-1024, 3071].

Shape parameters come from ``numpy.random.default_rng(seed)``; the texture
comes from a ``torch.Generator`` seeded with the same seed on the requested
device, so generation of the large batched workloads can run on the GPU.
The texture is therefore device dependent: a test that compares two
implementations generates once and hands both the same array.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

AIR_HU = -1000.0
BODY_HU = 40.0
TEXTURE_SIGMA_HU = 20.0
BONE_HU = 700.0
N_CLASSES = 6


@dataclass
class PhantomSpec:
    """Ellipsoids of one phantom: (centre xyz, semi-axes xyz, HU, label)."""

    body: tuple
    organs: list
    bones: list


def _draw_spec(rng: np.random.Generator, shape_xyz) -> PhantomSpec:
    n = np.asarray(shape_xyz, dtype=np.float64)
    centre = (n - 1.0) / 2.0
    body_c = centre + rng.uniform(-0.03, 0.03, 3) * n
    body_r = np.array(
        [rng.uniform(0.40, 0.47), rng.uniform(0.30, 0.40), rng.uniform(0.55, 0.75)]
    ) * n
    organs = []
    for i in range(int(rng.integers(3, 7))):
        c = body_c + rng.uniform(-0.5, 0.5, 3) * body_r
        r = rng.uniform(0.06, 0.18, 3) * n
        organs.append((c, r, float(rng.uniform(30.0, 80.0)), 1 + (i % 4)))
    bones = []
    for _ in range(int(rng.integers(2, 5))):
        c = body_c + rng.uniform(-0.7, 0.7, 3) * body_r
        r = rng.uniform(0.03, 0.08, 3) * n
        bones.append((c, r, BONE_HU, 5))
    return PhantomSpec(body=(body_c, body_r, BODY_HU, 0), organs=organs, bones=bones)


def _inside(c, r, shape_xyz, device):
    nx, ny, nz = shape_xyz
    x = (torch.arange(nx, device=device, dtype=torch.float32) - float(c[0])) / float(r[0])
    y = (torch.arange(ny, device=device, dtype=torch.float32) - float(c[1])) / float(r[1])
    z = (torch.arange(nz, device=device, dtype=torch.float32) - float(c[2])) / float(r[2])
    return (x * x)[None, None, :] + (y * y)[None, :, None] + (z * z)[:, None, None] <= 1.0


def make_phantom(shape_xyz, seed: int, dtype: str = "float32", device="cpu"):
    """Return ``(image, label)`` torch tensors of shape ``[nz, ny, nx]``.

    ``image`` is float32 (or int16 when ``dtype == "int16"``); ``label`` is
    uint8 with classes 0..5.
    """
    shape_xyz = tuple(int(v) for v in shape_xyz)
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    spec = _draw_spec(rng, shape_xyz)
    dev = torch.device(device)
    img = torch.full((nz, ny, nx), AIR_HU, dtype=torch.float32, device=dev)
    lab = torch.zeros((nz, ny, nx), dtype=torch.uint8, device=dev)
    body = _inside(spec.body[0], spec.body[1], shape_xyz, dev)
    img[body] = BODY_HU
    for c, r, hu, label in spec.organs + spec.bones:
        m = _inside(c, r, shape_xyz, dev) & body
        img[m] = hu
        lab[m] = label
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    tex = torch.randn((nz, ny, nx), generator=gen, device=dev, dtype=torch.float32)
    img = torch.where(body, img + TEXTURE_SIGMA_HU * tex, img)
    if dtype == "int16":
        img = torch.clamp(torch.round(img), -1024.0, 3071.0).to(torch.int16)
    elif dtype != "float32":
        raise ValueError(f"unsupported phantom dtype {dtype!r}")
    return img.contiguous(), lab.contiguous()

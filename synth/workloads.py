"""The five synthetic workloads and small parity cases (all seeded).

Each builder returns a :class:`Workload`: a list of :class:`VolumeCase`
records (input image/label, output grid, affine, photometric and noise
parameters) plus the per-workload extras (probability maps ``p`` for the IOU
loss, upstream gradients ``g`` for the adjoint).  Arrays are torch tensors on
the requested device; parameters are numpy float32.

Workloads (sizes x*y*z):

0. one float32 128*128*64 phantom -> 128*128*64 crop (trilinear image,
   nearest label, intensity affine, noise);
1. 64 float32 phantoms, in-plane U{96..160}, slices U{80..240}, each warped
   into a 120*120*160 crop;
2. 8 float32 128^3 phantoms, identity photometric, no noise, with a seeded
   N(0, 1) upstream gradient on the output grid;
3. 8 uint8 label volumes 120*120*160 warped nearest-neighbour and fed to the
   IOU loss with p = softmax over 6 channels of N(0, 2^2) logits;
4. 16 int16 phantoms 512*512*U{300..600} resampled with a 3 mm / 0.7 mm
   downscale into 128*128*160 float32 crops, with p and g as above.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from .params import AffineSpec, random_affine, random_photometric
from .phantom import N_CLASSES, make_phantom

FILL_HU = -1000.0


@dataclass
class VolumeCase:
    image: torch.Tensor                 # [nz, ny, nx] float32 or int16
    label: Optional[torch.Tensor]       # [nz, ny, nx] uint8 or None
    out_shape: tuple                    # (onx, ony, onz)
    T: np.ndarray                       # float32 [3, 4]
    photo_a: np.float32 = np.float32(1.0)
    photo_b: np.float32 = np.float32(0.0)
    sigma: np.float32 = np.float32(0.0)
    fill_image: np.float32 = np.float32(FILL_HU)
    fill_label: int = 0
    noise_id: int = 0
    flags: int = 0            # 1: window/level clamp to [0, 1]; 2: occlusion
    occ_z0: np.float32 = np.float32(0.0)
    occ_dz: np.float32 = np.float32(0.0)

    @property
    def in_shape(self):
        nz, ny, nx = self.image.shape
        return (nx, ny, nz)

    @property
    def n_out(self) -> int:
        return int(np.prod(self.out_shape))


@dataclass
class Workload:
    name: str
    vols: list
    seed: int
    n_classes: int = N_CLASSES
    p: Optional[torch.Tensor] = None    # packed [sum_b C * nvox_b] float32
    g: Optional[list] = None            # per volume, output shape, float32
    extra: dict = field(default_factory=dict)

    @property
    def n_out(self) -> int:
        return sum(v.n_out for v in self.vols)


def _gen(device, seed):
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def softmax_probs(shape_cxyz_list, seed, device, logit_std=2.0, n_classes=N_CLASSES):
    """Packed class probabilities: per volume ``[C][onz][ony][onx]``
    = softmax over C of N(0, logit_std^2) logits, volumes concatenated."""
    gen = _gen(device, seed)
    parts = []
    for (onx, ony, onz) in shape_cxyz_list:
        z = torch.randn((n_classes, onz, ony, onx), generator=gen,
                        device=torch.device(device), dtype=torch.float32) * logit_std
        parts.append(torch.softmax(z, dim=0).reshape(-1))
    return torch.cat(parts)


def class_logits(shape_cxyz_list, seed, device, logit_std=2.0, n_classes=N_CLASSES):
    """Packed class scores: per volume ``[C][onz][ony][onx]`` of
    N(0, logit_std^2), volumes concatenated (the inputs of the fused softmax)."""
    gen = _gen(device, seed)
    parts = [torch.randn((n_classes, onz, ony, onx), generator=gen, device=torch.device(device),
                         dtype=torch.float32).reshape(-1) * logit_std
             for (onx, ony, onz) in shape_cxyz_list]
    return torch.cat(parts)


def upstream_grads(shape_list, seed, device):
    gen = _gen(device, seed)
    return [torch.randn((onz, ony, onx), generator=gen, device=torch.device(device),
                        dtype=torch.float32) for (onx, ony, onz) in shape_list]


def make_case(in_shape_xyz, out_shape_xyz, seed, *, dtype="float32", device="cpu",
              spec: AffineSpec = AffineSpec(), photometric=True, with_label=True,
              noise_id=0) -> VolumeCase:
    img, lab = make_phantom(in_shape_xyz, seed, dtype=dtype, device=device)
    rng = np.random.default_rng([int(seed), 7])
    t, _ = random_affine(rng, in_shape_xyz, out_shape_xyz, spec)
    if photometric:
        a, b, s = random_photometric(rng)
    else:
        a, b, s = np.float32(1.0), np.float32(0.0), np.float32(0.0)
    return VolumeCase(image=img, label=lab if with_label else None,
                      out_shape=tuple(int(v) for v in out_shape_xyz), T=t,
                      photo_a=a, photo_b=b, sigma=s, noise_id=noise_id)


def config0(device="cpu") -> Workload:
    v = make_case((128, 128, 64), (128, 128, 64), seed=0, device=device)
    return Workload("plain 128x128x64", [v], seed=0)


def config1(device="cpu", n_vols: int = 64, first: int = 0) -> Workload:
    rng = np.random.default_rng(11)
    nxy = rng.integers(96, 161, 64)
    nz = rng.integers(80, 241, 64)
    vols = []
    for b in range(first, first + n_vols):
        vols.append(make_case((int(nxy[b]), int(nxy[b]), int(nz[b])), (120, 120, 160),
                              seed=1 + b, device=device, noise_id=b))
    return Workload("batched 64 uneven -> 120x120x160", vols, seed=1)


def config2(device="cpu", n_vols: int = 8) -> Workload:
    vols = [make_case((128, 128, 128), (128, 128, 128), seed=200 + b, device=device,
                      photometric=False, noise_id=b) for b in range(n_vols)]
    g = upstream_grads([v.out_shape for v in vols], seed=2, device=device)
    return Workload("differentiable 8x128^3", vols, seed=2, g=g)


def config3(device="cpu", n_vols: int = 8) -> Workload:
    vols = [make_case((120, 120, 160), (120, 120, 160), seed=300 + b, device=device,
                      noise_id=b) for b in range(n_vols)]
    p = softmax_probs([v.out_shape for v in vols], seed=3, device=device)
    return Workload("fused warp+IOU 8x120x120x160", vols, seed=3, p=p)


def config4(device="cpu", n_vols: int = 16, first: int = 0) -> Workload:
    rng = np.random.default_rng(44)
    nz = rng.integers(300, 601, 16)
    down = 3.0 / 0.7
    spec = AffineSpec(max_shift_vox=10.0 * down, extra_scale=(down, down, down))
    vols = [make_case((512, 512, int(nz[b])), (128, 128, 160), seed=400 + b, dtype="int16",
                      device=device, spec=spec, noise_id=b)
            for b in range(first, first + n_vols)]
    p = softmax_probs([v.out_shape for v in vols], seed=4, device=device)
    g = upstream_grads([v.out_shape for v in vols], seed=5, device=device)
    return Workload("training step 16x512^2x300-600 int16 -> 128x128x160", vols, seed=4,
                    p=p, g=g)


BUILDERS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}

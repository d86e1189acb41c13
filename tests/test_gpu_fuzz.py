"""Seeded randomized parity of the CUDA path against the FP64 oracle, mixing
in one batch everything the hand-picked cases cover separately: random input
and output shapes from 1 to 40 voxels per axis, rotations up to 60 degrees,
scales 0.5-2, shear, reflections, both input types, photometric draws with
noise, and window/level and occlusion flags.  The forward (image + label) and,
for the float32 unwindowed volumes, the adjoint (input and affine) and the
Dice loss on class scores are checked voxel by voxel."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth.params import AffineSpec, random_affine, random_photometric, random_window_occlusion
from synth.phantom import make_phantom
from synth.workloads import VolumeCase, class_logits, upstream_grads

import _gpu as G

pytestmark = pytest.mark.gpu

SPEC = AffineSpec(max_rot_deg=60.0, scale_range=(0.5, 2.0), max_shift_vox=6.0, max_shear=0.3,
                  reflect_prob=(0.3, 0.3, 0.3))


def _cases(n, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for b in range(n):
        si = tuple(int(v) for v in rng.integers(1, 41, 3))
        so = tuple(int(v) for v in rng.integers(1, 41, 3))
        dtype = "int16" if rng.random() < 0.3 else "float32"
        img, lab = make_phantom(si, seed=seed * 1000 + b, dtype=dtype)
        T, _ = random_affine(rng, si, so, SPEC)
        a, bb, s = random_photometric(rng)
        v = VolumeCase(image=img, label=lab, out_shape=so, T=T, photo_a=a, photo_b=bb, sigma=s,
                       noise_id=int(rng.integers(0, 2 ** 31)))
        r = rng.random()
        if r < 0.25:          # window/level (+ occlusion half of the time)
            wa, wb, ws_, z0, dz = random_window_occlusion(rng, so[2])
            v.photo_a, v.photo_b, v.sigma = wa, wb, ws_
            v.flags = 1 | (2 if rng.random() < 0.5 else 0)
            v.occ_z0, v.occ_dz = z0, dz
        elif r < 0.45:        # occlusion only
            _, _, _, z0, dz = random_window_occlusion(rng, so[2])
            v.flags, v.occ_z0, v.occ_dz = 2, z0, dz
        cases.append(v)
    return G.to_device(cases)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_batches_forward(seed):
    cases = _cases(40, seed)
    gi, gl = G.run_fwd(cases, seed=seed + 100)
    for b, v in enumerate(cases):
        img, lab, tie, _ = ref.warp_fwd(v, seed + 100)
        tol = G.IMG_TOL * (float(v.photo_a) if v.flags & 1 else 1.0)
        G.check_image(gi[b], img, f"seed {seed} vol {b}", tol=max(tol, 1e-6))
        G.check_labels(gl[b], lab, tie, f"seed {seed} vol {b}")


@pytest.mark.parametrize("seed", [4, 5])
def test_random_batches_adjoint_and_loss(seed):
    from test_gpu_bwd import run_bwd
    from test_gpu_loss_variants import check_loss, run_loss
    cases = [v for v in _cases(40, seed)
             if v.image.dtype == torch.float32 and not (v.flags & 1)]
    grads = upstream_grads([v.out_shape for v in cases], seed=seed, device="cuda")
    gin, gaff = run_bwd(cases, grads)
    floored = 0
    for b, v in enumerate(cases):
        ri, rt, _ = ref.warp_bwd(v, grads[b])
        G.check_grad(gin[b], ri, f"grad_in {b}")
        floor = 1e-7 * G.summand_scale(v, grads[b].cpu().numpy())
        floored += G.check_grad_affine(gaff[b], rt, f"grad_T {b}", floor=floor)
    print(f"grad_T: {floored} of {len(cases)} volumes had a gradient cancelled below the "
          "float32 rounding scale of its terms and used that floor")
    x = class_logits([v.out_shape for v in cases], seed=seed, device="cuda")
    loss, gx = run_loss(cases, x, 6, 1, 2.0, True)
    rl, rg, _ = ref.warp_loss(cases, x, 6, 1, 2.0, True)
    check_loss(loss, rl)
    G.check_grad(gx, rg, "Dice^2 on scores")

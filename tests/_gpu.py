"""Helpers of the GPU parity tests: run the CUDA path through the C ABI on
synthetic cases and compare with the FP64 oracle at the stated tolerances.

Tolerances of the parity checks:
* image: |gpu - oracle| <= 2e-3 HU absolute;
* labels: bit-exact except voxels whose FP64 source coordinate lies within
  1e-5 of a rounding tie (counted and reported);
* gradients: per element |d| <= 1e-4 (|ref| + rms(ref)); affine gradient
  ||d||_inf <= 1e-4 ||ref||_inf per volume.
"""
from __future__ import annotations

import numpy as np
import torch

IMG_TOL = 2e-3
GRAD_RTOL = 1e-4


def aw():
    from paper_1811_11226_b300 import augwarp
    return augwarp


def to_device(cases, device="cuda"):
    for v in cases:
        v.image = v.image.to(device).contiguous()
        if v.label is not None:
            v.label = v.label.to(device).contiguous()
    return cases


def batch_for(cases, with_image=True, with_label=True):
    A = aw()
    outs_i, outs_l = [], []
    for v in cases:
        onx, ony, onz = v.out_shape
        outs_i.append(torch.full((onz, ony, onx), np.nan, dtype=torch.float32, device="cuda")
                      if with_image else None)
        outs_l.append(torch.full((onz, ony, onx), 77, dtype=torch.uint8, device="cuda")
                      if (with_label and v.label is not None) else None)
    batch = A.VolumeBatch([v.image for v in cases], np.stack([v.T for v in cases]),
                          [v.out_shape for v in cases], labels=[v.label for v in cases],
                          out_images=outs_i, out_labels=outs_l,
                          photo_a=[v.photo_a for v in cases], photo_b=[v.photo_b for v in cases],
                          noise_sigma=[v.sigma for v in cases],
                          fill_image=[v.fill_image for v in cases],
                          fill_label=[v.fill_label for v in cases],
                          noise_ids=[v.noise_id for v in cases],
                          flags=[getattr(v, "flags", 0) for v in cases],
                          occ_z0=[getattr(v, "occ_z0", 0.0) for v in cases],
                          occ_dz=[getattr(v, "occ_dz", 0.0) for v in cases])
    return batch, outs_i, outs_l


def run_fwd(cases, seed, batched=True, variant=None):
    A = aw()
    batch, oi, ol = batch_for(cases)
    ws = A.make_workspace(len(cases))
    if variant is not None:
        A.aug_set_variant(A.OP_FWD, variant)
    try:
        if batched:
            A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
        else:
            for b in range(batch.n):
                A.aug_warp_fwd_volume(batch.h_descs[b:b + 1], seed)
        st, bad = A.aug_read_device_status(ws)
    finally:
        if variant is not None:
            A.aug_set_variant(A.OP_FWD, -1)
    torch.cuda.synchronize()
    assert st == 0, (st, bad)
    return ([None if t is None else t.cpu().numpy() for t in oi],
            [None if t is None else t.cpu().numpy() for t in ol])


def check_image(gpu, ref, what="", tol=IMG_TOL):
    """Image parity; ``tol`` defaults to 2e-3 HU (scale it by the intensity
    affine's slope for window/level outputs in [0, 1])."""
    assert gpu.shape == ref.shape
    assert np.all(np.isfinite(gpu)), f"{what}: non-finite output"
    err = np.abs(gpu.astype(np.float64) - ref)
    worst = float(err.max()) if err.size else 0.0
    assert worst <= tol, f"{what}: max |gpu - oracle| = {worst:.3e} (tolerance {tol:.1e})"
    return worst


def check_labels(gpu, ref, tie, what=""):
    keep = tie == 0
    bad = int(np.count_nonzero(gpu[keep] != ref[keep]))
    assert bad == 0, f"{what}: {bad} non-tie label mismatches"
    return int(np.count_nonzero(~keep)), int(np.count_nonzero(gpu[~keep] != ref[~keep]))


def check_grad(gpu, ref, what=""):
    ref = np.asarray(ref, np.float64)
    d = np.abs(np.asarray(gpu, np.float64) - ref)
    scale = np.abs(ref) + np.sqrt(np.mean(ref ** 2))
    worst = float(np.max(d / np.maximum(scale, 1e-300))) if d.size else 0.0
    assert np.all(d <= GRAD_RTOL * scale), f"{what}: worst relative error {worst:.3e}"
    return worst


def summand_scale(v, g):
    """Bound on the L1 norm of the terms whose sum is an affine-gradient entry,
    before any cancellation: each dv/ds_r is a signed sum of tap values with
    weights adding up to 2, so |terms| <= |a g| * 2 max|V| * max obar.  It is
    the scale of an entry whose exact value vanishes (e.g. all taps equal to
    the fill value, where the FP64 reference keeps ~1e-13 of rounding)."""
    ag = float(np.sum(np.abs(np.float64(v.photo_a) * np.asarray(g, np.float64))))
    vmax = max(float(np.max(np.abs(v.image.float().cpu().numpy()))), abs(float(v.fill_image)))
    return ag * 2.0 * vmax * max(v.out_shape)


def check_grad_affine(gpu, ref, what="", floor=0.0):
    """||gpu - ref||_inf <= 1e-4 ||ref||_inf per volume.  A volume whose exact
    gradient (nearly) vanishes has no usable relative bound: only where
    1e-4 ||ref||_inf falls below `floor` (pass 1e-7 * summand_scale, the
    float32 rounding scale of the un-cancelled terms) is the bound `floor`
    instead.  Returns how many volumes used the floor."""
    ref = np.asarray(ref, np.float64).reshape(-1, 12)
    gpu = np.asarray(gpu, np.float64).reshape(-1, 12)
    used = 0
    for b in range(ref.shape[0]):
        rel = GRAD_RTOL * np.max(np.abs(ref[b]))
        lim = rel
        if rel < floor:
            lim = floor
            used += 1
        err = np.max(np.abs(gpu[b] - ref[b]))
        assert err <= lim, f"{what} volume {b}: {err:.3e} > {lim:.3e}"
    return used

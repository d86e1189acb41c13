"""The pipelined forward from host buffers (aug_warp_fwd_host, Sec. 4's
host <-> device FIFO) gives bit-identical outputs to the device-resident
batched forward, for several chunk sizes (one chunk, chunks that do not divide
the batch, one volume per chunk), page-locked and pageable host memory, mixed
input types, image-only and label-only volumes; argument errors."""
import numpy as np
import pytest
import torch

from synth.params import AffineSpec
from synth.workloads import make_case

import _gpu as G

pytestmark = pytest.mark.gpu


def _cases(n, seed0):
    rng = np.random.default_rng(seed0)
    spec = AffineSpec(max_rot_deg=30.0, scale_range=(0.7, 1.4), max_shift_vox=4.0)
    out = []
    for b in range(n):
        si = tuple(int(v) for v in rng.integers(5, 60, 3))
        so = tuple(int(v) for v in rng.integers(3, 50, 3))
        out.append(make_case(si, so, seed=seed0 + b, spec=spec, noise_id=b,
                             dtype="int16" if b % 3 == 1 else "float32"))
    return out


def _host_run(A, cases, seed, chunk, pinned, drop_image=(), drop_label=()):
    imgs = [v.image.contiguous() for v in cases]
    labs = [v.label.contiguous() for v in cases]
    if pinned:
        imgs = [t.pin_memory() for t in imgs]
        labs = [t.pin_memory() for t in labs]
    oi = [None if b in drop_image else
          torch.full(tuple(reversed(v.out_shape)), np.nan, pin_memory=pinned)
          for b, v in enumerate(cases)]
    ol = [None if b in drop_label else
          torch.full(tuple(reversed(v.out_shape)), 77, dtype=torch.uint8, pin_memory=pinned)
          for b, v in enumerate(cases)]
    h = A.host_descriptors(imgs, np.stack([v.T for v in cases]), [v.out_shape for v in cases],
                           labels=labs, out_images=oi, out_labels=ol,
                           photo_a=[v.photo_a for v in cases], photo_b=[v.photo_b for v in cases],
                           noise_sigma=[v.sigma for v in cases],
                           noise_ids=[v.noise_id for v in cases])
    A.aug_warp_fwd_host(h, seed, chunk)
    torch.cuda.synchronize()
    return oi, ol


@pytest.mark.parametrize("chunk,pinned", [(64, True), (5, True), (1, True), (4, False)])
def test_host_pipeline_equals_device_batch(chunk, pinned):
    A = G.aw()
    cases = _cases(13, 300 + chunk)
    seed = 4242
    dev_i, dev_l = G.run_fwd(G.to_device(_cases(13, 300 + chunk)), seed)
    oi, ol = _host_run(A, cases, seed, chunk, pinned)
    for b in range(len(cases)):
        assert np.array_equal(oi[b].numpy(), dev_i[b], equal_nan=False), b
        assert np.array_equal(ol[b].numpy(), dev_l[b]), b


def test_image_only_and_label_only_volumes():
    A = G.aw()
    cases = _cases(6, 900)
    dev_i, dev_l = G.run_fwd(G.to_device(_cases(6, 900)), 5)
    oi, ol = _host_run(A, cases, 5, 4, True, drop_image=(1, 4), drop_label=(0, 2))
    for b in range(6):
        if b not in (1, 4):
            assert np.array_equal(oi[b].numpy(), dev_i[b])
        if b not in (0, 2):
            assert np.array_equal(ol[b].numpy(), dev_l[b])


def test_argument_errors():
    A = G.aw()
    cases = _cases(2, 50)
    h = A.host_descriptors([v.image for v in cases], np.stack([v.T for v in cases]),
                           [v.out_shape for v in cases],
                           out_images=[torch.zeros(tuple(reversed(v.out_shape)))
                                       for v in cases])
    with pytest.raises(A.AugError) as e:
        A.aug_warp_fwd_host(h, 1, 0)
    assert e.value.status == A.AUG_ERR_INVALID_ARG
    bad = h.copy()
    bad["out_nx"][1] = 0
    with pytest.raises(A.AugError) as e:
        A.aug_warp_fwd_host(bad, 1, 2)
    assert e.value.status == A.AUG_ERR_DESCRIPTOR

"""GPU parity of the forward's z + 1 tap-plane reuse (along fully interior
z-runs, and across the interior quads of runs that straddle the input
boundary) on outputs whose z-runs are long enough for both: every reuse
variant must equal the variant without reuse bit for bit, and the default
must match the FP64 oracle at every voxel.  Covers float32 and int16 input,
image-only and label-only outputs, magnification (cells that stay put
between z steps), minification (cells that skip a plane) and an output
that extends past the input in z (runs that enter and leave it)."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth.params import AffineSpec
from synth.workloads import make_case

import _gpu as G

pytestmark = pytest.mark.gpu


def _reuse_variants(A):
    n = A.aug_num_variants(A.OP_FWD)
    return [v for v in range(n)
            if any(t in A.aug_variant_name(A.OP_FWD, v) for t in ("_zr", "_zq"))]


def _cases():
    mild = AffineSpec(max_rot_deg=15.0, scale_range=(0.9, 1.1), max_shift_vox=4.0)
    mag = AffineSpec(max_rot_deg=10.0, scale_range=(0.6, 0.7), max_shift_vox=2.0)
    mini = AffineSpec(max_rot_deg=10.0, scale_range=(1.3, 1.45), max_shift_vox=2.0)
    shapes = [((72, 66, 100), (48, 40, 96), mild, "float32"),
              ((61, 70, 90), (41, 37, 64), mild, "int16"),
              ((50, 47, 60), (45, 50, 70), mag, "float32"),
              ((90, 96, 150), (40, 44, 64), mini, "float32"),
              ((60, 58, 50), (40, 42, 96), mild, "float32")]
    return [make_case(si, so, seed=8100 + b, dtype=dt, spec=sp, noise_id=b)
            for b, (si, so, sp, dt) in enumerate(shapes)]


@pytest.fixture(scope="module")
def cases():
    return G.to_device(_cases())


def _run(cases, seed, variant, with_image=True, with_label=True):
    A = G.aw()
    batch, oi, ol = G.batch_for(cases, with_image=with_image, with_label=with_label)
    ws = A.make_workspace(len(cases))
    A.aug_set_variant(A.OP_FWD, variant)
    try:
        A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
        st, bad = A.aug_read_device_status(ws)
    finally:
        A.aug_set_variant(A.OP_FWD, -1)
    torch.cuda.synchronize()
    assert st == 0, (st, bad)
    return ([None if t is None else t.cpu().numpy() for t in oi],
            [None if t is None else t.cpu().numpy() for t in ol])


def test_reuse_variants_equal_no_reuse_bitwise(cases):
    A = G.aw()
    seed = 0xA5A5_0101
    reuse = _reuse_variants(A)
    assert len(reuse) >= 2
    for wi, wl in ((True, True), (True, False), (False, True)):
        base_i, base_l = _run(cases, seed, 0, wi, wl)
        for var in reuse:
            gi, gl = _run(cases, seed, var, wi, wl)
            name = A.aug_variant_name(A.OP_FWD, var)
            for b in range(len(cases)):
                if wi:
                    assert np.array_equal(gi[b], base_i[b]), (name, b, "image")
                if wl:
                    assert np.array_equal(gl[b], base_l[b]), (name, b, "label")


def test_default_matches_oracle_every_voxel(cases):
    seed = 0xA5A5_0202
    gi, gl = G.run_fwd(cases, seed)
    for b, v in enumerate(cases):
        img, lab, tie, _ = ref.warp_fwd(v, seed)
        G.check_image(gi[b], img, f"reuse case {b}")
        G.check_labels(gl[b], lab, tie, f"reuse case {b}")

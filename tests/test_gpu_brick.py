"""GPU parity of the shared-memory brick forward (the batched forward that
stages each tile's input footprint in shared memory, Sec. 4's sampling served
from the brick) against the FP64 oracle and, bitwise, against the
direct-gather kernel.

The brick copies 4-element chunks whose alignment depends on the input's row
length and on its base address, so the cases cover every nx mod 4, image and
label arrays that start 0..3 elements (bytes for labels) past an aligned
address, tiles that cross the input boundary on every side, warps entirely
outside the input, image-only and label-only outputs, the occlusion and window
steps, and int16 input and strong minification (which take the direct path
inside the same kernel)."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import workloads
from synth.params import AffineSpec, random_window_occlusion
from synth.workloads import make_case

import _gpu as G

pytestmark = pytest.mark.gpu


def _brick_variants(A):
    n = A.aug_num_variants(A.OP_FWD)
    return [v for v in range(n) if A.aug_variant_name(A.OP_FWD, v).startswith("brick")]


def _direct_default(A):
    return A.aug_get_variant(A.OP_FWD) if not A.aug_variant_name(
        A.OP_FWD, A.aug_get_variant(A.OP_FWD)).startswith("brick") else 10


def _misaligned(cases):
    """Re-home each case's image and label at element offset b % 4 (image)
    and byte offset (b + 1) % 4 (labels) inside one shared buffer each."""
    imgs, labs = [], []
    for b, v in enumerate(cases):
        n = v.image.numel()
        buf = torch.empty(n + 8, dtype=v.image.dtype, device="cuda")
        off = b % 4
        buf[off:off + n].copy_(v.image.reshape(-1))
        v.image = buf[off:off + n].view(v.image.shape)
        lb = torch.empty(n + 8, dtype=torch.uint8, device="cuda")
        lo = (b + 1) % 4
        lb[lo:lo + n].copy_(v.label.reshape(-1))
        v.label = lb[lo:lo + n].view(v.label.shape)
        imgs.append(buf)
        labs.append(lb)
    return cases, (imgs, labs)


def _alignment_cases():
    rng = np.random.default_rng(77)
    spec = AffineSpec(max_rot_deg=20.0, scale_range=(0.85, 1.2), max_shift_vox=6.0)
    cases = []
    for b in range(12):
        nx = 40 + b                       # every nx mod 4, three times
        si = (nx, int(rng.integers(20, 50)), int(rng.integers(12, 40)))
        so = (int(rng.integers(30, 70)), int(rng.integers(20, 60)), int(rng.integers(9, 45)))
        cases.append(make_case(si, so, seed=7000 + b, spec=spec, noise_id=b))
    return cases


@pytest.fixture(scope="module")
def aligned_cases():
    cases, keep = _misaligned(G.to_device(_alignment_cases()))
    yield cases
    del keep


def test_brick_variants_match_oracle_on_misaligned_inputs(aligned_cases):
    A = G.aw()
    seed = 0xB51C
    refs = [ref.warp_fwd(v, seed) for v in aligned_cases]
    for var in _brick_variants(A):
        gi, gl = G.run_fwd(aligned_cases, seed, variant=var)
        name = A.aug_variant_name(A.OP_FWD, var)
        for b, v in enumerate(aligned_cases):
            img, lab, tie, _ = refs[b]
            G.check_image(gi[b], img, f"{name} case {b}")
            G.check_labels(gl[b], lab, tie, f"{name} case {b}")


def test_brick_variants_equal_direct_bitwise(aligned_cases):
    A = G.aw()
    seed = 31
    di, dl = G.run_fwd(aligned_cases, seed, variant=_direct_default(A))
    for var in _brick_variants(A):
        gi, gl = G.run_fwd(aligned_cases, seed, variant=var)
        for b in range(len(aligned_cases)):
            assert np.array_equal(gi[b], di[b]), (var, b)
            assert np.array_equal(gl[b], dl[b]), (var, b)


def test_brick_image_only_and_label_only():
    A = G.aw()
    cases = G.to_device(_alignment_cases()[:5])
    seed = 12
    for var in _brick_variants(A):
        A.aug_set_variant(A.OP_FWD, var)
        try:
            for with_image, with_label in ((True, False), (False, True)):
                batch, oi, ol = G.batch_for(cases, with_image=with_image, with_label=with_label)
                ws = A.make_workspace(len(cases))
                A.aug_warp_fwd(batch.d_descs, batch.n, seed, ws)
                assert A.aug_read_device_status(ws)[0] == 0
                torch.cuda.synchronize()
                for b, v in enumerate(cases):
                    img, lab, tie, _ = ref.warp_fwd(v, seed)
                    if with_image:
                        G.check_image(oi[b].cpu().numpy(), img, f"image-only {var} {b}")
                    else:
                        G.check_labels(ol[b].cpu().numpy(), lab, tie, f"label-only {var} {b}")
        finally:
            A.aug_set_variant(A.OP_FWD, -1)


def test_brick_window_occlusion_int16_and_minification():
    A = G.aw()
    rng = np.random.default_rng(5)
    cases = []
    for b in range(6):
        v = make_case((37 + b, 30, 26), (41, 33, 29), seed=7100 + b, noise_id=b,
                      dtype="int16" if b == 4 else "float32")
        a, bb, s, z0, dz = random_window_occlusion(rng, 29)
        if b % 2 == 0:
            v.photo_a, v.photo_b, v.sigma, v.flags = a, bb, s, 1
        if b != 3:
            v.occ_z0, v.occ_dz, v.flags = z0, dz, v.flags | 2
        cases.append(v)
    # 3x minification: the brick exceeds shared memory, the direct path runs
    far = make_case((120, 110, 90), (30, 25, 20), seed=7200, noise_id=9,
                    spec=AffineSpec(extra_scale=(3.0, 3.0, 3.0), max_shift_vox=2.0))
    cases.append(far)
    cases = G.to_device(cases)
    seed = 4
    for var in _brick_variants(A):
        gi, gl = G.run_fwd(cases, seed, variant=var)
        for b, v in enumerate(cases):
            img, lab, tie, _ = ref.warp_fwd(v, seed + 0)
            tol = G.IMG_TOL * (float(v.photo_a) if v.flags & 1 else 1.0)
            G.check_image(gi[b], img, f"variant {var} case {b}", tol=max(tol, 1e-6))
            G.check_labels(gl[b], lab, tie, f"variant {var} case {b}")


def test_brick_small_cases_of_the_forward_tests():
    """The forward tests' small cases (45-degree rotations, scale 0.6-1.6,
    shear, reflections, a 1-voxel input, int16, an output entirely outside)
    through every brick variant, every voxel against the oracle."""
    from test_gpu_fwd import _small_cases
    A = G.aw()
    small = G.to_device(_small_cases())
    seed = 0x5151
    refs = [ref.warp_fwd(v, seed) for v in small]
    for var in _brick_variants(A):
        gi, gl = G.run_fwd(small, seed, variant=var)
        for b in range(len(small)):
            img, lab, tie, _ = refs[b]
            G.check_image(gi[b], img, f"variant {var} case {b}")
            G.check_labels(gl[b], lab, tie, f"variant {var} case {b}")


def test_brick_config1_equals_direct_bitwise():
    """The benchmark's 64-volume batch, packed back to back in one buffer per
    kind as the benchmark packs it (so most volumes start at unaligned
    addresses): every brick variant gives the direct kernel's output bitwise."""
    A = G.aw()
    w = workloads.config1(device="cuda")
    n_img = sum(v.image.numel() for v in w.vols)
    img_all = torch.empty(n_img, device="cuda")
    lab_all = torch.empty(n_img, dtype=torch.uint8, device="cuda")
    a = 0
    for v in w.vols:
        n = v.image.numel()
        img_all[a:a + n].copy_(v.image.reshape(-1))
        lab_all[a:a + n].copy_(v.label.reshape(-1))
        v.image = img_all[a:a + n].view(v.image.shape)
        v.label = lab_all[a:a + n].view(v.label.shape)
        a += n
    seed = 2024
    di, dl = G.run_fwd(w.vols, seed, variant=_direct_default(A))
    for var in _brick_variants(A):
        gi, gl = G.run_fwd(w.vols, seed, variant=var)
        for b in range(len(w.vols)):
            assert np.array_equal(gi[b], di[b]), (var, b)
            assert np.array_equal(gl[b], dl[b]), (var, b)

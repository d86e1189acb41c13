"""GPU parity of the gather adjoint (one thread per input voxel summing over
the output voxels whose cells contain it, the inverse footprint) against the
FP64 oracle adjoint: small cases with 40-degree rotations, scale 0.7-1.4 and
shear, the full 8 x 128^3 workload, occluded slabs, bitwise reproducibility
of grad_in (each sum is taken by one thread in a fixed order, no atomics), and
the reported limit (a strongly magnifying affine is AUG_ERR_UNSUPPORTED)."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import workloads
from synth.params import AffineSpec, random_window_occlusion
from synth.workloads import make_case, upstream_grads

import _gpu as G
from test_gpu_bwd import _cases, run_bwd

pytestmark = pytest.mark.gpu


def _gather_variants():
    A = G.aw()
    n = A.aug_num_variants(A.OP_BWD)
    return [v for v in range(n) if A.aug_variant_name(A.OP_BWD, v).startswith("gather")]


def test_gather_adjoint_small_cases_and_reproducible():
    cases = _cases()
    grads = upstream_grads([v.out_shape for v in cases], seed=31, device="cuda")
    refs = [ref.warp_bwd(v, grads[b]) for b, v in enumerate(cases)]
    assert _gather_variants()
    for var in _gather_variants():
        gin, gaff = run_bwd(cases, grads, variant=var)
        gin2, _ = run_bwd(cases, grads, variant=var, want_gt=False)
        for b in range(len(cases)):
            ri, rt, _ = refs[b]
            G.check_grad(gin[b], ri, f"variant {var} grad_in case {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} grad_T case {b}")
            assert np.array_equal(gin[b], gin2[b]), (var, b)


def test_gather_adjoint_config2_full_size():
    w = workloads.config2(device="cuda")
    refs = [ref.warp_bwd(v, w.g[b], want_grad_in=True) for b, v in enumerate(w.vols)]
    for var in _gather_variants():
        gin, gaff = run_bwd(w.vols, w.g, variant=var)
        for b in range(len(w.vols)):
            ri, rt, _ = refs[b]
            G.check_grad(gin[b], ri, f"variant {var} config2 grad_in {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} config2 grad_T {b}")


def test_gather_adjoint_occlusion():
    rng = np.random.default_rng(19)
    cases = []
    for b in range(3):
        v = make_case((29 + b, 27, 21), (30, 24, 26), seed=7500 + b, noise_id=b)
        _, _, _, z0, dz = random_window_occlusion(rng, 26)
        v.occ_z0, v.occ_dz, v.flags = np.float32(z0), np.float32(max(dz, 3.0)), 2
        cases.append(v)
    cases = G.to_device(cases)
    grads = upstream_grads([v.out_shape for v in cases], seed=32, device="cuda")
    for var in _gather_variants():
        gin, gaff = run_bwd(cases, grads, variant=var)
        for b, v in enumerate(cases):
            ri, rt, _ = ref.warp_bwd(v, grads[b])
            G.check_grad(gin[b], ri, f"variant {var} occluded grad_in {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} occluded grad_T {b}")


def test_gather_adjoint_reports_strong_magnification():
    A = G.aw()
    v = make_case((12, 12, 12), (40, 40, 40), seed=7600,
                  spec=AffineSpec(max_rot_deg=0.0, scale_range=(0.05, 0.05), max_shift_vox=0.0))
    cases = G.to_device([v])
    grads = upstream_grads([v.out_shape], seed=33, device="cuda")
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    gptr = A.pointer_array(grads, "cuda")
    gin = [torch.full_like(v.image, np.nan)]
    ws = A.make_workspace(1)
    A.aug_set_variant(A.OP_BWD, _gather_variants()[0])
    try:
        A.aug_warp_bwd(batch.d_descs, 1, gptr, A.pointer_array(gin, "cuda"), None, ws)
        st, bad = A.aug_read_device_status(ws)
    finally:
        A.aug_set_variant(A.OP_BWD, -1)
    assert (st, bad) == (A.AUG_ERR_UNSUPPORTED, 0)
    assert bool(torch.all(gin[0] == 0))

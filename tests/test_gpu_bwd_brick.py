"""GPU parity of the brick adjoint (the input footprint of each tile in shared
memory: the image brick for dv/ds, a gradient brick for grad_in flushed with
global reductions) against the FP64 oracle adjoint, for every brick variant:
small cases with 40-degree rotations, scale 0.7-1.4 and shear (boundary
tiles, outputs partly outside the input), the full 8 x 128^3 workload, each
output alone, occluded slabs, int16 input (the direct path inside the same
kernel) and the reproducibility of grad_T (a fixed reduction order)."""
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


def _brick_variants():
    A = G.aw()
    n = A.aug_num_variants(A.OP_BWD)
    return [v for v in range(n) if A.aug_variant_name(A.OP_BWD, v).startswith("bbrick")]


def test_brick_adjoint_small_cases():
    cases = _cases()
    grads = upstream_grads([v.out_shape for v in cases], seed=21, device="cuda")
    refs = [ref.warp_bwd(v, grads[b]) for b, v in enumerate(cases)]
    assert _brick_variants()
    for var in _brick_variants():
        gin, gaff = run_bwd(cases, grads, variant=var)
        for b in range(len(cases)):
            ri, rt, _ = refs[b]
            G.check_grad(gin[b], ri, f"variant {var} grad_in case {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} grad_T case {b}")


def test_brick_adjoint_config2_full_size():
    w = workloads.config2(device="cuda")
    refs = [ref.warp_bwd(v, w.g[b]) for b, v in enumerate(w.vols)]
    for var in _brick_variants():
        gin, gaff = run_bwd(w.vols, w.g, variant=var)
        for b in range(len(w.vols)):
            ri, rt, _ = refs[b]
            G.check_grad(gin[b], ri, f"variant {var} config2 grad_in {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} config2 grad_T {b}")


def test_brick_adjoint_each_output_alone_and_reproducible():
    cases = _cases()
    grads = upstream_grads([v.out_shape for v in cases], seed=22, device="cuda")
    for var in _brick_variants():
        gi_only, _ = run_bwd(cases, grads, want_gt=False, variant=var)
        _, gt_only = run_bwd(cases, grads, want_gin=False, variant=var)
        _, gt_again = run_bwd(cases, grads, variant=var)
        assert np.array_equal(gt_only, gt_again), var
        for b, v in enumerate(cases):
            ri, rt, _ = ref.warp_bwd(v, grads[b])
            G.check_grad(gi_only[b], ri, f"variant {var} grad_in only {b}")
            G.check_grad_affine(gt_only[b], rt, f"variant {var} grad_T only {b}")


def test_brick_adjoint_occlusion_and_int16():
    rng = np.random.default_rng(9)
    cases = []
    for b in range(3):
        v = make_case((30 + b, 26, 22), (28, 25, 24), seed=7300 + b, noise_id=b)
        _, _, _, z0, dz = random_window_occlusion(rng, 24)
        v.occ_z0, v.occ_dz, v.flags = np.float32(z0), np.float32(max(dz, 3.0)), 2
        cases.append(v)
    cases = G.to_device(cases)
    grads = upstream_grads([v.out_shape for v in cases], seed=23, device="cuda")
    down = 3.0 / 0.7
    spec = AffineSpec(max_shift_vox=10.0 * down, extra_scale=(down, down, down))
    i16 = make_case((300, 280, 90), (40, 36, 20), seed=7400, dtype="int16", device="cuda",
                    spec=spec)
    gi16 = upstream_grads([i16.out_shape], seed=24, device="cuda")
    for var in _brick_variants():
        gin, gaff = run_bwd(cases, grads, variant=var)
        for b, v in enumerate(cases):
            ri, rt, _ = ref.warp_bwd(v, grads[b])
            G.check_grad(gin[b], ri, f"variant {var} occluded grad_in {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} occluded grad_T {b}")
        _, gaff16 = run_bwd([i16], gi16, want_gin=False, variant=var)
        _, rt16, _ = ref.warp_bwd(i16, gi16[0], want_grad_in=False)
        G.check_grad_affine(gaff16[0], rt16, f"variant {var} int16 grad_T")

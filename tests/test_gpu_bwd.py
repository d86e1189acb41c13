"""GPU parity of the warp adjoint (input volume and 12 affine parameters)
against the FP64 oracle adjoint, which is itself pinned to the operator
transpose and to central finite differences.  Tolerance: 1e-4 relative."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import workloads
from synth.params import AffineSpec
from synth.workloads import make_case, upstream_grads

import _gpu as G

pytestmark = pytest.mark.gpu


def run_bwd(cases, grads, want_gin=True, want_gt=True, variant=None):
    A = G.aw()
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    g = [t.to("cuda").contiguous() for t in grads]
    gptr = A.pointer_array(g, "cuda")
    gin = [torch.full_like(v.image, np.nan, dtype=torch.float32) for v in cases] \
        if want_gin else None
    giptr = A.pointer_array(gin, "cuda") if want_gin else None
    gaff = torch.full((len(cases), 3, 4), np.nan, device="cuda") if want_gt else None
    ws = A.make_workspace(len(cases))
    if variant is not None:
        A.aug_set_variant(A.OP_BWD, variant)
    try:
        A.aug_warp_bwd(batch.d_descs, batch.n, gptr, giptr, gaff, ws)
        st, bad = A.aug_read_device_status(ws)
    finally:
        if variant is not None:
            A.aug_set_variant(A.OP_BWD, -1)
    assert st == 0, (st, bad)
    return ([t.cpu().numpy() for t in gin] if want_gin else None,
            gaff.cpu().numpy() if want_gt else None)


def _cases():
    wild = AffineSpec(max_rot_deg=40.0, scale_range=(0.7, 1.4), max_shift_vox=3.0,
                      max_shear=0.2)
    shapes = [((21, 17, 13), (19, 23, 11)), ((8, 8, 8), (8, 8, 8)), ((40, 9, 30), (33, 31, 9))]
    cases = [make_case(si, so, seed=700 + n, spec=wild, noise_id=n)
             for n, (si, so) in enumerate(shapes)]
    return G.to_device(cases)


def test_small_cases_match_oracle_adjoint():
    cases = _cases()
    grads = upstream_grads([v.out_shape for v in cases], seed=11, device="cuda")
    gin, gaff = run_bwd(cases, grads)
    for b, v in enumerate(cases):
        ri, rt, _ = ref.warp_bwd(v, grads[b])
        G.check_grad(gin[b], ri, f"grad_in case {b}")
        G.check_grad_affine(gaff[b], rt, f"grad_T case {b}")


def test_variants_and_optional_outputs():
    A = G.aw()
    cases = _cases()
    grads = upstream_grads([v.out_shape for v in cases], seed=12, device="cuda")
    base_i, base_t = run_bwd(cases, grads)
    for var in range(A.aug_num_variants(A.OP_BWD)):
        gi, gt = run_bwd(cases, grads, variant=var)
        for b in range(len(cases)):
            G.check_grad(gi[b], base_i[b])
            G.check_grad_affine(gt[b], base_t[b])
    _, gt_only = run_bwd(cases, grads, want_gin=False)
    gi_only, _ = run_bwd(cases, grads, want_gt=False)
    # grad_T is reduced in a fixed order: bitwise reproducible.
    assert np.array_equal(gt_only, base_t)
    for b in range(len(cases)):
        G.check_grad(gi_only[b], base_i[b])


def test_config2_full_size():
    w = workloads.config2(device="cuda")
    gin, gaff = run_bwd(w.vols, w.g)
    worst = 0.0
    for b, v in enumerate(w.vols):
        ri, rt, _ = ref.warp_bwd(v, w.g[b])
        worst = max(worst, G.check_grad(gin[b], ri, f"config2 grad_in {b}"))
        G.check_grad_affine(gaff[b], rt, f"config2 grad_T {b}")
    print(f"config2: worst relative grad_in error {worst:.2e}")


def test_scatter_variants_config2_two_volumes():
    """Every scatter variant with the x-merge (plain and per-quad
    re-classified) against the oracle on two full 128^3 volumes, whose long
    interior runs take the merge paths; the affine gradient alone too."""
    A = G.aw()
    w = workloads.config2(device="cuda", n_vols=2)
    refs = [ref.warp_bwd(v, w.g[b]) for b, v in enumerate(w.vols)]
    names = [(v, A.aug_variant_name(A.OP_BWD, v)) for v in range(A.aug_num_variants(A.OP_BWD))]
    picked = [v for v, nm in names if "atomic_xmerge" in nm]
    assert len(picked) >= 3
    for var in picked:
        gin, gaff = run_bwd(w.vols, w.g, variant=var)
        _, gt_only = run_bwd(w.vols, w.g, want_gin=False, variant=var)
        assert np.array_equal(gt_only, gaff), var
        for b in range(len(w.vols)):
            ri, rt, _ = refs[b]
            G.check_grad(gin[b], ri, f"variant {var} config2 grad_in {b}")
            G.check_grad_affine(gaff[b], rt, f"variant {var} config2 grad_T {b}")


def test_int16_affine_gradient():
    # Full-resolution int16 input, 3 mm / 0.7 mm downscale, a smaller crop
    # centred like the full-size one.
    down = 3.0 / 0.7
    spec = AffineSpec(max_shift_vox=10.0 * down, extra_scale=(down, down, down))
    v = make_case((512, 512, 333), (64, 48, 40), seed=401, dtype="int16", device="cuda",
                  spec=spec)
    g = upstream_grads([v.out_shape], seed=13, device="cuda")
    _, gaff = run_bwd([v], g, want_gin=False)
    _, rt, _ = ref.warp_bwd(v, g[0], want_grad_in=False)
    G.check_grad_affine(gaff[0], rt, "int16 grad_T")


def test_autograd_function():
    A = G.aw()
    cases = G.to_device([make_case((24, 20, 16), (24, 20, 16), seed=800 + b, noise_id=b)
                         for b in range(3)])
    image = torch.stack([v.image for v in cases]).requires_grad_(True)
    affine = torch.tensor(np.stack([v.T for v in cases]), device="cuda", requires_grad=True)
    out = A.AugWarp.apply(image, affine, (24, 20, 16))
    g = torch.randn_like(out)
    (out * g).sum().backward()
    for b, v in enumerate(cases):
        v.photo_a, v.photo_b, v.sigma = np.float32(1), np.float32(0), np.float32(0)
        img, _, _, _ = ref.warp_fwd(v, 0, want_label=False)
        G.check_image(out[b].detach().cpu().numpy(), img)
        ri, rt, _ = ref.warp_bwd(v, g[b])
        G.check_grad(image.grad[b].cpu().numpy(), ri)
        G.check_grad_affine(affine.grad[b].cpu().numpy(), rt)

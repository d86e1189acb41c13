"""Edge cases of the CUDA path through the C ABI, each against the FP64 oracle:
batches larger than one scheduler chunk (hundreds of volumes, mixed float32 /
int16), label-only and image-only descriptors, a non-zero fill label, the
largest allowed dimension, affine entries at the allowed limit, CUDA-graph
replay after the descriptors are edited in place, the autotuner, and the
argument / descriptor error paths."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth.params import AffineSpec
from synth.workloads import VolumeCase, make_case, softmax_probs, upstream_grads

import _gpu as G

pytestmark = pytest.mark.gpu


def _many(n, seed0):
    rng = np.random.default_rng(seed0)
    spec = AffineSpec(max_rot_deg=30.0, scale_range=(0.7, 1.4), max_shift_vox=3.0)
    cases = []
    for b in range(n):
        si = tuple(int(v) for v in rng.integers(2, 14, 3))
        so = tuple(int(v) for v in rng.integers(1, 12, 3))
        cases.append(make_case(si, so, seed=seed0 + b, spec=spec, noise_id=b,
                               dtype="int16" if b % 3 == 0 else "float32"))
    return G.to_device(cases)


def _first_variant(op, prefix):
    A = G.aw()
    for v in range(A.aug_num_variants(op)):
        if A.aug_variant_name(op, v).startswith(prefix):
            return v
    raise AssertionError(prefix)


@pytest.mark.parametrize("prefix", [None, "brick", "bulk"])
def test_forward_many_volumes_across_scheduler_chunks(prefix):
    A = G.aw()
    cases = _many(300, 5000)
    seed = 17
    variant = None if prefix is None else _first_variant(A.OP_FWD, prefix)
    gi, gl = G.run_fwd(cases, seed, variant=variant)
    for b, v in enumerate(cases):
        img, lab, tie, _ = ref.warp_fwd(v, seed)
        G.check_image(gi[b], img, f"{prefix} vol {b}")
        G.check_labels(gl[b], lab, tie, f"{prefix} vol {b}")


@pytest.mark.parametrize("prefix", [None, "bbrick", "gather"])
def test_adjoint_many_volumes_across_scheduler_chunks(prefix):
    from test_gpu_bwd import run_bwd
    A = G.aw()
    cases = [v for v in _many(400, 7000) if v.image.dtype == torch.float32]
    assert len(cases) > 256
    grads = upstream_grads([v.out_shape for v in cases], seed=3, device="cuda")
    variant = None if prefix is None else _first_variant(A.OP_BWD, prefix)
    gin, gaff = run_bwd(cases, grads, variant=variant)
    floored = 0
    for b, v in enumerate(cases):
        ri, rt, _ = ref.warp_bwd(v, grads[b])
        G.check_grad(gin[b], ri, f"grad_in {b}")
        floor = 1e-7 * G.summand_scale(v, grads[b].cpu().numpy())
        floored += G.check_grad_affine(gaff[b], rt, f"grad_T {b}", floor=floor)
    print(f"grad_T: {floored} of {len(cases)} volumes had a gradient cancelled below the "
          "float32 rounding scale of its terms and used that floor")


def test_iou_many_volumes_across_scheduler_chunks():
    from test_gpu_iou import check_loss, run_iou
    cases = _many(270, 9000)
    p = softmax_probs([v.out_shape for v in cases], seed=4, device="cuda")
    loss, gp = run_iou(cases, p, 6)
    rl, rg, _ = ref.warp_iou(cases, p, 6)
    check_loss(loss, rl)
    G.check_grad(gp, rg, "grad_p")


def test_label_only_and_image_only_descriptors_and_fill_label():
    A = G.aw()
    cases = G.to_device([make_case((20, 18, 15), (17, 19, 13), seed=11 + b, noise_id=b)
                         for b in range(3)])
    cases[2].fill_label = 9
    cases[2].T = cases[2].T.copy()
    cases[2].T[:, 3] += np.float32(6.0)  # part of the crop outside the input
    batch, oi, ol = G.batch_for(cases)
    batch.h_descs["out_image"][0] = 0      # labels only
    batch.h_descs["out_label"][1] = 0      # image only
    batch.upload()
    ws = A.make_workspace(3)
    A.aug_warp_fwd(batch.d_descs, 3, 5, ws)
    assert A.aug_read_device_status(ws)[0] == 0
    assert torch.isnan(oi[0]).all() and (ol[1] == 77).all()
    img1, _, _, _ = ref.warp_fwd(cases[1], 5)
    G.check_image(oi[1].cpu().numpy(), img1)
    _, lab0, tie0, _ = ref.warp_fwd(cases[0], 5)
    G.check_labels(ol[0].cpu().numpy(), lab0, tie0)
    img2, lab2, tie2, _ = ref.warp_fwd(cases[2], 5)
    G.check_image(oi[2].cpu().numpy(), img2)
    G.check_labels(ol[2].cpu().numpy(), lab2, tie2)
    assert (ol[2].cpu().numpy() == 9).any()


def test_largest_dimension_and_extreme_affine():
    img = torch.randn((1, 1, 8192), device="cuda") * 100
    lab = (torch.arange(8192, device="cuda") % 6).to(torch.uint8).reshape(1, 1, 8192)
    T = np.zeros((3, 4), np.float32)
    T[0, 0] = 1.0
    T[1, 1] = 1.0
    T[2, 2] = 1.0
    a = VolumeCase(image=img, label=lab, out_shape=(8192, 2, 3), T=T, sigma=np.float32(3.0))
    T2 = np.zeros((3, 4), np.float32)
    T2[0, 0], T2[1, 1], T2[2, 2] = 64.0, -64.0, 64.0
    T2[0, 3], T2[1, 3], T2[2, 3] = -1048576.0, 1048576.0, 0.25
    b = VolumeCase(image=torch.randn((5, 6, 7), device="cuda"), label=None,
                   out_shape=(3, 4, 8192), T=T2, noise_id=1)
    T3 = np.zeros((3, 4), np.float32)
    T3[0, 0], T3[1, 1], T3[2, 2] = 0.01, 0.02, 0.015
    c = VolumeCase(image=torch.randn((9, 9, 9), device="cuda"), label=None,
                   out_shape=(700, 300, 5), T=T3, noise_id=2)
    gi, gl = G.run_fwd([a, b, c], seed=8)
    for k, v in enumerate([a, b, c]):
        img_r, lab_r, tie, _ = ref.warp_fwd(v, 8)
        G.check_image(gi[k], img_r, f"case {k}")
        if lab_r is not None:
            G.check_labels(gl[k], lab_r, tie)


def test_graph_replay_with_descriptors_edited_in_place():
    A = G.aw()
    cases = G.to_device([make_case((25, 21, 17), (22, 20, 18), seed=60 + b, noise_id=b)
                         for b in range(4)])
    batch, oi, ol = G.batch_for(cases)
    ws = A.make_workspace(4)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A.aug_warp_fwd(batch.d_descs, 4, 3, ws)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            A.aug_warp_fwd(batch.d_descs, 4, 3, ws)
    rng = np.random.default_rng(1)
    for rep in range(3):
        for v in cases:
            v.T = v.T.copy()
            v.T[:, 3] += rng.uniform(-2, 2, 3).astype(np.float32)
            v.sigma = np.float32(rng.uniform(0, 40))
        batch.h_descs["affine"] = np.stack([v.T.reshape(12) for v in cases])
        batch.h_descs["noise_sigma"] = [v.sigma for v in cases]
        batch.upload()
        with torch.cuda.stream(stream):
            g.replay()
        torch.cuda.synchronize()
        for b, v in enumerate(cases):
            img, lab, tie, _ = ref.warp_fwd(v, 3)
            G.check_image(oi[b].cpu().numpy(), img, f"replay {rep} vol {b}")
            G.check_labels(ol[b].cpu().numpy(), lab, tie)


def test_autotuner_selects_a_variant_and_results_do_not_change():
    A = G.aw()
    cases = G.to_device([make_case((30, 26, 22), (28, 24, 20), seed=80 + b, noise_id=b)
                         for b in range(3)])
    base_i, base_l = G.run_fwd(cases, seed=2)
    batch, oi, ol = G.batch_for(cases)
    ws = A.make_workspace(3)
    try:
        best, ms = A.aug_autotune(A.OP_FWD, batch, ws, seed=2, reps=2)
        assert 0 <= best < A.aug_num_variants(A.OP_FWD) and ms > 0
        assert A.aug_get_variant(A.OP_FWD) == best
        A.aug_warp_fwd(batch.d_descs, 3, 2, ws)
        torch.cuda.synchronize()
        for b in range(3):
            assert np.array_equal(oi[b].cpu().numpy(), base_i[b])
            assert np.array_equal(ol[b].cpu().numpy(), base_l[b])
    finally:
        A.aug_set_variant(A.OP_FWD, -1)


def test_error_paths():
    A = G.aw()
    L = A.lib()
    cases = G.to_device([make_case((10, 10, 10), (8, 8, 8), seed=1, dtype="int16")])
    batch, oi, ol = G.batch_for(cases)
    ws = A.make_workspace(1)
    # Workspace too small / misaligned.
    with pytest.raises(A.AugError) as e:
        A.aug_warp_fwd(batch.d_descs, 1, 0, ws[: ws.numel() // 2])
    assert e.value.status == A.AUG_ERR_WORKSPACE
    with pytest.raises(A.AugError):
        A.aug_warp_fwd(batch.d_descs, 1, 0, ws[1:])
    # int16 input with an input gradient requested: descriptor error, recorded on the device.
    g = upstream_grads([cases[0].out_shape], seed=1, device="cuda")
    gin = [torch.zeros((10, 10, 10), device="cuda")]
    A.aug_warp_bwd(batch.d_descs, 1, A.pointer_array(g, "cuda"), A.pointer_array(gin, "cuda"),
                   None, ws)
    st, bad = A.aug_read_device_status(ws)
    assert st == A.AUG_ERR_DESCRIPTOR and bad == 0
    # IOU without a label volume.
    batch2, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    batch2.h_descs["label"][0] = 0
    batch2.upload()
    ws2 = A.make_workspace(1, 6)
    p = softmax_probs([cases[0].out_shape], seed=1, device="cuda")
    A.iou_loss_fwd_bwd(batch2.d_descs, 1, p, 6, torch.empty(1, device="cuda"), None, ws2)
    assert A.aug_read_device_status(ws2)[0] == A.AUG_ERR_DESCRIPTOR
    assert L.aug_read_device_status(None, None, 1, None) == A.AUG_ERR_WORKSPACE

"""GPU parity of the fused label-warp + soft IOU loss (Sec. 5.C) against the
FP64 oracle (label warp followed by the loss), plus the closed-form perfect
prediction case and fused == unfused."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import workloads
from synth.params import AffineSpec
from synth.workloads import make_case, softmax_probs

import _gpu as G

pytestmark = pytest.mark.gpu


def run_iou(cases, p, C, want_grad=True, variant=None):
    A = G.aw()
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    loss = torch.full((len(cases),), np.nan, device="cuda")
    gp = torch.full_like(p, np.nan) if want_grad else None
    ws = A.make_workspace(len(cases), C)
    if variant is not None:
        A.aug_set_variant(A.OP_IOU, variant)
    try:
        A.iou_loss_fwd_bwd(batch.d_descs, batch.n, p, C, loss, gp, ws)
        st, bad = A.aug_read_device_status(ws)
    finally:
        if variant is not None:
            A.aug_set_variant(A.OP_IOU, -1)
    assert st == 0, (st, bad)
    return loss.cpu().numpy(), (gp.cpu().numpy() if want_grad else None)


def check_loss(gpu, refl):
    assert np.max(np.abs(gpu - refl)) <= 1e-5 * max(1.0, np.max(np.abs(refl)))


def _cases():
    wild = AffineSpec(max_rot_deg=40.0, scale_range=(0.7, 1.4), max_shift_vox=3.0)
    shapes = [((30, 22, 19), (33, 17, 21)), ((8, 8, 8), (9, 7, 5)), ((50, 40, 12), (41, 37, 14))]
    return G.to_device([make_case(si, so, seed=900 + n, spec=wild, noise_id=n)
                        for n, (si, so) in enumerate(shapes)])


@pytest.mark.parametrize("C", [6, 3, 1, 8])
def test_small_cases_match_oracle(C):
    cases = _cases()
    p = softmax_probs([v.out_shape for v in cases], seed=21, device="cuda", n_classes=C)
    loss, gp = run_iou(cases, p, C)
    rl, rg, _ = ref.warp_iou(cases, p, C)
    check_loss(loss, rl)
    G.check_grad(gp, rg, f"grad_p C={C}")
    loss2, _ = run_iou(cases, p, C, want_grad=False)
    assert np.array_equal(loss2, loss)


def test_variants_bitwise_equal():
    A = G.aw()
    cases = _cases()
    p = softmax_probs([v.out_shape for v in cases], seed=22, device="cuda")
    base = run_iou(cases, p, 6)
    for var in range(A.aug_num_variants(A.OP_IOU)):
        l, g = run_iou(cases, p, 6, variant=var)
        check_loss(l, base[0])
        G.check_grad(g, base[1])


def test_perfect_prediction_and_fused_equals_unfused():
    """p = one-hot(warped labels) gives loss 0 and the closed-form gradient
    (-1/|y| on the class, +1/|y| elsewhere, scaled by 1/(B C)); the labels
    used are produced by the forward kernel, so this also checks that the
    fused loss sees exactly the labels the forward warp writes."""
    cases = _cases()
    _, gl = G.run_fwd(cases, seed=0)
    C = 6
    parts = [np.eye(C, dtype=np.float32)[np.minimum(l.reshape(-1), C - 1)].T.reshape(-1)
             for l in gl]
    p = torch.from_numpy(np.concatenate(parts)).cuda()
    loss, gp = run_iou(cases, p, C)
    assert np.all(np.abs(loss) < 1e-6)
    off = 0
    B = len(cases)
    for b, l in enumerate(gl):
        y = l.reshape(-1)
        for c in range(C):
            Y = np.count_nonzero(y == c)
            seg = gp[off + c * y.size: off + (c + 1) * y.size]
            if Y == 0:
                assert np.all(seg == 0)
            else:
                exp = np.where(y == c, -1.0 / Y, 1.0 / Y) / (B * C)
                G.check_grad(seg, exp)
        off += C * y.size
    # Unfused: oracle loss on the labels the forward kernel wrote.
    p = softmax_probs([v.out_shape for v in cases], seed=23, device="cuda")
    loss, _ = run_iou(cases, p, C, want_grad=False)
    ph = p.cpu().numpy()
    off = 0
    for b, l in enumerate(gl):
        n = l.size
        lc, _, _ = ref.iou(ph[off: off + C * n].reshape(C, n), l.reshape(-1), C)
        assert abs(loss[b] - lc.mean()) < 1e-5
        off += C * n


def test_config3_full_size():
    w = workloads.config3(device="cuda")
    loss, gp = run_iou(w.vols, w.p, 6)
    rl, rg, _ = ref.warp_iou(w.vols, w.p, 6)
    check_loss(loss, rl)
    worst = G.check_grad(gp, rg, "config3 grad_p")
    print(f"config3: loss {loss}, worst relative grad error {worst:.2e}")


def test_autograd_function():
    A = G.aw()
    cases = G.to_device([make_case((20, 18, 16), (20, 18, 16), seed=950 + b, noise_id=b)
                         for b in range(2)])
    p = softmax_probs([v.out_shape for v in cases], seed=24, device="cuda")
    pt = p.reshape(2, 6, 16, 18, 20).clone().requires_grad_(True)
    labels = torch.stack([v.label for v in cases])
    affine = torch.tensor(np.stack([v.T for v in cases]), device="cuda")
    loss = A.IouLoss.apply(pt, labels, affine)
    loss.backward()
    rl, rg, _ = ref.warp_iou(cases, p, 6)
    assert abs(loss.item() - rl.mean()) < 1e-5
    G.check_grad(pt.grad.reshape(-1).cpu().numpy(), rg)

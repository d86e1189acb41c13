"""GPU parity of the overlap-loss variants of Sec. 5.C in the fused label-warp
kernels (Dice, the p^m family, and the softmax over class scores fused in)
against the FP64 oracle, plus: the plain IOU call is the same computation,
tile variants agree, one-hot predictions give Dice 0, a single class under the
softmax has zero gradient, full-size 8x120x120x160, argument errors, autograd."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import workloads
from synth.params import AffineSpec
from synth.workloads import class_logits, make_case, softmax_probs

import _gpu as G

pytestmark = pytest.mark.gpu

# (kind, power, logits)
VARIANTS = [(1, 1.0, False), (0, 2.0, False), (1, 0.5, False), (0, 1.0, True),
            (1, 1.0, True), (0, 3.0, True), (1, 1.5, True), (1, 4.0, False)]


def run_loss(cases, x, C, kind, power, logits, want_grad=True, variant=None):
    A = G.aw()
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    loss = torch.full((len(cases),), np.nan, device="cuda")
    gx = torch.full_like(x, np.nan) if want_grad else None
    ws = A.make_workspace(len(cases), C)
    if variant is not None:
        A.aug_set_variant(A.OP_IOU, variant)
    try:
        A.seg_loss_fwd_bwd(batch.d_descs, batch.n, x, C, loss, gx, ws, kind, power, logits)
        st, bad = A.aug_read_device_status(ws)
    finally:
        if variant is not None:
            A.aug_set_variant(A.OP_IOU, -1)
    assert st == 0, (st, bad)
    return loss.cpu().numpy(), (gx.cpu().numpy() if want_grad else None)


def check_loss(gpu, refl):
    assert np.max(np.abs(gpu - refl)) <= 1e-5 * max(1.0, np.max(np.abs(refl))), (gpu, refl)


def _cases():
    wild = AffineSpec(max_rot_deg=40.0, scale_range=(0.7, 1.4), max_shift_vox=3.0)
    shapes = [((30, 22, 19), (33, 17, 21)), ((8, 8, 8), (9, 7, 5)), ((50, 40, 12), (41, 37, 14))]
    return G.to_device([make_case(si, so, seed=1900 + n, spec=wild, noise_id=n)
                        for n, (si, so) in enumerate(shapes)])


def _inputs(cases, C, logits, seed):
    shapes = [v.out_shape for v in cases]
    if logits:
        return class_logits(shapes, seed=seed, device="cuda", n_classes=C)
    return softmax_probs(shapes, seed=seed, device="cuda", n_classes=C)


@pytest.mark.parametrize("kind,power,logits", VARIANTS)
@pytest.mark.parametrize("C", [6, 3, 8, 1])
def test_small_cases_match_oracle(kind, power, logits, C):
    cases = _cases()
    x = _inputs(cases, C, logits, seed=31 + C)
    loss, gx = run_loss(cases, x, C, kind, power, logits)
    rl, rg, _ = ref.warp_loss(cases, x, C, kind, power, logits)
    check_loss(loss, rl)
    G.check_grad(gx, rg, f"grad kind={kind} m={power} logits={logits} C={C}")
    loss2, _ = run_loss(cases, x, C, kind, power, logits, want_grad=False)
    assert np.array_equal(loss2, loss)


def test_plain_iou_is_the_same_computation():
    A = G.aw()
    cases = _cases()
    p = softmax_probs([v.out_shape for v in cases], seed=40, device="cuda")
    l1, g1 = run_loss(cases, p, 6, A.AUG_LOSS_IOU, 1.0, False)
    from test_gpu_iou import run_iou
    l0, g0 = run_iou(cases, p, 6)
    assert np.array_equal(l0, l1) and np.array_equal(g0, g1)


@pytest.mark.parametrize("kind,power,logits", [(1, 2.0, True), (0, 1.0, True), (1, 0.5, False)])
def test_tile_variants_agree(kind, power, logits):
    A = G.aw()
    cases = _cases()
    x = _inputs(cases, 6, logits, seed=41)
    base = run_loss(cases, x, 6, kind, power, logits)
    for var in range(A.aug_num_variants(A.OP_IOU)):
        l, g = run_loss(cases, x, 6, kind, power, logits, variant=var)
        check_loss(l, base[0])
        G.check_grad(g, base[1])


def test_one_hot_prediction_gives_zero_dice_and_single_class_softmax_no_gradient():
    cases = _cases()
    _, gl = G.run_fwd(cases, seed=0)
    C = 6
    parts = [np.eye(C, dtype=np.float32)[np.minimum(l.reshape(-1), C - 1)].T.reshape(-1)
             for l in gl]
    p = torch.from_numpy(np.concatenate(parts)).cuda()
    for power in (1.0, 2.5):
        loss, _ = run_loss(cases, p, C, 1, power, False)
        assert np.all(np.abs(loss) < 1e-6)
    x = class_logits([v.out_shape for v in cases], seed=42, device="cuda", n_classes=1)
    _, gx = run_loss(cases, x, 1, 0, 2.0, True)
    assert np.all(gx == 0.0)


@pytest.mark.parametrize("kind,power", [(1, 2.0), (0, 1.0)])
def test_full_size_8x120x120x160_with_softmax(kind, power):
    w = workloads.config3(device="cuda")
    x = class_logits([v.out_shape for v in w.vols], seed=3, device="cuda")
    loss, gx = run_loss(w.vols, x, 6, kind, power, True)
    rl, rg, _ = ref.warp_loss(w.vols, x, 6, kind, power, True)
    check_loss(loss, rl)
    worst = G.check_grad(gx, rg, "full-size grad_x")
    print(f"kind {kind} m {power}: loss {loss}, worst relative grad error {worst:.2e}")


def test_argument_errors():
    A = G.aw()
    cases = _cases()[:1]
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    x = softmax_probs([cases[0].out_shape], seed=1, device="cuda")
    loss = torch.empty(1, device="cuda")
    ws = A.make_workspace(1, 6)
    for kind, power in [(2, 1.0), (-1, 1.0), (0, 0.0), (0, -1.0), (0, float("nan")),
                        (1, float("inf"))]:
        with pytest.raises(A.AugError) as e:
            A.seg_loss_fwd_bwd(batch.d_descs, 1, x, 6, loss, None, ws, kind, power, False)
        assert e.value.status == A.AUG_ERR_INVALID_ARG


def test_autograd_function():
    A = G.aw()
    cases = G.to_device([make_case((20, 18, 16), (20, 18, 16), seed=1950 + b, noise_id=b)
                         for b in range(2)])
    x = class_logits([v.out_shape for v in cases], seed=43, device="cuda")
    xt = x.reshape(2, 6, 16, 18, 20).clone().requires_grad_(True)
    labels = torch.stack([v.label for v in cases])
    affine = torch.tensor(np.stack([v.T for v in cases]), device="cuda")
    loss = A.SegLoss.apply(xt, labels, affine, A.AUG_LOSS_DICE, 2.0, True)
    loss.backward()
    rl, rg, _ = ref.warp_loss(cases, x, 6, 1, 2.0, True)
    assert abs(loss.item() - rl.mean()) < 1e-5
    G.check_grad(xt.grad.reshape(-1).cpu().numpy(), rg)

"""The allocation-free IOU entry point against the regular one.

iou_loss_fwd_bwd_noalloc serves callers that are not allowed to allocate
device memory (a framework that owns the whole memory budget, a loop that may
not allocate after start-up): it runs the same kernels with the library's own
fixed scratch array instead of a caller workspace.  This file is collected last
so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from synth.params import AffineSpec
from synth.workloads import make_case, softmax_probs

import _gpu as G

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point_twice():
    A = G.aw()
    spec = AffineSpec(max_rot_deg=30.0, scale_range=(0.8, 1.25), max_shift_vox=3.0)
    shapes = [((34, 28, 21), (31, 23, 19)), ((17, 40, 12), (25, 18, 22)),
              ((60, 55, 30), (48, 40, 26))]
    cases = G.to_device([make_case(si, so, seed=990 + n, spec=spec, noise_id=n)
                         for n, (si, so) in enumerate(shapes)])
    C = 6
    p = softmax_probs([v.out_shape for v in cases], seed=31, device="cuda", n_classes=C)
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    n = batch.n
    # Existing entry point, with a caller workspace.
    ws = A.make_workspace(n, C)
    ref_loss = torch.empty(n, device="cuda")
    ref_grad = torch.empty_like(p)
    A.iou_loss_fwd_bwd(batch.d_descs, n, p, C, ref_loss, ref_grad, ws)
    assert A.aug_read_device_status(ws)[0] == 0
    ref_loss, ref_grad = ref_loss.cpu().numpy(), ref_grad.cpu().numpy()
    # Two calls in a row: the second reuses the scratch the first left behind.
    for call in range(2):
        loss = torch.full((n,), np.nan, device="cuda")
        grad = torch.full_like(p, np.nan)
        status = torch.full((2,), -7, dtype=torch.int32, device="cuda")
        A.iou_loss_fwd_bwd_noalloc(batch.d_descs, n, p, C, loss, grad, status)
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0, -1], call
        got_loss = loss.cpu().numpy()
        assert np.max(np.abs(got_loss - ref_loss)) <= 1e-5 * max(1.0, np.abs(ref_loss).max())
        G.check_grad(grad.cpu().numpy(), ref_grad, f"no-alloc call {call}")


def _workspace_reference(A, batch, p, C, with_grad=True):
    ws = A.make_workspace(batch.n, C)
    loss = torch.empty(batch.n, device="cuda")
    grad = torch.empty_like(p) if with_grad else None
    A.iou_loss_fwd_bwd(batch.d_descs, batch.n, p, C, loss, grad, ws)
    assert A.aug_read_device_status(ws)[0] == 0
    return loss.cpu().numpy(), None if grad is None else grad.cpu().numpy()


def test_noalloc_at_its_limits_and_loss_only():
    """64 volumes and 8 classes fill the array's partial-sum slots to their
    documented size (its 256-block cap applies to both passes); then a call
    without a gradient buffer writes the loss and nothing else."""
    A = G.aw()
    spec = AffineSpec(max_rot_deg=20.0, scale_range=(0.9, 1.1), max_shift_vox=2.0)
    rng = np.random.default_rng(17)
    cases = []
    for n in range(64):
        si = tuple(int(v) for v in rng.integers(6, 20, 3))
        so = tuple(int(v) for v in rng.integers(5, 18, 3))
        cases.append(make_case(si, so, seed=2000 + n, spec=spec, noise_id=n))
    cases = G.to_device(cases)
    C = 8
    p = softmax_probs([v.out_shape for v in cases], seed=32, device="cuda", n_classes=C)
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    ref_loss, ref_grad = _workspace_reference(A, batch, p, C)
    loss = torch.full((64,), np.nan, device="cuda")
    grad = torch.full_like(p, np.nan)
    status = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    A.iou_loss_fwd_bwd_noalloc(batch.d_descs, 64, p, C, loss, grad, status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, -1]
    assert np.max(np.abs(loss.cpu().numpy() - ref_loss)) <= 1e-5 * max(1.0, np.abs(ref_loss).max())
    G.check_grad(grad.cpu().numpy(), ref_grad, "no-alloc at 64 volumes x 8 classes")
    # loss only: the same losses, and a gradient buffer passed to nobody stays as it was
    untouched = torch.full_like(p, 123.0)
    loss2 = torch.full((64,), np.nan, device="cuda")
    A.iou_loss_fwd_bwd_noalloc(batch.d_descs, 64, p, C, loss2, None, status)
    torch.cuda.synchronize()
    assert np.array_equal(loss2.cpu().numpy(), loss.cpu().numpy())
    assert bool(torch.all(untouched == 123.0))


def test_noalloc_reports_an_invalid_descriptor():
    """(status, bad volume) follow aug_read_device_status: the first invalid
    descriptor's index, and (0, -1) again on the next valid call."""
    A = G.aw()
    cases = G.to_device([make_case((20, 18, 14), (16, 15, 12), seed=3100 + n, noise_id=n)
                         for n in range(3)])
    C = 4
    p = softmax_probs([v.out_shape for v in cases], seed=33, device="cuda", n_classes=C)
    batch, _, _ = G.batch_for(cases, with_image=False, with_label=False)
    # volume 1 without its label array (the descriptor's second field, bytes
    # 8..15 of its 144): a descriptor error for the loss
    bad = batch.d_descs.clone().view(batch.n, 144)
    bad[1, 8:16] = 0
    loss = torch.empty(3, device="cuda")
    status = torch.full((2,), -7, dtype=torch.int32, device="cuda")
    A.iou_loss_fwd_bwd_noalloc(bad, 3, p, C, loss, None, status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [A.AUG_ERR_DESCRIPTOR, 1]
    A.iou_loss_fwd_bwd_noalloc(batch.d_descs, 3, p, C, loss, None, status)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, -1]


def test_noalloc_rejects_sizes_beyond_its_limit():
    A = G.aw()
    L = A.lib()
    dummy = torch.zeros(16, device="cuda")
    assert L.iou_loss_fwd_bwd_noalloc(A._ptr(dummy), 65, A._ptr(dummy), 6, A._ptr(dummy), None,
                                      None, None) == A.AUG_ERR_INVALID_ARG
    assert L.iou_loss_fwd_bwd_noalloc(A._ptr(dummy), 2, A._ptr(dummy), 9, A._ptr(dummy), None,
                                      None, None) == A.AUG_ERR_UNSUPPORTED

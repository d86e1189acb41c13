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
        assert status.cpu().tolist() == [0, 0], call
        got_loss = loss.cpu().numpy()
        assert np.max(np.abs(got_loss - ref_loss)) <= 1e-5 * max(1.0, np.abs(ref_loss).max())
        G.check_grad(grad.cpu().numpy(), ref_grad, f"no-alloc call {call}")


def test_noalloc_rejects_sizes_beyond_its_limit():
    A = G.aw()
    L = A.lib()
    dummy = torch.zeros(16, device="cuda")
    assert L.iou_loss_fwd_bwd_noalloc(A._ptr(dummy), 65, A._ptr(dummy), 6, A._ptr(dummy), None,
                                      None, None) == A.AUG_ERR_INVALID_ARG
    assert L.iou_loss_fwd_bwd_noalloc(A._ptr(dummy), 2, A._ptr(dummy), 9, A._ptr(dummy), None,
                                      None, None) == A.AUG_ERR_UNSUPPORTED

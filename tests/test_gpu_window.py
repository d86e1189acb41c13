"""GPU parity of the occlusion and window/level steps (Sec. 4) against the FP64
oracle, on the batched and the per-volume forward and on the adjoint.  Window
outputs are in [0, 1]: the 2e-3 HU image tolerance is scaled by the window's
slope a = 1/(hi - lo)."""
import numpy as np
import pytest

from oracle import ref
from synth.params import AffineSpec, random_window_occlusion
from synth.workloads import make_case, upstream_grads

import _gpu as G

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(31)
    spec = AffineSpec(max_rot_deg=30.0, scale_range=(0.8, 1.25), max_shift_vox=4.0)
    shapes = [((40, 36, 30), (37, 33, 28)), ((24, 30, 18), (20, 26, 35)),
              ((50, 20, 25), (45, 23, 17)), ((16, 16, 16), (16, 16, 13))]
    cases = []
    for n, (si, so) in enumerate(shapes):
        v = make_case(si, so, seed=1100 + n, spec=spec, noise_id=n,
                      dtype="int16" if n == 2 else "float32")
        a, b, s, z0, dz = random_window_occlusion(rng, so[2])
        v.flags = [1, 2, 3, 3][n]
        if v.flags & 1:
            v.photo_a, v.photo_b, v.sigma = a, b, s
        v.occ_z0, v.occ_dz = z0, dz
        cases.append(v)
    # Integer slab ends: the inclusive bounds are decided exactly.
    cases[3].occ_z0, cases[3].occ_dz = np.float32(4.0), np.float32(3.0)
    return G.to_device(cases)


@pytest.mark.parametrize("batched", [True, False])
def test_window_and_occlusion_match_oracle(batched):
    cases = _cases()
    seed = 4242
    gi, gl = G.run_fwd(cases, seed, batched=batched)
    for b, v in enumerate(cases):
        img, lab, tie, _ = ref.warp_fwd(v, seed)
        tol = G.IMG_TOL * (float(v.photo_a) if v.flags & 1 else 1.0)
        G.check_image(gi[b], img, f"case {b}", tol=tol)
        G.check_labels(gl[b], lab, tie, f"case {b}")
        if v.flags & 2:
            k = np.arange(v.out_shape[2])
            occ = (k >= np.float64(v.occ_z0)) & (k <= np.float64(v.occ_z0) + np.float64(v.occ_dz))
            assert np.all(gi[b][occ] == 0.0)
        if v.flags & 1:
            assert gi[b].min() >= 0.0 and gi[b].max() <= 1.0


def test_adjoint_of_occluded_warp_and_window_rejected():
    from test_gpu_bwd import run_bwd
    A = G.aw()
    cases = _cases()
    occl = [v for v in cases if v.flags == 2]
    g = upstream_grads([v.out_shape for v in occl], seed=5, device="cuda")
    gin, gaff = run_bwd(occl, g)
    for b, v in enumerate(occl):
        ri, rt, _ = ref.warp_bwd(v, g[b])
        G.check_grad(gin[b], ri)
        G.check_grad_affine(gaff[b], rt)
    win = [cases[0]]
    gw = upstream_grads([win[0].out_shape], seed=6, device="cuda")
    batch, _, _ = G.batch_for(win, with_image=False, with_label=False)
    ws = A.make_workspace(1)
    gaff = __import__("torch").empty((1, 3, 4), device="cuda")
    A.aug_warp_bwd(batch.d_descs, 1, A.pointer_array(gw, "cuda"), None, gaff, ws)
    st, bad = A.aug_read_device_status(ws)
    assert st == A.AUG_ERR_DESCRIPTOR and bad == 0

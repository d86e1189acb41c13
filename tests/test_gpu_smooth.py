"""GPU parity of the anti-aliasing Gaussian (Sec. 5.A) with the FP64 oracle:
ragged volumes that cross the 64 x 8 x 64 CTA tile in every direction, both
input types, every radius the kernel is built for (and sigma = 0 axes), a
smoothing + downscaling warp chain, sampled points of full-resolution
512 x 512 x 300-600 int16 volumes, and argument errors.

Tolerance, from the arithmetic: each output is three float32 sums of K = 2R+1
products (x, then y, then z) with float32 weights, so
|gpu - oracle| <= (3K + 3) 2^-24 max|E|, E the input extended by the fill."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth.params import AffineSpec
from synth.phantom import make_phantom
from synth.workloads import VolumeCase

import _gpu as G

pytestmark = pytest.mark.gpu


def tol(sigma, img, fill):
    K = 2 * max(ref.gauss_radius(s) for s in sigma) + 1
    m = max(float(np.max(np.abs(img.astype(np.float64)))), abs(fill))
    return (3 * K + 3) * 2.0 ** -24 * m


def run(imgs, sigmas, fill=-1000.0, host=True):
    A = G.aw()
    outs = [torch.full(im.shape, np.nan, dtype=torch.float32, device="cuda") for im in imgs]
    A.aug_smooth(imgs, outs, sigmas, fill)
    torch.cuda.synchronize()
    assert A.aug_smooth_status() == 0
    return [o.cpu().numpy() for o in outs] if host else outs


CASES = [((1, 1, 1), (0.7, 0.7, 0.7)), ((2, 3, 5), (1.0953, 1.0953, 1.0953)),
         ((130, 9, 70), (1.0953, 0.5, 0.0)), ((65, 17, 129), (2.0, 0.3, 1.4)),
         ((70, 40, 64), (0.0, 0.0, 0.0)), ((33, 20, 100), (2.6, 2.6, 2.6)),
         ((64, 8, 64), (0.9, 1.2, 1.9)), ((20, 30, 40), (0.6, 0.6, 0.6)),
         ((10, 11, 12), (0.3, 0.2, 0.1))]


@pytest.mark.parametrize("dtype", ["float32", "int16"])
def test_volumes_match_oracle(dtype):
    imgs, sig, refs = [], [], []
    for n, (shape, sigma) in enumerate(CASES):
        nz, ny, nx = shape
        img, _ = make_phantom((nx, ny, nz), seed=500 + n, dtype=dtype)
        imgs.append(img.cuda().contiguous())
        sig.append(sigma)
    outs = run(imgs, sig)
    for n, (img, sigma, out) in enumerate(zip(imgs, sig, outs)):
        h = img.cpu().numpy()
        exp = ref.smooth(h, sigma, -1000.0)
        err = float(np.max(np.abs(out - exp)))
        assert np.all(np.isfinite(out))
        assert err <= tol(sigma, h, -1000.0), (n, err, tol(sigma, h, -1000.0))


def test_smooth_then_downscaling_warp_matches_oracle_chain():
    A = G.aw()
    img, lab = make_phantom((90, 80, 70), seed=77, dtype="int16")
    u = 0.7
    s = A.aug_antialias_sigma(3.0, u)
    assert abs(s - ref.antialias_sigma(3.0, u)) < 1e-7
    sm = run([img.cuda().contiguous()], [(s, s, s)])[0]
    exp_sm = ref.smooth(img.numpy(), (s, s, s), -1000.0)
    bound = tol((s, s, s), img.numpy(), -1000.0)
    assert np.max(np.abs(sm - exp_sm)) <= bound
    from synth.params import random_affine
    down = 3.0 / u
    T, _ = random_affine(np.random.default_rng(5), (90, 80, 70), (21, 19, 16),
                         AffineSpec(max_shift_vox=3.0, extra_scale=(down, down, down)))
    gpu_case = G.to_device([VolumeCase(image=torch.from_numpy(sm), label=None,
                                       out_shape=(21, 19, 16), T=T)])
    gi, _ = G.run_fwd(gpu_case, seed=3)
    oracle_case = VolumeCase(image=torch.from_numpy(exp_sm.astype(np.float32)), label=None,
                             out_shape=(21, 19, 16), T=T)
    ro, _, _, _ = ref.warp_fwd(oracle_case, 3)
    # The warp's weights add up to 1, so the smoothing bound carries over.
    G.check_image(gi[0], ro, "smoothed + warped", tol=G.IMG_TOL + bound)


def test_full_resolution_volumes_on_sampled_points():
    from synth import workloads
    w = workloads.config4(device="cuda", n_vols=3)
    s = G.aw().aug_antialias_sigma(3.0, 0.7)
    imgs = [v.image for v in w.vols]
    outs = run(imgs, [(s, s, s)] * len(imgs), host=False)
    rng = np.random.default_rng(9)
    for img, out in zip(imgs, outs):
        h = img.cpu().numpy()
        n = h.size
        # corners, faces and random interior points
        nz, ny, nx = h.shape
        q = np.concatenate([rng.integers(0, n, 4000),
                            [0, n - 1, nx - 1, nx * ny - 1, (nz - 1) * nx * ny]])
        exp = ref.smooth_points(h, (s, s, s), -1000.0, q)
        got = out.reshape(-1)[torch.from_numpy(q).cuda()].cpu().numpy()
        err = float(np.max(np.abs(got - exp)))
        assert err <= tol((s, s, s), h, -1000.0), err


def test_argument_errors():
    A = G.aw()
    img = torch.zeros((4, 5, 6), device="cuda")
    out = torch.zeros((4, 5, 6), device="cuda")
    for sig, status in [((3.0, 0.0, 0.0), A.AUG_ERR_UNSUPPORTED),
                        ((-0.5, 0.0, 0.0), A.AUG_ERR_INVALID_ARG),
                        ((float("nan"), 0.0, 0.0), A.AUG_ERR_INVALID_ARG)]:
        with pytest.raises(A.AugError) as e:
            A.aug_smooth([img], [out], [sig])
        assert e.value.status == status
    with pytest.raises(A.AugError) as e:
        A.aug_smooth([img], [img], [(1.0, 1.0, 1.0)])      # in place
    assert e.value.status == A.AUG_ERR_INVALID_ARG


def test_bounded_wait_runs_out_and_is_reported():
    """No tile copy is issued: the block's wait for its first tile runs out
    (after about a second), status 1 is recorded and the block returns; the
    context stays usable and a normal call afterwards reports 0."""
    import time
    A = G.aw()
    img = torch.zeros((8, 16, 64), dtype=torch.int16, device="cuda")   # one 64x16 tile, TMA path
    out = torch.zeros((8, 16, 64), device="cuda")
    assert A.aug_smooth_status() == 0
    t0 = time.time()
    A.aug_test_smooth_wait_timeout([img], [out], [(0.5, 0.5, 0.5)])
    torch.cuda.synchronize()
    assert A.aug_smooth_status() == 1
    assert time.time() - t0 < 60.0
    outs = run([img], [(0.5, 0.5, 0.5)])
    assert np.all(np.isfinite(outs[0]))

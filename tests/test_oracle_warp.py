"""Pins of the oracle's warp and its adjoint against what the mathematics fixes.

Sec. 4 defines the output as I_in(Ax + b) sampled trilinearly (labels: nearest
voxel).  The pins below do not re-run the oracle's own formulas:

* identity / integer translation / signed permutation warps reproduce the
  (shifted, permuted) input exactly, and a permutation followed by its inverse
  round-trips;
* the whole warp equals SciPy's ``ndimage.affine_transform`` (order 1,
  ``grid-constant`` boundary = per-tap fill) and its labels equal order 0;
* trilinear interpolation reproduces an affine intensity ramp exactly, so a
  ramp warped by A equals the ramp evaluated at A o + b;
* a fractional shift along one axis equals ``numpy.interp`` on each row;
* on 8^3 volumes the operator matrix, built column by column from impulses,
  is the linear part of the warp, and the oracle's input gradient is its
  transpose (adjoint identity);
* the affine gradient equals per-voxel central differences (step 1e-4) on
  every voxel whose interpolation cell does not change over the step (there
  the output is exactly linear in each T entry).
"""
import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

from oracle import ref
from synth.params import AffineSpec, random_affine
from synth.phantom import make_phantom
from synth.workloads import VolumeCase


def case(img, lab, out_shape, T, a=1.0, b=0.0, sigma=0.0, fill=-1000.0, noise_id=0):
    return VolumeCase(image=torch.as_tensor(img), label=None if lab is None else torch.as_tensor(lab),
                      out_shape=tuple(out_shape), T=np.asarray(T, np.float32),
                      photo_a=np.float32(a), photo_b=np.float32(b), sigma=np.float32(sigma),
                      fill_image=np.float32(fill), noise_id=noise_id)


def ident(shift=(0, 0, 0)):
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = np.eye(3)
    T[:, 3] = shift
    return T


@pytest.fixture(scope="module")
def phantom():
    img, lab = make_phantom((23, 17, 12), seed=5)
    return img.numpy(), lab.numpy()


@pytest.mark.parametrize("dtype", ["float32", "int16"])
def test_identity_is_exact(dtype):
    img, lab = make_phantom((19, 14, 9), seed=1, dtype=dtype)
    out, olab, tie, nt = ref.warp_fwd(case(img, lab, (19, 14, 9), ident()), seed=0)
    assert np.array_equal(out, img.numpy().astype(np.float64))
    assert np.array_equal(olab, lab.numpy())
    assert nt == 0


def test_integer_translation_is_exact_shift(phantom):
    img, lab = phantom
    nz, ny, nx = img.shape
    d = (3, -2, 1)
    out_shape = (20, 19, 14)
    out, olab, _, _ = ref.warp_fwd(case(img, lab, out_shape, ident(d), fill=-7.0), seed=0)
    pad = 40
    big = np.pad(img.astype(np.float64), pad, constant_values=-7.0)
    bigl = np.pad(lab, pad, constant_values=0)
    onx, ony, onz = out_shape
    sl = (slice(pad + d[2], pad + d[2] + onz), slice(pad + d[1], pad + d[1] + ony),
          slice(pad + d[0], pad + d[0] + onx))
    assert np.array_equal(out, big[sl])
    assert np.array_equal(olab, bigl[sl])


def _signed_perm(rng, n):
    perm = rng.permutation(3)
    sign = rng.choice([-1, 1], 3)
    A = np.zeros((3, 3))
    A[np.arange(3), perm] = sign
    b = np.where(sign < 0, n - 1, 0).astype(np.float64)
    return A, b


def test_signed_permutations_exact_and_round_trip():
    rng = np.random.default_rng(3)
    n = 11
    img, lab = make_phantom((n, n, n), seed=9)
    img, lab = img.numpy(), lab.numpy()
    for _ in range(6):
        A, b = _signed_perm(rng, n)
        T = np.concatenate([A, b[:, None]], 1).astype(np.float32)
        out, olab, _, _ = ref.warp_fwd(case(img, lab, (n, n, n), T), seed=0)
        # Expected by integer index arithmetic: out[o] = in[A o + b].
        k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        o = np.stack([i, j, k], -1).reshape(-1, 3)
        s = (o @ A.T + b).astype(np.int64)
        exp = img[s[:, 2], s[:, 1], s[:, 0]].reshape(n, n, n)
        assert np.array_equal(out, exp.astype(np.float64))
        assert np.array_equal(olab, lab[s[:, 2], s[:, 1], s[:, 0]].reshape(n, n, n))
        # Inverse map: A^-1 (s - b).
        Ai = np.linalg.inv(A)
        Ti = np.concatenate([Ai, (-Ai @ b)[:, None]], 1).astype(np.float32)
        back, backl, _, _ = ref.warp_fwd(case(out.astype(np.float32), olab, (n, n, n), Ti), 0)
        assert np.array_equal(back, img.astype(np.float64))
        assert np.array_equal(backl, lab)


def _scipy_warp(img, T, out_shape, fill, order):
    # SciPy works on array axes (z, y, x): reverse both index orders.
    M = np.asarray(T, np.float64)[::-1, :3][:, ::-1]
    off = np.asarray(T, np.float64)[::-1, 3]
    onx, ony, onz = out_shape
    return ndi.affine_transform(img.astype(np.float64), M, offset=off, output_shape=(onz, ony, onx),
                                order=order, mode="grid-constant", cval=fill, prefilter=False)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_matches_scipy_affine_transform(seed):
    rng = np.random.default_rng(100 + seed)
    in_shape = tuple(int(v) for v in rng.integers(6, 30, 3))
    out_shape = tuple(int(v) for v in rng.integers(5, 28, 3))
    spec = AffineSpec(max_rot_deg=40.0, scale_range=(0.6, 1.7), max_shift_vox=6.0,
                      max_shear=0.3, reflect_prob=(0.3, 0.3, 0.3))
    T, _ = random_affine(rng, in_shape, out_shape, spec)
    dtype = "int16" if seed == 3 else "float32"
    img, lab = make_phantom(in_shape, seed=seed, dtype=dtype)
    img, lab = img.numpy(), lab.numpy()
    a, b = 1.07, -12.5
    out, olab, tie, _ = ref.warp_fwd(case(img, lab, out_shape, T, a=a, b=b, fill=-1000.0), 0)
    exp = np.float64(np.float32(a)) * _scipy_warp(img, T, out_shape, -1000.0, 1) + np.float64(
        np.float32(b))
    assert np.max(np.abs(out - exp)) <= 1e-9 * max(1.0, np.max(np.abs(exp)))
    expl = _scipy_warp(lab, T, out_shape, 0.0, 0).astype(np.uint8)
    keep = tie == 0
    assert keep.mean() > 0.99
    assert np.array_equal(olab[keep], expl[keep])


def test_affine_ramp_is_reproduced_exactly():
    # Trilinear interpolation is exact on affine functions (all 8 taps inside).
    rng = np.random.default_rng(7)
    n = (24, 20, 16)
    coef = np.array([3.0, -2.0, 5.0, 11.0])
    k, j, i = np.meshgrid(*[np.arange(v) for v in n[::-1]], indexing="ij")
    ramp = (coef[0] * i + coef[1] * j + coef[2] * k + coef[3]).astype(np.float32)
    spec = AffineSpec(max_rot_deg=30.0, scale_range=(0.7, 1.2), max_shift_vox=2.0, max_shear=0.2)
    for _ in range(3):
        T, _ = random_affine(rng, n, (12, 10, 9), spec)
        out, _, _, _ = ref.warp_fwd(case(ramp, None, (12, 10, 9), T, fill=0.0), 0)
        kk, jj, ii = np.meshgrid(np.arange(9), np.arange(10), np.arange(12), indexing="ij")
        o = np.stack([ii, jj, kk, np.ones_like(ii)], -1).astype(np.float64)
        s = o @ np.asarray(T, np.float64).T
        inside = np.all((np.floor(s) >= 0) & (np.floor(s) <= np.array(n) - 2), axis=-1)
        assert inside.mean() > 0.5
        exp = s @ coef[:3] + coef[3]
        assert np.max(np.abs(out[inside] - exp[inside])) < 1e-9


def test_fractional_shift_matches_numpy_interp(phantom):
    img, _ = phantom
    nz, ny, nx = img.shape
    dx = 0.375
    T = ident((-2.0 + dx, 0, 0))
    out, _, _, _ = ref.warp_fwd(case(img, None, (nx + 5, ny, nz), T, fill=-5.0), 0)
    xs = np.arange(nx + 5) - 2.0 + dx
    for z in range(nz):
        for y in range(ny):
            row = np.concatenate([[-5.0], img[z, y].astype(np.float64), [-5.0]])
            exp = np.interp(xs, np.arange(-1, nx + 1), row, left=-5.0, right=-5.0)
            assert np.max(np.abs(out[z, y] - exp)) < 1e-9


def _operator(T, n, out_n, fill):
    cols = []
    for m in range(n ** 3):
        e = np.zeros(n ** 3, np.float32)
        e[m] = 1.0
        o, _, _, _ = ref.warp_fwd(case(e.reshape(n, n, n), None, (out_n,) * 3, T, fill=0.0), 0)
        cols.append(o.reshape(-1))
    return np.stack(cols, 1)


def test_brute_force_operator_and_adjoint_8cubed():
    rng = np.random.default_rng(11)
    n = 8
    spec = AffineSpec(max_rot_deg=35.0, scale_range=(0.8, 1.25), max_shift_vox=1.5, max_shear=0.2)
    T, _ = random_affine(rng, (n, n, n), (n, n, n), spec)
    M = _operator(T, n, n, 0.0)
    v = rng.standard_normal(n ** 3).astype(np.float32)
    g = rng.standard_normal(n ** 3).astype(np.float32)
    fill, a = 3.5, 1.3
    out, _, _, _ = ref.warp_fwd(case(v.reshape(n, n, n), None, (n, n, n), T, a=a, fill=fill), 0)
    ones_w = M @ np.ones(n ** 3)
    exp = np.float64(np.float32(a)) * (M @ v.astype(np.float64) + fill * (1.0 - ones_w))
    assert np.max(np.abs(out.reshape(-1) - exp)) < 1e-12 * 100
    gi, gt, _ = ref.warp_bwd(case(v.reshape(n, n, n), None, (n, n, n), T, a=a, fill=fill),
                             g.reshape(n, n, n))
    exp_gi = np.float64(np.float32(a)) * (M.T @ g.astype(np.float64))
    assert np.max(np.abs(gi.reshape(-1) - exp_gi)) < 1e-12 * 100
    # <M v, g> = <v, M^T g>
    lhs = np.dot(M @ v.astype(np.float64), g)
    rhs = np.dot(v.astype(np.float64), gi.reshape(-1)) / np.float64(np.float32(a))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_affine_gradient_matches_central_differences():
    rng = np.random.default_rng(21)
    n_in, n_out = (14, 12, 10), (10, 9, 8)
    img, _ = make_phantom(n_in, seed=4)
    img = img.numpy()
    T, _ = random_affine(rng, n_in, n_out, AffineSpec(max_shift_vox=1.0))
    g = rng.standard_normal(n_out[::-1]).astype(np.float32)
    a = 0.95
    _, gt, dvds = ref.warp_bwd(case(img, None, n_out, T, a=a), g, want_grad_in=False,
                               want_dvds=True)
    kk, jj, ii = np.meshgrid(*[np.arange(v) for v in n_out[::-1]], indexing="ij")
    obar = np.stack([ii, jj, kk, np.ones_like(ii)], -1).astype(np.float64)
    af = np.float64(np.float32(a))
    total_checked = 0
    for r in range(3):
        for c in range(4):
            h = np.float32(1e-4)
            Tp, Tm = T.copy(), T.copy()
            Tp[r, c] = np.float32(T[r, c] + h)
            Tm[r, c] = np.float32(T[r, c] - h)
            heff = (np.float64(Tp[r, c]) - np.float64(Tm[r, c])) / 2.0
            op, _, _, _ = ref.warp_fwd(case(img, None, n_out, Tp, a=a), 0)
            om, _, _, _ = ref.warp_fwd(case(img, None, n_out, Tm, a=a), 0)
            fd = (op - om) / (2.0 * heff)
            sp = obar @ Tp.astype(np.float64).T
            sm = obar @ Tm.astype(np.float64).T
            same = np.all(np.floor(sp) == np.floor(sm), axis=-1)
            assert same.mean() > 0.9
            analytic = af * dvds[..., r] * obar[..., c]
            scale = np.max(np.abs(analytic)) + 1.0
            assert np.max(np.abs(fd[same] - analytic[same])) < 1e-6 * scale
            total_checked += int(same.sum())
            # Summed with g over the voxels that stay in their cell.
            gsum = np.sum(g.astype(np.float64)[same] * fd[same])
            asum = np.sum(g.astype(np.float64)[same] * analytic[same])
            assert abs(gsum - asum) < 1e-6 * (np.sum(np.abs(g[same] * analytic[same])) + 1.0)
            # The reported gradient is the sum over all voxels.
            full = np.sum(g.astype(np.float64) * analytic)
            assert abs(gt[r, c] - full) < 1e-9 * (abs(full) + np.sum(np.abs(g * analytic)))
    assert total_checked > 0

"""The seeded generators: centre invariant of the random affine (Sec. 4:
b = c + d - Ac guarantees Ac + b = c + d) and the phantom recipe."""
import numpy as np

from synth.params import AffineSpec, random_affine
from synth.phantom import make_phantom


def test_centre_invariant():
    rng = np.random.default_rng(0)
    for _ in range(50):
        n_in = rng.integers(8, 600, 3)
        n_out = rng.integers(8, 200, 3)
        spec = AffineSpec(max_rot_deg=30, max_shear=0.2, reflect_prob=(0.5, 0.5, 0.5),
                          extra_scale=tuple(rng.uniform(0.5, 4.5, 3)))
        T, d = random_affine(rng, n_in, n_out, spec)
        c_in, c_out = (n_in - 1) / 2.0, (n_out - 1) / 2.0
        got = T[:, :3].astype(np.float64) @ c_out + T[:, 3]
        assert np.max(np.abs(got - (c_in + d))) < 1e-4 * (1 + np.abs(T).max() * n_out.max())


def test_rotation_part_is_orthogonal_times_scale():
    rng = np.random.default_rng(1)
    T, _ = random_affine(rng, (64, 64, 64), (64, 64, 64), AffineSpec(scale_range=(1.0, 1.0)))
    A = T[:, :3].astype(np.float64)
    assert np.allclose(A.T @ A, np.eye(3), atol=1e-6)


def test_phantom_recipe():
    img, lab = make_phantom((40, 36, 30), seed=3)
    img, lab = img.numpy(), lab.numpy()
    assert img.dtype == np.float32 and lab.dtype == np.uint8
    assert set(np.unique(lab)) <= set(range(6))
    air = img == -1000.0
    assert air.any() and (lab[air] == 0).all()
    assert (lab == 5).any()
    i16, l16 = make_phantom((40, 36, 30), seed=3, dtype="int16")
    assert i16.dtype.is_floating_point is False and int(i16.min()) >= -1024
    assert np.array_equal(l16.numpy(), lab)
    again, _ = make_phantom((40, 36, 30), seed=3)
    assert np.array_equal(again.numpy(), img)

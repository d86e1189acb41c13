"""Pins of the oracle's parameter sampler (Sec. 4):

* the centre property the paper states, A c_out + b = c_in + d;
* zero ranges give the identity plus the centre shift (closed form);
* a pure rotation is orthogonal with determinant +1, a certain reflection
  flips the sign of its axis, a pure scale is diagonal inside its range, a
  pure generic perturbation stays within +-g of the identity;
* angles recovered from pure z rotations are U[-r, r] (KS test) and reach
  both ends; reflection frequencies match their probabilities;
* one uniform is checked against the known-answer-pinned Philox words;
* window draws map lo to 0 and hi to 1; occlusion draws stay in range and
  cover every output slice equally;
* the same (seed, draw, volume) repeats, and a different one differs.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import ref

IN, OUT = (90, 80, 70), (64, 60, 50)


def spec(**kw):
    s = dict(rot_max=(0.0, 0.0, 0.0), scale_min=(1.0, 1.0, 1.0), scale_max=(1.0, 1.0, 1.0),
             reflect_prob=(0.0, 0.0, 0.0), shear_max=0.0, generic_max=0.0,
             extra_scale=(1.0, 1.0, 1.0), shift_max=(0.0, 0.0, 0.0), photo_a=(1.0, 1.0),
             photo_b=(0.0, 0.0), sigma=(0.0, 0.0), window_lo=(-1000.0, -1000.0),
             window_hi=(1000.0, 1000.0), occ_max_frac=0.0)
    s.update(kw)
    return s


FULL = spec(rot_max=(0.3, 0.2, 0.26), scale_min=(0.9, 0.85, 0.9), scale_max=(1.1, 1.2, 1.1),
            reflect_prob=(0.5, 0.3, 0.1), shear_max=0.05, generic_max=0.02,
            extra_scale=(1.0, 1.0, 2.0), shift_max=(10.0, 8.0, 5.0))


def draw(sp, mask=ref.DRAW_AFFINE, seed=7, d=0, vol=0, **kw):
    return ref.sample_params(sp, mask, seed, d, vol, IN, OUT, **kw)


def test_centre_maps_to_displaced_centre():
    c_in = (np.asarray(IN, np.float64) - 1) / 2
    c_out = (np.asarray(OUT, np.float64) - 1) / 2
    for d in range(50):
        r = draw(FULL, d=d, vol=d % 7)
        A64, b32 = r["A"], r["T"][:, 3].astype(np.float64)
        # FP64 matrix with the float32 offset: error is the offset's rounding.
        err = A64 @ c_out + b32 - (c_in + r["d"])
        assert np.all(np.abs(err) <= np.abs(b32) * 2.0 ** -24 + 1e-12)
        assert np.all(np.abs(r["d"]) <= np.asarray([10.0, 8.0, 5.0]))
        # float32 entries are the rounded FP64 matrix
        assert np.array_equal(r["T"][:, :3], A64.astype(np.float32))


def test_zero_ranges_give_identity_plus_centre_shift():
    r = draw(spec(), d=3, vol=2)
    exp = np.zeros((3, 4), np.float32)
    exp[:, :3] = np.eye(3)
    exp[:, 3] = (np.asarray(IN) - np.asarray(OUT)) / 2.0
    assert np.array_equal(r["T"], exp)


def test_rotation_is_orthogonal_and_proper():
    for d in range(20):
        A = draw(spec(rot_max=(0.5, 0.4, 0.3)), d=d)["A"]
        assert np.allclose(A.T @ A, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(A) - 1.0) < 1e-14


def test_certain_reflection_flips_its_axis():
    for axis in range(3):
        p = [0.0, 0.0, 0.0]
        p[axis] = 1.0
        A = draw(spec(reflect_prob=tuple(p)), d=axis)["A"]
        e = np.ones(3)
        e[axis] = -1.0
        assert np.array_equal(A, np.diag(e))


def test_scale_and_generic_stay_in_their_ranges():
    lo, hi = np.asarray([0.8, 0.9, 1.2]), np.asarray([0.9, 1.3, 1.25])
    for d in range(30):
        A = draw(spec(scale_min=tuple(lo), scale_max=tuple(hi), extra_scale=(1.0, 2.0, 0.5)),
                 d=d)["A"]
        assert np.count_nonzero(A - np.diag(np.diag(A))) == 0
        s = np.diag(A) / np.asarray([1.0, 2.0, 0.5])
        assert np.all((s >= lo - 1e-15) & (s <= hi + 1e-15))
        G = draw(spec(generic_max=0.03), d=d)["A"] - np.eye(3)
        assert np.all(np.abs(G) <= 0.03) and np.any(G != 0)


def test_rotation_angles_are_uniform_and_fill_the_range():
    r = 0.4
    ang = np.asarray([math.atan2(draw(spec(rot_max=(0.0, 0.0, r)), d=d)["A"][1, 0],
                                 draw(spec(rot_max=(0.0, 0.0, r)), d=d)["A"][0, 0])
                      for d in range(2000)])
    assert np.all(np.abs(ang) <= r + 1e-15)
    assert ang.min() < -0.99 * r and ang.max() > 0.99 * r
    assert stats.kstest(ang, stats.uniform(loc=-r, scale=2 * r).cdf).pvalue > 1e-3


def test_reflection_frequency_matches_probability():
    n = 4000
    p = (0.5, 0.3, 0.1)
    signs = np.asarray([np.sign(np.diag(draw(spec(reflect_prob=p), d=d, vol=1)["A"]))
                        for d in range(n)])
    freq = np.mean(signs < 0, axis=0)
    se = np.sqrt(np.asarray(p) * (1 - np.asarray(p)) / n)
    assert np.all(np.abs(freq - np.asarray(p)) < 6 * se)


def test_first_uniform_comes_from_the_pinned_philox_words():
    seed, d, vol = 0x1234_5678_9ABC_DEF0, (5 << 32) | 17, 9
    ctr = np.asarray([[0, vol, d & 0xFFFFFFFF, 0x80000000 | (d >> 32)]], np.uint32)
    w = ref.philox(ctr, seed)[0]
    r = 0.25
    A = ref.sample_params(spec(rot_max=(r, 0.0, 0.0)), ref.DRAW_AFFINE, seed, d, vol, IN,
                          OUT)["A"]
    u0 = (int(w[0]) >> 8) * 2.0 ** -24
    g = float(np.float32(r)) * (2 * u0 - 1)     # angle about x from the first uniform
    assert abs(math.atan2(A[2, 1], A[1, 1]) - g) < 1e-15


def test_window_and_photometric_draws():
    sp = spec(window_lo=(-1000.0, -150.0), window_hi=(230.0, 1500.0), sigma=(0.0, 50.0),
              photo_a=(0.9, 1.1), photo_b=(-50.0, 50.0))
    for d in range(40):
        w = draw(sp, mask=ref.DRAW_WINDOW, d=d)
        a, b = np.float64(w["photo_a"]), np.float64(w["photo_b"])
        lo, hi = -b / a, (1 - b) / a
        assert -1000.0 - 1e-3 <= lo <= -150.0 + 1e-3 and 230.0 - 1e-3 <= hi <= 1500.0 + 1e-3
        assert w["flags"] == 1 and 0.0 <= w["sigma"] <= 50.0 * a * (1 + 1e-6)
        p = draw(sp, mask=ref.DRAW_PHOTO, d=d)
        assert 0.9 <= p["photo_a"] <= 1.1 and -50 <= p["photo_b"] <= 50
        assert 0 <= p["sigma"] <= 50 and p["flags"] == 0
        # the intensity draw's sigma is the window's times (hi - lo)
        assert abs(p["sigma"] - w["sigma"] / a) <= 1e-4 * (1 + p["sigma"])


def test_occlusion_draw_ranges_and_slice_coverage():
    onz = OUT[2]
    hits = np.zeros(onz)
    n = 6000
    for d in range(n):
        o = draw(spec(occ_max_frac=0.3), mask=ref.DRAW_OCCLUDE, d=d)
        dmax = 0.3 * onz
        assert o["flags"] == 2 and 0 <= o["occ_dz"] <= dmax and -dmax <= o["occ_z0"] <= onz - 1
        k = np.arange(onz)
        hits += (k >= o["occ_z0"]) & (k <= o["occ_z0"] + o["occ_dz"])
    p = hits / n
    se = np.sqrt(p.mean() * (1 - p.mean()) / n)
    assert np.max(np.abs(p - p.mean())) < 6 * se + 2e-3


def test_groups_not_drawn_are_left_alone_and_draws_repeat():
    T0 = np.arange(12, dtype=np.float32).reshape(3, 4)
    r = draw(FULL, mask=ref.DRAW_OCCLUDE, T=T0, photo=(2.0, 3.0, 4.0), flags=1,
             occ=(0.0, 0.0))
    assert np.array_equal(r["T"], T0) and (r["photo_a"], r["photo_b"], r["sigma"]) == (2, 3, 4)
    assert r["flags"] == 3
    a = draw(FULL, d=11, vol=4)
    assert np.array_equal(a["T"], draw(FULL, d=11, vol=4)["T"])
    for other in (draw(FULL, d=12, vol=4), draw(FULL, d=11, vol=5), draw(FULL, seed=8, d=11, vol=4)):
        assert not np.array_equal(a["T"], other["T"])

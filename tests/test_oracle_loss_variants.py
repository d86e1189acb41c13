"""Pins of the Dice and IOU^m loss variants (Sec. 5.C):

* Dice is 0 for a perfect prediction and equals 1 - 2|p & y| / (|p| + |y|) for
  binary p (set operations);
* the paper's counter-example p = (0, 1), y = (1, 0) violates the triangle
  inequality for Dice (but not for IOU);
* IOU^m and Dice^m equal IOU and Dice for m = 1 and for binary p
  (property 1), differ for fractional p, and are monotone in each p_k
  (property 2);
* every gradient matches FP64 central differences.
"""
import numpy as np
import pytest

from oracle import ref


def one(p, y, kind, m=1.0):
    p = np.asarray(p, np.float32)
    P = np.stack([1.0 - p, p]).astype(np.float32)
    lc, _, g = ref.loss(P, np.asarray(y, np.uint8), 2, kind, m)
    return lc[1], g[1]


def test_dice_perfect_and_binary():
    rng = np.random.default_rng(0)
    for _ in range(30):
        n = int(rng.integers(1, 300))
        p = rng.random(n) < 0.5
        y = rng.random(n) < 0.5
        if not (p.any() or y.any()):
            continue
        l, _ = one(p.astype(np.float32), y, ref.LOSS_DICE)
        assert abs(l - (1 - 2 * np.sum(p & y) / (p.sum() + y.sum()))) < 1e-15
        l0, _ = one(y.astype(np.float32), y, ref.LOSS_DICE)
        assert l0 == 0.0


def test_dice_counterexample_to_triangle_inequality():
    p = np.array([0, 1], bool)
    y = np.array([1, 0], bool)
    u = p | y
    d = lambda a, b, k: one(a.astype(np.float32), b, k)[0]
    assert d(p, y, ref.LOSS_DICE) > d(p, u, ref.LOSS_DICE) + d(y, u, ref.LOSS_DICE)
    assert d(p, y, ref.LOSS_IOU) <= d(p, u, ref.LOSS_IOU) + d(y, u, ref.LOSS_IOU)


@pytest.mark.parametrize("kind", [ref.LOSS_IOU, ref.LOSS_DICE])
def test_power_family_reduces_on_binary_inputs(kind):
    rng = np.random.default_rng(1)
    y = rng.random(200) < 0.3
    p = rng.random(200).astype(np.float32)
    pb = (rng.random(200) < 0.4).astype(np.float32)
    base = one(pb, y, kind)[0]
    binary = np.sum((pb > 0) & y), np.sum(pb > 0), np.sum(y)
    exact = (1 - binary[0] / (binary[1] + binary[2] - binary[0]) if kind == 0
             else 1 - 2 * binary[0] / (binary[1] + binary[2]))
    assert abs(base - exact) < 1e-15
    for m in (0.5, 2.0, 3.5):
        assert abs(one(pb, y, kind, m)[0] - base) < 1e-15
        assert one(p, y, kind, m)[0] != one(p, y, kind)[0]
        _, g = one(p, y, kind, m)
        assert np.all(g[y] <= 0) and np.all(g[~y] >= 0)


@pytest.mark.parametrize("kind,m", [(1, 1.0), (0, 2.0), (0, 1.5), (1, 0.5), (1, 3.0)])
def test_variant_gradients_match_central_differences(kind, m):
    rng = np.random.default_rng(2 + kind)
    n = 40
    y = rng.random(n) < 0.5
    p = (0.05 + 0.9 * rng.random(n)).astype(np.float32)
    _, g = one(p, y, kind, m)
    h = np.float32(2.0 ** -14)
    for k in range(n):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (one(pp, y, kind, m)[0] - one(pm, y, kind, m)[0]) / (np.float64(pp[k]) - np.float64(pm[k]))
        assert abs(fd - g[k]) < 1e-6 * (abs(g[k]) + 1e-3)


def test_loss_kind0_agrees_with_the_iou_routine():
    rng = np.random.default_rng(9)
    C, n = 5, 700
    y = rng.integers(0, C, n).astype(np.uint8)
    p = rng.dirichlet(np.ones(C), n).T.astype(np.float32)
    a = ref.loss(p, y, C, ref.LOSS_IOU)
    b = ref.iou(p, y, C)
    for u, w in zip(a, b):
        assert np.array_equal(u, w)


def test_logits_of_log_probabilities_give_the_probability_loss():
    """softmax(log p) = p when the p of a voxel sum to 1, for every kind."""
    rng = np.random.default_rng(10)
    C, n = 4, 500
    y = rng.integers(0, C, n).astype(np.uint8)
    p = rng.dirichlet(np.ones(C), n).T
    x = np.log(p).astype(np.float32)
    p32 = np.exp(x.astype(np.float64))
    p32 = (p32 / p32.sum(0)).astype(np.float32)
    for kind, m in [(0, 1.0), (1, 1.0), (0, 2.5), (1, 0.7)]:
        lz, sz, _ = ref.loss(x, y, C, kind, m, logits=True)
        lp, sp, _ = ref.loss(p32, y, C, kind, m)
        assert np.max(np.abs(lz - lp)) < 1e-6 and np.max(np.abs(sz - sp)) < 1e-3


@pytest.mark.parametrize("kind,m", [(0, 1.0), (1, 1.0), (0, 3.0), (1, 0.6)])
def test_logit_gradient_is_shift_invariant_and_matches_differences(kind, m):
    """Adding one constant to all class scores of a voxel leaves the softmax
    and so the loss unchanged, hence the gradient sums to 0 over classes;
    each entry matches FP64 central differences of the class-mean loss."""
    rng = np.random.default_rng(11 + kind)
    C, n = 3, 30
    y = rng.integers(0, C, n).astype(np.uint8)
    # Scores on a 2^-12 grid, so that x + 3 is exact in float32.
    x = (np.round(2.0 * rng.standard_normal((C, n)) * 4096) / 4096).astype(np.float32)
    lc, _, g = ref.loss(x, y, C, kind, m, logits=True, grad_scale=1.0 / C)
    assert np.max(np.abs(g.sum(0))) < 1e-15 * max(1.0, np.max(np.abs(g))) * C * 8
    shifted, _, _ = ref.loss(x + np.float32(3.0), y, C, kind, m, logits=True)
    assert np.max(np.abs(shifted - lc)) < 1e-12
    h = np.float32(2.0 ** -10)
    for c in range(C):
        for k in range(0, n, 3):
            xp, xm = x.copy(), x.copy()
            xp[c, k] += h
            xm[c, k] -= h
            fp = ref.loss(xp, y, C, kind, m, logits=True)[0].mean()
            fm = ref.loss(xm, y, C, kind, m, logits=True)[0].mean()
            fd = (fp - fm) / (np.float64(xp[c, k]) - np.float64(xm[c, k]))
            assert abs(fd - g[c, k]) < 1e-6 * (abs(g[c, k]) + 1e-3), (c, k)

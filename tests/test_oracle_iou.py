"""Pins of the oracle's soft IOU loss (Sec. 5.C) against the facts the paper
states and the mathematics fixes:

* p = one-hot(y) (perfect prediction) gives loss 0 and the closed-form
  gradient -1/|y|_1 on the class voxels and 1/|y|_1 elsewhere;
* binary p gives 1 - Jaccard index, computed with set operations;
* false negatives only (p <= y) give eps/N, false positives only (p >= y)
  give eps/(N + eps), with eps = |p - y|_1 and N = |y|_1;
* the loss decreases in p_k where y_k = 1 and increases where y_k = 0;
* the gradient matches FP64 central differences;
* on binary inputs the loss is a metric (triangle inequality);
* an empty class with an empty prediction has loss 0 and zero gradient.
"""
import numpy as np
import pytest

from oracle import ref


def loss1(p, y):
    """Single-class loss through the oracle (class 1 of a 2-class encoding)."""
    p = np.asarray(p, np.float32)
    lab = np.asarray(y, np.uint8)
    P = np.stack([1.0 - p, p]).astype(np.float32)
    lc, sums, grad = ref.iou(P, lab, 2, 1.0)
    return lc[1], grad[1], sums[1]


def test_perfect_prediction_zero_loss_and_closed_form_gradient():
    rng = np.random.default_rng(0)
    C, n = 6, 5000
    y = rng.integers(0, C, n).astype(np.uint8)
    p = np.eye(C, dtype=np.float32)[y].T.copy()
    lc, sums, grad = ref.iou(p, y, C, 1.0)
    assert np.all(lc == 0.0)
    for c in range(C):
        Y = np.sum(y == c)
        assert sums[c, 0] == Y and sums[c, 1] == Y and sums[c, 2] == Y
        exp = np.where(y == c, -1.0 / Y, 1.0 / Y)
        assert np.allclose(grad[c], exp, rtol=1e-15, atol=0)


def test_binary_prediction_is_one_minus_jaccard():
    rng = np.random.default_rng(1)
    for _ in range(20):
        n = int(rng.integers(1, 400))
        p = rng.random(n) < rng.random()
        y = rng.random(n) < rng.random()
        if not (p.any() or y.any()):
            continue
        l, _, _ = loss1(p.astype(np.float32), y)
        jac = np.sum(p & y) / np.sum(p | y)
        assert abs(l - (1.0 - jac)) < 1e-15


def test_false_negative_and_false_positive_closed_forms():
    rng = np.random.default_rng(2)
    n = 3000
    y = (rng.random(n) < 0.3)
    N = y.sum()
    # False negatives: p <= y.
    p = np.where(y, rng.random(n), 0.0).astype(np.float32)
    eps = np.sum(np.abs(p.astype(np.float64) - y))
    l, _, _ = loss1(p, y)
    assert abs(l - eps / N) < 1e-12
    # False positives: p >= y.
    p = np.where(y, 1.0, rng.random(n) * 0.1).astype(np.float32)
    eps = np.sum(np.abs(p.astype(np.float64) - y))
    l, _, _ = loss1(p, y)
    assert abs(l - eps / (N + eps)) < 1e-12


def test_monotone_in_each_probability():
    rng = np.random.default_rng(3)
    y = rng.random(500) < 0.4
    p = rng.random(500).astype(np.float32)
    _, g, _ = loss1(p, y)
    assert np.all(g[y] < 0.0) and np.all(g[~y] > 0.0)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    n = 60
    y = rng.random(n) < 0.5
    p = (0.05 + 0.9 * rng.random(n)).astype(np.float32)
    _, g, _ = loss1(p, y)
    h = np.float32(2.0 ** -12)
    for k in range(n):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (loss1(pp, y)[0] - loss1(pm, y)[0]) / (np.float64(pp[k]) - np.float64(pm[k]))
        assert abs(fd - g[k]) < 1e-7 * (abs(g[k]) + 1e-3)


def test_triangle_inequality_on_binary_inputs():
    rng = np.random.default_rng(5)
    for _ in range(300):
        n = int(rng.integers(1, 12))
        a, b, c = (rng.random((3, n)) < 0.5)
        if not (a.any() and b.any() and c.any()):
            continue
        d = lambda u, v: loss1(u.astype(np.float32), v)[0]
        assert d(a, c) <= d(a, b) + d(b, c) + 1e-15


def test_empty_class_and_empty_prediction():
    y = np.zeros(10, np.uint8)
    p = np.stack([np.ones(10), np.zeros(10)]).astype(np.float32)
    lc, sums, grad = ref.iou(p, y, 2, 1.0)
    assert lc[1] == 0.0 and np.all(grad[1] == 0.0)
    assert lc[0] == 0.0


def test_batch_mean_and_gradient_scale():
    rng = np.random.default_rng(6)
    C, n = 3, 200
    y = rng.integers(0, C, n).astype(np.uint8)
    p = rng.random((C, n)).astype(np.float32)
    l1, _, g1 = ref.iou(p, y, C, 1.0)
    l2, _, g2 = ref.iou(p, y, C, 0.25)
    assert np.array_equal(l1, l2)
    assert np.allclose(g2, 0.25 * g1, rtol=1e-15, atol=0)

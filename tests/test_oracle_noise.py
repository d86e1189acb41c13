"""Pins of the oracle's noise stream (Sec. 4, additive Gaussian noise).

* Philox4x32-10 against the published known-answer vectors (golden file).
* The Box-Muller normals: mean 0, variance 1, kurtosis 3 within 5 standard
  errors over 4M samples, a Kolmogorov-Smirnov test against N(0, 1), and
  ~zero correlation between the paired cos/sin normals, between volumes and
  between seeds.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.replace("->", " ").split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        seed = key[0] | (key[1] << 32)
        got = ref.philox([ctr], seed)[0]
        assert [int(x) for x in got] == want


def test_philox_counter_sensitivity():
    # Flipping any single counter bit changes about half the output bits.
    base = np.zeros((1, 4), np.uint32)
    w0 = ref.philox(base, 123)[0]
    flips = []
    for word in range(4):
        for bit in (0, 7, 31):
            c = base.copy()
            c[0, word] ^= np.uint32(1 << bit)
            w = ref.philox(c, 123)[0]
            flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(w0, w)))
    assert 40 < np.mean(flips) < 88


@pytest.fixture(scope="module")
def normals():
    onx, ony, onz = 200, 100, 200          # 4M voxels, z-quads complete
    q = np.arange(onx * ony * onz, dtype=np.int64)
    return ref.noise(42, 0, onx, ony, q), (onx, ony, onz)


def test_noise_moments(normals):
    z, _ = normals
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 5.0 * np.sqrt(24.0 / n)
    # Box-Muller with u1 >= 2^-24 bounds |z| by sqrt(-2 ln 2^-24) = 5.77.
    assert np.abs(z).max() <= np.sqrt(-2.0 * np.log(2.0 ** -24)) + 1e-12


def test_noise_ks(normals):
    z, _ = normals
    res = stats.kstest(z[::4], "norm")
    assert res.pvalue > 1e-3


def test_noise_pairs_and_streams_uncorrelated(normals):
    z, (onx, ony, onz) = normals
    v = z.reshape(onz // 4, 4, ony, onx)
    n = v[:, 0].size
    lim = 5.0 / np.sqrt(n)
    # cos/sin of the same Box-Muller pair, and the two pairs of one Philox call.
    assert abs(np.corrcoef(v[:, 0].ravel(), v[:, 1].ravel())[0, 1]) < lim
    assert abs(np.corrcoef(v[:, 0].ravel(), v[:, 2].ravel())[0, 1]) < lim
    q = np.arange(200_000, dtype=np.int64)
    a = ref.noise(42, 0, onx, ony, q)
    b = ref.noise(42, 1, onx, ony, q)
    c = ref.noise(43, 0, onx, ony, q)
    lim = 5.0 / np.sqrt(q.size)
    assert abs(np.corrcoef(a, b)[0, 1]) < lim
    assert abs(np.corrcoef(a, c)[0, 1]) < lim
    assert np.array_equal(a, z[: q.size])

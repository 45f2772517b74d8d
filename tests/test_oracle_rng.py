"""Pins for the oracle's normal generator (Algorithm 1 step 4(a))."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import rng


def _kats(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kats(golden_dir)
    assert len(rows) == 3
    for ctr, key, want in rows:
        out = rng.philox4x32(np.array(ctr, dtype=np.uint32).reshape(4, 1),
                             np.array(key, dtype=np.uint32))
        assert [int(x) for x in out[:, 0]] == want


def test_philox_counter_layout():
    seed, level, sample = (7 << 32) | 11, 3, (5 << 32) | 9
    words = rng.philox_words(seed, level, sample, 16)
    for q in range(4):
        ctr = np.array([q, 9, 5, 3], dtype=np.uint32).reshape(4, 1)
        blk = rng.philox4x32(ctr, np.array([11, 7], dtype=np.uint32))[:, 0]
        assert list(words[4 * q: 4 * q + 4]) == list(blk)


def test_streams_differ_by_seed_level_sample():
    a = rng.philox_words(0, 0, 0, 64)
    assert not np.array_equal(a, rng.philox_words(1, 0, 0, 64))
    assert not np.array_equal(a, rng.philox_words(0, 1, 0, 64))
    assert not np.array_equal(a, rng.philox_words(0, 0, 1, 64))
    assert not np.array_equal(a, rng.philox_words(0, 0, 1 << 32, 64))


def test_log64_accuracy_and_special_values():
    x = np.concatenate([np.random.default_rng(0).random(200000) + 2.0 ** -60,
                        [2.0 ** -33, 0.5, 0.70710678, 0.7071067811865476, 1.0 - 2 ** -53, 1.0]])
    want = np.array([math.log(v) for v in x])
    got = rng.log64(x)
    nz = want != 0
    assert np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz])) < 2e-15
    assert rng.log64(np.array([1.0]))[0] == 0.0
    assert rng.log64(np.array([0.5]))[0] == -0.6931471805599453


def test_log32_accuracy():
    x = (np.random.default_rng(1).random(200000) + 2.0 ** -30).astype(np.float32)
    want = np.log(x.astype(np.float64))
    got = rng.log32(x).astype(np.float64)
    nz = np.abs(want) > 1e-3
    assert np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz])) < 5e-7
    assert np.max(np.abs(got - want)) < 1e-7 * 23


def test_sincospi_accuracy():
    t = np.concatenate([np.linspace(0.0, 2.0, 100001), [0.25, 0.5, 0.75, 1.0, 1.5]])
    s, c = rng.sincospi64(t)
    assert np.max(np.abs(s - np.sin(np.pi * t))) < 2e-15
    assert np.max(np.abs(c - np.cos(np.pi * t))) < 2e-15
    assert np.max(np.abs(s * s + c * c - 1.0)) < 4e-16 * 8
    t32 = t.astype(np.float32)
    s, c = rng.sincospi32(t32)
    ref = np.pi * t32.astype(np.float64)
    assert np.max(np.abs(s - np.sin(ref))) < 3e-7
    assert np.max(np.abs(c - np.cos(ref))) < 3e-7


def test_normals_deterministic_and_fp32_close():
    a = rng.normals64(3, 2, 17, 4096)
    b = rng.normals64(3, 2, 17, 4096)
    assert a.view(np.uint64).tolist() == b.view(np.uint64).tolist()
    f = rng.normals32(3, 2, 17, 4096)
    assert f.dtype == np.float32
    assert np.max(np.abs(f.astype(np.float64) - a)) < 5e-6


def test_box_muller_matches_library_trig():
    """The spec's own ln/sin/cos against the library functions: the normals
    differ from a libm Box-Muller only by rounding."""
    w = rng.philox_words(5, 0, 0, 40000).reshape(-1, 4)
    u = (w.astype(np.float64) + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(u[:, 0]))
    z0 = r * np.cos(2 * np.pi * u[:, 1])
    z1 = r * np.sin(2 * np.pi * u[:, 1])
    xi = rng.normals64(5, 0, 0, 40000).reshape(-1, 4)
    assert np.max(np.abs(xi[:, 0] - z0)) < 1e-13
    assert np.max(np.abs(xi[:, 1] - z1)) < 1e-13


@pytest.mark.parametrize("prec", [64, 32])
def test_normal_moments(prec):
    n = 1 << 20
    z = np.concatenate([rng.normals(11, 0, s, n // 4, prec) for s in range(4)]).astype(np.float64)
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0) * se
    # half-normal moments, §2.4 (proof of Theorem 1):
    # E|xi|^(2k) = (2k)!/(k! 2^k), E|xi|^(2k+1) = sqrt(2/pi) 2^k k!
    a = np.abs(z)
    for p in range(1, 7):
        k = p // 2
        exact = (math.factorial(2 * k) / (math.factorial(k) * 2 ** k) if p % 2 == 0
                 else math.sqrt(2 / math.pi) * 2 ** k * math.factorial(k))
        sd = math.sqrt(np.var(a ** p) / n)
        assert abs((a ** p).mean() - exact) < 5 * sd, (p, (a ** p).mean(), exact)
    assert stats.kstest(z[:200000], "norm").pvalue > 1e-4
    # independence of the two outputs of a Box-Muller pair
    assert abs(np.corrcoef(z[0::2][:200000], z[1::2][:200000])[0, 1]) < 5 / math.sqrt(200000)

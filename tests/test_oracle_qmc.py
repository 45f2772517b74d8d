"""Pins of the lattice sampler of the oracle (oracle/qmc.py)."""
import numpy as np
from scipy import special, stats

from oracle import covariance as ocv
from oracle import embedding as oem
from oracle import qmc
from oracle import rng


def test_korobov_vector_and_one_dimensional_projections():
    N, a = 256, 77
    z = qmc.korobov(a, N, 40)
    assert z[0] == 1 and all(z[r] == (a * z[r - 1]) % N for r in range(1, 40))
    assert np.all(z % 2 == 1)            # odd a, N = 2^m: every z_r is a unit mod N
    i = np.arange(N)
    for r in (0, 1, 7, 39):              # each 1D projection is the full grid {k/N}
        pts = np.sort((i * z[r]) % N)
        assert np.array_equal(pts, i)


def test_ranks_order_the_frequencies():
    P = 8
    rk = qmc.ranks(P)
    assert sorted(rk) == list(range(P * P))
    assert rk[0] == 0                               # k = (0, 0) first
    # next: the four wavenumber-1 frequencies (1,0), (7,0), (0,1), (0,7) in index order
    first = sorted(range(P * P), key=lambda j: rk[j])[1:5]
    assert first == [1, 7, 8, 56]
    # then the squared wavenumber 2 (the diagonal neighbours (1,1), (7,1), (1,7),
    # (7,7)) before 4 (the axis frequencies (2,0), (6,0), (0,2), (0,6)); an
    # order by d(k1) + d(k2) would tie them and put j = 2 first
    nxt = sorted(range(P * P), key=lambda j: rk[j])[5:13]
    assert nxt == [9, 15, 57, 63, 2, 6, 16, 48]
    # a decreasing isotropic spectral density: eigenvalues fall along the order
    e = oem.setup_embedding(ocv.MATERN, 1.5, 0.2, 1.0, 8, oem.PAD_DOUBLING)
    lam = e.Lam.reshape(-1)[np.argsort(qmc.ranks(e.P))]
    assert stats.spearmanr(np.arange(lam.size), lam).correlation < -0.9


def test_shifts_are_the_philox_stream_of_their_own_counter():
    d = qmc.shifts(5, 3, 2, 16)
    w = rng.philox_words(5, qmc.SHIFT_LEVEL, (3 << 32) | 2, 16)
    assert np.array_equal(d, (w.astype(np.float64) + 0.5) * 2.0 ** -32)
    assert np.all((d > 0) & (d < 1))
    assert not np.array_equal(d, qmc.shifts(5, 3, 3, 16))
    assert not np.array_equal(d, qmc.shifts(5, 4, 2, 16))
    big = qmc.shifts(1, 0, 0, 4096)
    assert stats.kstest(big, "uniform").pvalue > 1e-3


def test_uniforms_are_exact_and_inside_the_open_interval():
    N = 1 << 20
    zr = np.array([1, 3, N - 1, 12345], dtype=np.int64)
    delta = np.array([0.25, 0.5, 0.75, 0.999], dtype=np.float64)
    for i in (0, 1, 1000, N - 1):
        y = qmc.lattice_uniforms(zr, N, i, delta)
        want = np.array([((i * z) % N) / N + d for z, d in zip(zr, delta)])
        want -= np.floor(want)
        assert np.array_equal(y, want)
        assert np.all((y > 0) & (y < 1))


def test_inverse_normal_is_symmetric_and_matches_ndtri():
    y = np.array([2.0 ** -40, 2.0 ** -7, 0.3125, 0.5, 0.6875, 1 - 2.0 ** -7, 1 - 2.0 ** -40])
    x = qmc.inv_normal(y)
    assert np.allclose(x, special.ndtri(y), rtol=1e-12, atol=1e-12)
    assert np.allclose(qmc.inv_normal(1.0 - y), -x, rtol=1e-12, atol=1e-12)


def test_shifted_lattice_integrates_a_one_dimensional_moment():
    """E[xi] = 0, E[xi^2] = 1: a randomly shifted full lattice in one dimension
    is a shifted equal-weight rule; with 4096 points the unbounded tails of
    Phi^-1 limit the error to O(log N / N)."""
    N = 4096
    for shift in range(4):
        d = qmc.shifts(11, 0, shift, 4)[:1]
        ys = np.array([qmc.lattice_uniforms(np.array([1]), N, i, d)[0] for i in range(N)])
        xi = qmc.inv_normal(ys)
        assert abs(np.mean(xi ** 2) - 1.0) < 1e-2
        assert abs(np.mean(xi)) < 5e-3


def test_lattice_field_has_the_embedding_covariance_on_average():
    """Averaged over random shifts the lattice normals are i.i.d. N(0,1) in
    each coordinate, so the pointwise variance of Z is sum Lambda / s."""
    n = 4
    e = oem.setup_embedding(ocv.MATERN, 0.5, 0.2, 1.0, n, oem.PAD_DOUBLING)
    full = np.ones(e.Lam.shape, dtype=bool)
    vals = []
    for shift in range(200):
        kf, _ = qmc.sample_k_qmc(e, full, None, 16, 5, 3, 0, shift, 7)
        vals.append(np.log(kf))
    z = np.array(vals)
    var = z.var(axis=0, ddof=1).mean()
    assert abs(var - e.Lam.sum() / e.Lam.size) < 0.25 * e.Lam.sum() / e.Lam.size


def test_lattice_points_have_the_character_property():
    """A rank-1 lattice rule with generating vector z averages the character
    exp(2 pi i h.y) over its N points to 1 when h.z = 0 mod N and to 0
    otherwise (the dual-lattice property of lattice rules); a random shift
    Delta only multiplies the average by exp(2 pi i h.Delta).  Checked on the
    oracle's points in a 4-dimensional projection, so a wrong product, modulus
    or shift in lattice_uniforms fails."""
    N, a = 512, 1597
    z = qmc.korobov(a, N, 64)
    coords = np.array([0, 5, 17, 63])
    zr = z[coords]
    rng_ = np.random.default_rng(4)
    delta = rng_.random(coords.size)
    pts0 = np.array([qmc.lattice_uniforms(zr, N, i, np.zeros(coords.size)) for i in range(N)])
    pts = np.array([qmc.lattice_uniforms(zr, N, i, delta) for i in range(N)])
    hs = [rng_.integers(-40, 41, coords.size) for _ in range(200)]
    # a few vectors in the dual lattice: h.z = 0 mod N
    hs += [np.array([N - zr[1], 1, 0, 0]), np.array([zr[2], 0, -1, 0]), np.array([0, 0, 0, N])]
    seen_dual = 0
    for h in hs:
        dual = int(np.dot(h, zr)) % N == 0
        seen_dual += dual
        avg0 = np.mean(np.exp(2j * np.pi * (pts0 @ h)))
        avg = np.mean(np.exp(2j * np.pi * (pts @ h)))
        assert abs(avg0 - (1.0 if dual else 0.0)) < 1e-11
        assert abs(avg - avg0 * np.exp(2j * np.pi * np.dot(h, delta))) < 1e-11
    assert seen_dual >= 3

"""Randomly shifted rank-1 lattice points in place of the normals of
Algorithm 1 step 4(a): the quasi-Monte Carlo sampler that turns the MLMC
estimator of §3.4 into multilevel quasi-Monte Carlo (the paper's outlook, §5).

    y_j = frac( (i z_r(j) mod N) / N + Delta_j ),     xi_j = Phi^{-1}(y_j)

for lattice point i = 0..N-1 (N a power of two), where r(j) is the rank of
grid frequency j = k1 + P k2 in increasing wavenumber d(k1)^2 + d(k2)^2,
d(k) = min(k, P - k), ties by j: the low frequencies, where a decreasing
spectral density puts the large eigenvalues, get the first lattice
dimensions (an exact integer order, so that it cannot depend on the rounding
of the computed eigenvalues, which are equal in symmetric groups), z_r = a^r mod N is
the Korobov generating vector of an odd parameter a, and Delta is a uniform
random shift drawn from the same Philox4x32-10 generator as the Monte Carlo
normals (key = seed, counter = (j/4, shift index, level, 0xFFFFFFFF), word
j mod 4, Delta = (word + 0.5) 2^-32).  Each shift gives an unbiased estimate;
independent shifts give the error estimate.

TEST INFRASTRUCTURE ONLY (see the package header).
"""
import numpy as np
from scipy import special

from . import field
from . import rng

SHIFT_LEVEL = 0xFFFFFFFF


def korobov(a, N, s):
    """z_r = a^r mod N, r = 0..s-1."""
    z = np.empty(s, dtype=np.int64)
    v = 1 % N
    for r in range(s):
        z[r] = v
        v = (v * a) % N
    return z


def ranks(P):
    """rank[j], j = k1 + P k2: position of frequency j in increasing
    d(k1)^2 + d(k2)^2 (ties by j)."""
    k = np.arange(P)
    d = np.minimum(k, P - k)
    key = (d[None, :] ** 2 + d[:, None] ** 2).reshape(-1)     # [k2][k1] -> j
    order = np.argsort(key, kind="stable")
    rk = np.empty(order.size, dtype=np.int64)
    rk[order] = np.arange(order.size)
    return rk


def shifts(seed, level, shift, s):
    """Delta_j, j = 0..s-1 (s a multiple of 4)."""
    w = rng.philox_words(seed, SHIFT_LEVEL, (level << 32) | shift, s)
    return (w.astype(np.float64) + 0.5) * 2.0 ** -32


def lattice_uniforms(zr, N, i, delta):
    """y_j = frac((i z_r(j) mod N)/N + Delta_j): exact in FP64 for N <= 2^32
    (the product i z_r < 2^64 in unsigned 64-bit arithmetic)."""
    a = ((np.uint64(i) * zr.astype(np.uint64)) % np.uint64(N)).astype(np.float64) / N
    y = a + delta
    return y - np.floor(y)


def inv_normal(y):
    """Phi^{-1}(y), evaluated on the smaller tail (symmetric)."""
    return np.where(y < 0.5, special.ndtri(y), -special.ndtri(1.0 - y))


def lattice_normals(Lam, N, a, seed, level, shift, i):
    s = Lam.size
    zr = korobov(a, N, s)[ranks(Lam.shape[0])]
    return inv_normal(lattice_uniforms(zr, N, i, shifts(seed, level, shift, s)))


def sample_k_qmc(emb, mask_f, mask_c, N, a, seed, level, shift, i, naive=None):
    """k_fine and k_coarse of lattice point i of shift `shift` (Algorithm 1
    step 4 with the lattice normals)."""
    xi = lattice_normals(emb.Lam, N, a, seed, level, shift, i)
    return field.k_from_normals(emb, mask_f, mask_c, xi, naive)

"""Circulant embedding set-up: Algorithm 1 steps 1-3 and Algorithm 2 step 4(b).

Grid: (m+1) x (m+1) vertices x_p = p/m on [0,1]^2, ordered x-fastest (§2.1.2).
Embedding: the first column of the block-circulant S is the P x P array
    c[i2, i1] = C_pad(d(i1)/m, d(i2)/m),  d(i) = min(i, P - i),  P = 2(m + J),
(§2.1.2 for J = 0; §2.2 for the padded matrix), with C_pad = C (classical
padding, which evaluates C itself at the padded lags) or C_ext of Eq. (2.7)
(smooth periodisation, l = 1 + J/m).  Arrays are indexed [i2, i1], so the
C-order flattening is the paper's x-fastest lexicographic order.

Eigenvalues, Algorithm 1 step 3: Lambda = sqrt(s) F s with the unitary F of
Eq. (2.6) (exponent +2 pi i), i.e. the unnormalised +i DFT of c, computed here
by a naive separable DFT (two dense matrix products).  Positivity check and
padding loop, step 3(a)-(b).  Smoothing, §2.4 and Algorithm 2 step 4(b).

Readings of the paper taken here (each listed in the design notes):
* positivity tolerance: min Lambda >= -1e-12 max Lambda; entries in
  [-1e-12 max, 0) are set to 0;
* padding search: P doubles (J = P/2 - m) until the check passes, for both
  the classical and the smooth-periodisation extension;
* tau = number of eigenvalues dropped (the smallest); keep = s - tau;
* ties at the cut: if the keep-th and (keep+1)-th largest eigenvalues a >= b
  satisfy a - b <= tie_rel_tol |a|, every Lambda_j <= a + tie_rel_tol |a| is
  dropped, so a tie group is never split; otherwise exactly the keep largest
  are kept.
"""
from dataclasses import dataclass

import numpy as np

from . import covariance as cv

PAD_NONE = 0
PAD_DOUBLING = 1
PAD_SMOOTH = 2

PSD_REL_TOL = 1e-12


def lag_index(P):
    i = np.arange(P)
    return np.minimum(i, P - i)


def first_column(kind, nu, lam, sigma2, m, J, mode):
    """The P x P first column c[i2, i1] of the (padded) embedding matrix S."""
    P = 2 * (m + J)
    t = lag_index(P) / float(m)
    t1 = t[None, :]
    t2 = t[:, None]
    if mode == PAD_SMOOTH:
        ell = 1.0 + J / float(m)
        return cv.c_ext(kind, t1, t2, nu, lam, sigma2, ell)
    return cv.cov(kind, *np.broadcast_arrays(t1, t2), nu, lam, sigma2)


def dft_matrix(P):
    """D[p, q] = exp(+2 pi i p q / P), the unnormalised matrix of Eq. (2.6)."""
    pq = np.outer(np.arange(P), np.arange(P)) % P
    return np.exp(2j * np.pi * pq / P)


def dft2_naive(a):
    """sum_{q1,q2} a[q2, q1] exp(+2 pi i (p1 q1 + p2 q2)/P) by two matrix products."""
    P = a.shape[0]
    D = dft_matrix(P)
    return D @ a @ D.T


NAIVE_DFT_MAX_P = 1024


def eigenvalues(c):
    """Algorithm 1 step 3: Lambda = sqrt(s) F s (complex; the caller checks Im).

    Naive DFT up to P = 1024; above that numpy's FFT serves as the same
    unnormalised +i transform (ifft2 * s), pinned against the naive DFT at
    smaller P by the tests.
    """
    if c.shape[0] <= NAIVE_DFT_MAX_P:
        return dft2_naive(c)
    return np.fft.ifft2(c) * c.size


@dataclass
class Embedding:
    kind: int
    nu: float
    lam: float
    sigma2: float
    m: int
    J: int
    P: int
    mode: int
    Lam: np.ndarray          # P x P, real, clipped at 0
    lambda_min: float        # before clipping
    lambda_max: float
    max_imag: float

    @property
    def s(self):
        return self.P * self.P


class NotPSD(Exception):
    pass


def setup_embedding(kind, nu, lam, sigma2, m, mode=PAD_DOUBLING, J=None, max_P=8192):
    """Algorithm 1 steps 1-3 with the padding loop of step 3(b)."""
    if J is None:
        J = m if mode == PAD_SMOOTH else 0
    while True:
        P = 2 * (m + J)
        c = first_column(kind, nu, lam, sigma2, m, J, mode)
        L = eigenvalues(c)
        lmax = float(L.real.max())
        lmin = float(L.real.min())
        imag = float(np.abs(L.imag).max())
        if lmin >= -PSD_REL_TOL * lmax:
            Lam = L.real.copy()
            Lam[Lam < 0] = 0.0
            return Embedding(kind, nu, lam, sigma2, m, J, P, mode, Lam, lmin, lmax, imag)
        if mode == PAD_NONE or 2 * P > max_P:
            raise NotPSD((P, lmin, lmax))
        J = P - m            # P -> 2P


def smoothing_mask(Lam, keep, tie_rel_tol=1e-10):
    """Algorithm 2 step 4(b): keep the `keep` largest eigenvalues (keep < 0: all).

    Sorts Lambda non-increasingly (the permutation pi of §3.6), zeroes the
    tail, and maps back by pi^-1 -- returned as a boolean mask on the P x P
    grid, with the tie rule in the module docstring.
    """
    flat = Lam.ravel()
    s = flat.size
    if keep < 0 or keep >= s:
        return np.ones(Lam.shape, dtype=bool)
    if keep == 0:
        return np.zeros(Lam.shape, dtype=bool)
    order = np.argsort(-flat, kind="stable")
    a = flat[order[keep - 1]]
    b = flat[order[keep]]
    tol = tie_rel_tol * abs(a)
    if a - b > tol:
        mask = flat >= a
    else:
        mask = flat > a + tol
    return mask.reshape(Lam.shape)


def masked_eigenvalues(Lam, mask):
    return np.where(mask, Lam, 0.0)

"""Three-dimensional circulant embedding and field (§2.1-2.2 in d = 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper writes the method for d = 1, 2 and states that higher dimensions
follow the same pattern; the covariance (Eq. (2.2)-(2.3)), the smooth
periodisation (Eq. (2.7)) and the smoothing theorem are stated for general d.
This module is the d = 3 instance, read as follows:

* grid: (m+1)^3 vertices x_p = p/m on [0,1]^3, ordered x-fastest
  (index i1 + (m+1) i2 + (m+1)^2 i3); arrays are indexed [i3, i2, i1];
* embedding: P = 2(m + J) per direction, s = P^3, first column
      c[i3, i2, i1] = C_pad(d(i1)/m, d(i2)/m, d(i3)/m),  d(i) = min(i, P - i),
  C_pad = C (classical padding) or C_ext of Eq. (2.7) with the sum over
  n in Z^3, the cutoff taken of |x|_inf (l = 1 + J/m, kappa = 2l - 1);
* eigenvalues: the unnormalised +i DFT of c along each of the three axes
  (the three-fold Kronecker product of the one-dimensional Fourier matrix,
  Eq. (2.6)); positivity check, clipping, padding loop and smoothing masks
  as in two dimensions (embedding.py);
* field (Algorithm 1 step 4 in d = 3): w = Lambda~^(1/2) (.) xi, v = F w with
  the unitary three-dimensional F (1/sqrt(s) = P^(-3/2)), u = Re v + Im v
  (the Hartley form), Z = u on the first m+1 indices of each direction,
  k = exp(Z); normal j of a sample is index k1 + P k2 + P^2 k3 of xi;
* coarse field of an MLMC level: the same xi with the coarse mask, read at
  the even vertices (the fine field itself there when the masks agree).
"""
import numpy as np

from . import covariance as cv
from . import embedding as em
from . import rng


def cov3(kind, t1, t2, t3, nu, lam, sigma2):
    """Eq. (2.2) at the Euclidean norm of (t1, t2, t3); Eq. (2.3), p = 1, as a product."""
    t1, t2, t3 = np.broadcast_arrays(*(np.asarray(t, dtype=np.float64) for t in (t1, t2, t3)))
    if kind == cv.MATERN:
        return cv.matern(np.sqrt(t1 * t1 + t2 * t2 + t3 * t3), nu, lam, sigma2)
    if kind == cv.SEP_EXP:
        return sigma2 * np.exp(-(np.abs(t1) + np.abs(t2) + np.abs(t3)) / lam)
    raise ValueError("unknown covariance kind")


def c_ext3(kind, x1, x2, x3, nu, lam, sigma2, ell):
    """Eq. (2.7) in d = 3: sum over n in {-2..2}^3 of (C phi_kappa)(x + 2 l n).

    For |x|_inf <= l every shift that reaches the support |y|_inf <= kappa
    lies in {-2..2}^3 (as in the two-dimensional module).
    """
    kappa = 2.0 * ell - 1.0
    x1, x2, x3 = np.broadcast_arrays(*(np.asarray(t, dtype=np.float64) for t in (x1, x2, x3)))
    total = np.zeros(x1.shape)
    for n1 in range(-2, 3):
        for n2 in range(-2, 3):
            for n3 in range(-2, 3):
                y1 = x1 + 2.0 * ell * n1
                y2 = x2 + 2.0 * ell * n2
                y3 = x3 + 2.0 * ell * n3
                w = cv.cutoff_phi(np.maximum(np.maximum(np.abs(y1), np.abs(y2)), np.abs(y3)),
                                  kappa)
                nz = w > 0
                if np.any(nz):
                    total[nz] += cov3(kind, y1[nz], y2[nz], y3[nz], nu, lam, sigma2) * w[nz]
    return total


def first_column3(kind, nu, lam, sigma2, m, J, mode):
    """The P x P x P first column c[i3, i2, i1] of the padded embedding matrix.

    c depends on the indices only through the lags d(i) in 0..P/2, so C_pad is
    evaluated once per distinct lag triple and spread by indexing.
    """
    P = 2 * (m + J)
    t = np.arange(P // 2 + 1) / float(m)
    t1 = t[None, None, :]
    t2 = t[None, :, None]
    t3 = t[:, None, None]
    if mode == em.PAD_SMOOTH:
        cu = c_ext3(kind, t1, t2, t3, nu, lam, sigma2, 1.0 + J / float(m))
    else:
        cu = cov3(kind, t1, t2, t3, nu, lam, sigma2)
    d = em.lag_index(P)
    return cu[np.ix_(d, d, d)]


NAIVE_DFT_MAX_P = 128


def dft3_naive(a):
    """sum_q a[q3, q2, q1] exp(+2 pi i (p1 q1 + p2 q2 + p3 q3)/P): one dense
    matrix product per axis."""
    P = a.shape[0]
    D = em.dft_matrix(P)
    out = np.einsum("pq,abq->abp", D, a)
    out = np.einsum("pq,aqb->apb", D, out)
    return np.einsum("pq,qab->pab", D, out)


def dft3(a):
    """The same +i sum; numpy's FFT (ifftn * s) above NAIVE_DFT_MAX_P, pinned
    against the naive form at smaller P by the tests."""
    if a.shape[0] <= NAIVE_DFT_MAX_P:
        return dft3_naive(a)
    return np.fft.ifftn(a) * a.size


def setup_embedding3(kind, nu, lam, sigma2, m, mode=em.PAD_DOUBLING, J=None, max_P=512):
    """Algorithm 1 steps 1-3 in d = 3, with the padding loop of step 3(b).

    Returns embedding.Embedding with Lam of shape (P, P, P); its `s` property
    is P^2 there, so callers use Lam.size for s = P^3.
    """
    if J is None:
        J = m if mode == em.PAD_SMOOTH else 0
    while True:
        P = 2 * (m + J)
        L = dft3(first_column3(kind, nu, lam, sigma2, m, J, mode))
        lmax = float(L.real.max())
        lmin = float(L.real.min())
        imag = float(np.abs(L.imag).max())
        if lmin >= -em.PSD_REL_TOL * lmax:
            Lam = L.real.copy()
            Lam[Lam < 0] = 0.0
            return em.Embedding(kind, nu, lam, sigma2, m, J, P, mode, Lam, lmin, lmax, imag)
        if mode == em.PAD_NONE or 2 * P > max_P:
            raise em.NotPSD((P, lmin, lmax))
        J = P - m


def hartley_field3(lam_masked, xi, m):
    """u on the (m+1)^3 grid from masked eigenvalues and xi (length P^3)."""
    P = lam_masked.shape[0]
    w = np.sqrt(lam_masked) * xi.reshape(P, P, P)
    v = dft3(w) / np.sqrt(float(P) ** 3)
    u = v.real + v.imag
    return u[: m + 1, : m + 1, : m + 1]


def k_from_normals3(emb, mask_f, mask_c, xi):
    """Steps 4(b)-(f) in d = 3: k_fine ((m+1)^3) and k_coarse ((m/2+1)^3 or None)."""
    m = emb.m
    kf = np.exp(hartley_field3(em.masked_eigenvalues(emb.Lam, mask_f), xi, m))
    if mask_c is None:
        return kf, None
    if np.array_equal(mask_c, mask_f):
        return kf, kf[::2, ::2, ::2].copy()
    u = hartley_field3(em.masked_eigenvalues(emb.Lam, mask_c), xi, m)
    return kf, np.exp(u[::2, ::2, ::2])


def sample_k3(emb, mask_f, mask_c, seed, level, sample, precision=32):
    """One sample's fields from the Philox normals of (seed, level, sample)."""
    xi = rng.normals(seed, level, sample, emb.P ** 3, precision).astype(np.float64)
    return k_from_normals3(emb, mask_f, mask_c, xi)

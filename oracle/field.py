"""Per-sample field, Algorithm 1 step 4(a)-(f) (Algorithm 2 for the masked case).

    w = Lambda~^(1/2) (.) xi                 step 4(b), read with the square root
                                             that Z = (G Lambda^(1/2) xi)_R of
                                             §2.1.1-2.1.2 requires
    v = F w                                  step 4(c), F unitary, Eq. (2.6), +i
    u = Re v + Im v                          step 4(d), the Hartley form G = Re F + Im F
    Z_l = (u)_R_l, Z_(l-1) = (u)_R_(l-1)     step 4(e), R = first m+1 entries in
                                             each direction (§2.1.2); the coarse
                                             grid is every second vertex
    k = exp(Z)                               step 4(f)

Coarse field (MLMC level l >= 1): one xi in the level-l embedding drives both
fields; the coarse field uses its own mask (keep_coarse largest of the level-l
eigenvalues) and is read at the even vertices.  With identical masks the
coarse field is exactly the fine field at the even vertices.
"""
import numpy as np

from . import embedding as em
from . import rng


def hartley_field(lam_masked, xi, m, naive=None):
    """u restricted to the (m+1) x (m+1) grid, from masked eigenvalues and xi.

    v = F w = (1/sqrt(s)) sum_q w[q] exp(+2 pi i p.q/P); the naive separable
    DFT is used up to P = 512, numpy's ifft2 (the same +i sum divided by s)
    above.
    """
    P = lam_masked.shape[0]
    s = P * P
    w = np.sqrt(lam_masked) * xi.reshape(P, P)
    if naive is None:
        naive = P <= 512
    if naive:
        v = em.dft2_naive(w) / np.sqrt(s)
    else:
        v = np.fft.ifft2(w) * np.sqrt(s)
    u = v.real + v.imag
    return u[: m + 1, : m + 1]


def sample_k(emb, mask_f, mask_c, seed, level, sample, precision=64, naive=None):
    """k_fine ((m+1)^2) and k_coarse ((m/2+1)^2 or None) for one sample.

    precision selects the normal spec (FP64 or FP32 words); all arithmetic
    after the normals is FP64.
    """
    xi = rng.normals(seed, level, sample, emb.P * emb.P, precision).astype(np.float64)
    return k_from_normals(emb, mask_f, mask_c, xi, naive)


def k_from_normals(emb, mask_f, mask_c, xi, naive=None):
    """Steps 4(b)-(f) for given normals xi (length P*P, index k1 + P k2)."""
    P, m = emb.P, emb.m
    Lf = em.masked_eigenvalues(emb.Lam, mask_f)
    Zf = hartley_field(Lf, xi, m, naive)
    kf = np.exp(Zf)
    if mask_c is None:
        return kf, None
    if np.array_equal(mask_c, mask_f):
        kc = kf[::2, ::2].copy()
    else:
        Lc = em.masked_eigenvalues(emb.Lam, mask_c)
        kc = np.exp(hartley_field(Lc, xi, m, naive)[::2, ::2])
    return kf, kc

"""Covariance functions and the smooth periodisation (§2.1 and §2.2).

Matern covariance, Eq. (2.2):
    C(t) = sigma^2 2^(1-nu)/Gamma(nu) (sqrt(2 nu)|t|/lambda)^nu K_nu(sqrt(2 nu)|t|/lambda)
with C(0) = sigma^2.  Separable exponential covariance, Eq. (2.3) with p = 1:
    C(t) = sigma^2 exp(-|t|_1 / lambda).
Smooth periodisation, Eq. (2.7):
    C_ext(x) = sum_{n in Z^d} (C phi_kappa)(x + 2 l n),  phi_kappa(x) = phi(|x|_inf),
with l = 1 + J/m, kappa = 2l - 1 and the cutoff of §2.2
    phi(t) = eta((kappa-|t|)/(kappa-1)) / [eta((kappa-|t|)/(kappa-1)) + eta((|t|-1)/(kappa-1))],
    eta(x) = exp(-1/x) for x > 0, else 0.
"""
import numpy as np
from scipy import special

MATERN = 0
SEP_EXP = 1


def matern(r, nu, lam, sigma2):
    """Eq. (2.2) at Euclidean distance r >= 0 (general nu, via scipy's K_nu)."""
    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * r / lam
    out = np.full(r.shape, float(sigma2))
    pos = z > 0
    zp = z[pos]
    out[pos] = sigma2 * 2.0 ** (1.0 - nu) / special.gamma(nu) * zp ** nu * special.kv(nu, zp)
    return out


def sep_exp(t1, t2, lam, sigma2):
    """Eq. (2.3) with p = 1 for the lag vector (t1, t2)."""
    return sigma2 * np.exp(-(np.abs(t1) + np.abs(t2)) / lam)


def cov(kind, t1, t2, nu, lam, sigma2):
    t1 = np.asarray(t1, dtype=np.float64)
    t2 = np.asarray(t2, dtype=np.float64)
    if kind == MATERN:
        return matern(np.hypot(t1, t2), nu, lam, sigma2)
    if kind == SEP_EXP:
        return sep_exp(t1, t2, lam, sigma2)
    raise ValueError("unknown covariance kind")


def eta(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape)
    pos = x > 0
    out[pos] = np.exp(-1.0 / x[pos])
    return out


def cutoff_phi(t, kappa):
    """The C-infinity cutoff of §2.2: 1 on [-1, 1], 0 outside [-kappa, kappa]."""
    a = np.abs(np.asarray(t, dtype=np.float64))
    e1 = eta((kappa - a) / (kappa - 1.0))
    e2 = eta((a - 1.0) / (kappa - 1.0))
    return e1 / (e1 + e2)


def c_ext(kind, x1, x2, nu, lam, sigma2, ell):
    """Eq. (2.7) in d = 2: the 2l-periodic smooth extension of C.

    The sum over n in Z^2 is taken over n in {-2..2}^2, which contains every
    shift that can reach the support |x + 2 l n|_inf <= kappa = 2l - 1 for
    |x|_inf <= l.
    """
    kappa = 2.0 * ell - 1.0
    x1, x2 = np.broadcast_arrays(np.asarray(x1, dtype=np.float64),
                                 np.asarray(x2, dtype=np.float64))
    total = np.zeros(x1.shape)
    for n1 in range(-2, 3):
        for n2 in range(-2, 3):
            y1 = x1 + 2.0 * ell * n1
            y2 = x2 + 2.0 * ell * n2
            w = cutoff_phi(np.maximum(np.abs(y1), np.abs(y2)), kappa)
            nz = w > 0
            if np.any(nz):
                total[nz] += cov(kind, y1[nz], y2[nz], nu, lam, sigma2) * w[nz]
    return total

"""Pins for the oracle's covariance, embedding, padding and smoothing set-up."""
import math

import numpy as np
import pytest

from oracle import covariance as cv
from oracle import embedding as em
from oracle import field


def _circulant_2d(c):
    """Explicit s x s block-circulant S with first column c (index p1 + P p2)."""
    P = c.shape[0]
    p1, p2 = np.meshgrid(np.arange(P), np.arange(P), indexing="xy")
    p1 = p1.ravel()
    p2 = p2.ravel()
    return c[(p2[:, None] - p2[None, :]) % P, (p1[:, None] - p1[None, :]) % P]


def _hartley_matrix(P):
    """G = Re F + Im F for the unitary 2D F of §2.1.2 (exponent +2 pi i)."""
    p1, p2 = np.meshgrid(np.arange(P), np.arange(P), indexing="xy")
    p1 = p1.ravel()
    p2 = p2.ravel()
    th = 2 * np.pi * (np.outer(p1, p1) + np.outer(p2, p2)) / P
    return (np.cos(th) + np.sin(th)) / P


def _grid_index(m, P):
    j, i = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    return (i + P * j).ravel(), np.stack([i.ravel() / m, j.ravel() / m], axis=1)


def _brute_R(kind, nu, lam, sigma2, m):
    _, X = _grid_index(m, 2 * m)
    d = X[:, None, :] - X[None, :, :]
    return cv.cov(kind, d[..., 0], d[..., 1], nu, lam, sigma2)


def test_matern_closed_forms():
    r = np.linspace(0.0, 2.0, 401)
    lam = 0.27
    z = r / lam
    closed = {
        0.5: np.exp(-z),
        1.5: (1 + math.sqrt(3) * z) * np.exp(-math.sqrt(3) * z),
        2.5: (1 + math.sqrt(5) * z + 5 * z * z / 3) * np.exp(-math.sqrt(5) * z),
    }
    for nu, want in closed.items():
        got = cv.matern(r, nu, lam, 2.0)
        assert np.max(np.abs(got - 2.0 * want)) < 1e-12
    assert cv.matern(np.array([0.0]), 0.8, 0.1, 3.0)[0] == 3.0


def test_cutoff_phi_properties():
    kappa = 3.0
    t = np.linspace(-5, 5, 2001)
    phi = cv.cutoff_phi(t, kappa)
    assert np.all(phi[np.abs(t) <= 1] == 1.0)
    assert np.all(phi[np.abs(t) >= kappa] == 0.0)
    mid = (t >= 1) & (t <= kappa)
    # eta(a)/(eta(a)+eta(b)) with a + b = 1 gives phi(t) + phi(kappa + 1 - t) = 1
    assert np.max(np.abs(phi[mid] + cv.cutoff_phi(kappa + 1 - t[mid], kappa) - 1)) < 1e-15
    assert np.all(np.diff(phi[t >= 0]) <= 0)


@pytest.mark.parametrize("kind,nu", [(cv.MATERN, 0.5), (cv.MATERN, 1.5), (cv.SEP_EXP, 0.0)])
def test_c_ext_equals_c_on_unit_square_periodic_and_even(kind, nu):
    ell = 2.0
    x = np.linspace(0, 1, 21)
    X1, X2 = np.meshgrid(x, x)
    assert np.max(np.abs(cv.c_ext(kind, X1, X2, nu, 0.1, 1.0, ell)
                         - cv.cov(kind, X1, X2, nu, 0.1, 1.0))) < 1e-15
    y = np.linspace(-ell, 0, 17)
    Y1, Y2 = np.meshgrid(y, np.linspace(-0.3, 0.9, 5))
    a = cv.c_ext(kind, Y1, Y2, nu, 0.1, 1.0, ell)
    assert np.max(np.abs(a - cv.c_ext(kind, Y1 + 2 * ell, Y2, nu, 0.1, 1.0, ell))) < 1e-15
    assert np.max(np.abs(a - cv.c_ext(kind, -Y1, -Y2, nu, 0.1, 1.0, ell))) < 1e-15


@pytest.mark.parametrize("m,J", [(4, 4), (6, 2), (8, 3), (16, 16)])
def test_smooth_first_column_is_c_ext_on_the_grid_period(m, J):
    """Under smooth periodisation the embedding is the circulant of C_ext
    sampled on the grid (§2.2): the period of C_ext, 2l, must be the grid's
    period P/m = 2(m + J)/m, so the first column at every raw lag i/m (not
    only the folded lag min(i, P - i)/m) is C_ext there.  A wrong l keeps
    S restricted to R equal to R, so only this catches it."""
    kind, nu, lam, sigma2 = cv.MATERN, 0.5, 0.3, 1.0
    c = em.first_column(kind, nu, lam, sigma2, m, J, em.PAD_SMOOTH)
    P = c.shape[0]
    ell_grid = P / (2.0 * m)
    t = np.arange(P) / m
    T1, T2 = np.meshgrid(t, t)
    want = cv.c_ext(kind, T1, T2, nu, lam, sigma2, ell_grid)
    assert np.max(np.abs(c - want)) < 1e-14


@pytest.mark.parametrize("m,J,mode", [(4, 0, em.PAD_NONE), (4, 4, em.PAD_DOUBLING),
                                      (4, 4, em.PAD_SMOOTH), (6, 2, em.PAD_SMOOTH)])
def test_embedding_identity_against_brute_force(m, J, mode):
    """S = G Lambda G^T (§2.1.1-2.1.2) and S restricted to R = the covariance
    matrix built point by point."""
    kind, nu, lam, sigma2 = cv.MATERN, 1.5, 0.4, 1.3
    c = em.first_column(kind, nu, lam, sigma2, m, J, mode)
    P = c.shape[0]
    L = em.eigenvalues(c)
    assert np.max(np.abs(L.imag)) < 1e-12 * np.max(np.abs(L.real))
    S = _circulant_2d(c)
    G = _hartley_matrix(P)
    assert np.max(np.abs(G @ G.T - np.eye(P * P))) < 1e-13
    assert np.max(np.abs(G @ np.diag(L.real.ravel()) @ G.T - S)) < 1e-12
    idx, _ = _grid_index(m, P)
    R = _brute_R(kind, nu, lam, sigma2, m)
    assert np.max(np.abs(S[np.ix_(idx, idx)] - R)) < 1e-14
    assert abs(L.real.sum() - P * P * sigma2) < 1e-10 * P * P


def test_naive_dft_matches_fft_branch():
    c = em.first_column(cv.MATERN, 0.5, 0.2, 1.0, 16, 16, em.PAD_SMOOTH)
    a = em.dft2_naive(c)
    b = np.fft.ifft2(c) * c.size
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_separable_exponential_positive_and_kronecker():
    """Lemma 2: real positive eigenvalues without padding; Eq. (2.12): the 2D
    eigenvalues are the Kronecker product of the 1D ones (first column
    s^2D = s^1D (x) s^1D / sigma^2)."""
    for m, lam, sigma2 in [(8, 0.3, 1.0), (16, 0.1, 2.0), (32, 0.02, 0.5)]:
        c = em.first_column(cv.SEP_EXP, 0.0, lam, sigma2, m, 0, em.PAD_NONE)
        L = em.eigenvalues(c).real
        assert L.min() > 0
        P = 2 * m
        s1 = sigma2 * np.exp(-em.lag_index(P) / m / lam)
        L1 = (em.dft_matrix(P) @ s1).real
        assert np.max(np.abs(L - np.outer(L1, L1) / sigma2)) < 1e-11 * L.max()
        e = em.setup_embedding(cv.SEP_EXP, 0.0, lam, sigma2, m, em.PAD_NONE)
        assert e.P == 2 * m


def test_classical_padding_doubles_until_psd():
    """The 33 x 33 grid, Matern nu = 0.5, lambda = 0.3: the 64 x 64 embedding
    has negative eigenvalues; doubling gives 128 x 128 with all >= 0."""
    c = em.first_column(cv.MATERN, 0.5, 0.3, 1.0, 32, 0, em.PAD_DOUBLING)
    assert em.eigenvalues(c).real.min() < -1e-6
    e = em.setup_embedding(cv.MATERN, 0.5, 0.3, 1.0, 32, em.PAD_DOUBLING)
    assert (e.P, e.J) == (128, 32)
    assert e.Lam.min() >= 0
    with pytest.raises(em.NotPSD):
        em.setup_embedding(cv.MATERN, 0.5, 0.3, 1.0, 32, em.PAD_NONE)


def test_smooth_periodisation_psd_on_oscillatory_field():
    e = em.setup_embedding(cv.MATERN, 0.5, 0.02, 1.0, 16, em.PAD_SMOOTH)
    assert (e.P, e.J) == (64, 16)
    assert e.lambda_min > 0


def test_mask_keeps_exact_count_and_drops_tie_groups_whole():
    L = np.array([[5.0, 4.0, 4.0 * (1 + 1e-13), 4.0],
                  [3.0, 2.0, 1.0, 0.5]])
    assert em.smoothing_mask(L, -1).all()
    assert em.smoothing_mask(L, 8).all()
    assert em.smoothing_mask(L, 5).sum() == 5          # 3.0 vs 2.0: no tie at cut
    m2 = em.smoothing_mask(L, 2)                        # cut inside the 4-group
    assert m2.sum() == 1 and m2[0, 0]
    assert em.smoothing_mask(L, 4).sum() == 4           # group fully kept
    assert em.smoothing_mask(L, 0).sum() == 0


def test_mask_symmetric_on_real_spectrum():
    e = em.setup_embedding(cv.MATERN, 0.5, 0.3, 1.0, 32, em.PAD_DOUBLING)
    P = e.P
    for keep in (e.s - P, e.s // 4 - P // 2, 1000):
        mk = em.smoothing_mask(e.Lam, keep)
        neg = mk[(-np.arange(P)) % P][:, (-np.arange(P)) % P]
        assert np.array_equal(mk, neg)
        assert np.array_equal(mk, mk.T)
        assert mk.sum() <= keep


def _field_matrix(Lam_masked, m):
    """The linear map xi -> Z of the oracle sampler, column by column."""
    P = Lam_masked.shape[0]
    cols = []
    for j in range(P * P):
        e = np.zeros(P * P)
        e[j] = 1.0
        cols.append(field.hartley_field(Lam_masked, e, m).ravel())
    return np.array(cols).T


def test_sampler_covariance_exact_and_sign():
    """Z = (G Lambda^(1/2) xi)_R has covariance R exactly (§2.1.2); with a
    mask the covariance is (G Lambda~ G^T)_R and the pointwise variance is
    sum(Lambda~)/s; and the transform has the +i sign of Eq. (2.6)."""
    m = 4
    e = em.setup_embedding(cv.MATERN, 0.5, 0.5, 1.0, m, em.PAD_DOUBLING)
    Mz = _field_matrix(e.Lam, m)
    R = _brute_R(cv.MATERN, 0.5, 0.5, 1.0, m)
    assert np.max(np.abs(Mz @ Mz.T - R)) < 1e-13
    mk = em.smoothing_mask(e.Lam, e.s - 3 * e.P)
    Lt = em.masked_eigenvalues(e.Lam, mk)
    Mt = _field_matrix(Lt, m)
    G = _hartley_matrix(e.P)
    idx, _ = _grid_index(m, e.P)
    full = G @ np.diag(Lt.ravel()) @ G.T
    assert np.max(np.abs(Mt @ Mt.T - full[np.ix_(idx, idx)])) < 1e-13
    assert np.max(np.abs(np.diag(Mt @ Mt.T) - Lt.sum() / e.s)) < 1e-13
    # sign: a unit xi at frequency q gives sqrt(Lambda_q/s)(cos th + sin th),
    # th = 2 pi p.q / P; the -i convention would give cos th - sin th.
    P = e.P
    q1, q2 = 1, 2
    xi = np.zeros(P * P)
    xi[q1 + P * q2] = 1.0
    u = field.hartley_field(e.Lam, xi, m)
    j, i = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    th = 2 * np.pi * (i * q1 + j * q2) / P
    want = math.sqrt(e.Lam[q2, q1] / e.s) * (np.cos(th) + np.sin(th))
    assert np.max(np.abs(u - want)) < 1e-14


def test_sampler_naive_and_fft_branches_agree():
    e = em.setup_embedding(cv.MATERN, 1.5, 0.1, 1.0, 16, em.PAD_DOUBLING)
    xi = np.random.default_rng(0).standard_normal(e.s)
    a = field.hartley_field(e.Lam, xi, 16, naive=True)
    b = field.hartley_field(e.Lam, xi, 16, naive=False)
    assert np.max(np.abs(a - b)) < 1e-12


def test_smoothing_illustration_of_section_2_4():
    """The paper's illustration of smoothing (§2.4): separable exponential
    covariance (Eq. (2.3), p = 1), sigma2 = 1, lambda = 0.1 on a 32 x 32 mesh,
    tau = 7s/8 eigenvalues dropped.  Exact second moments of the oracle's
    sampler (its linear map xi -> Z, column by column), no sampling:
    * unsmoothed, the separable covariance needs no padding (Lemma 2) and the
      field has covariance C exactly: variance 1 and lag-h covariance
      exp(-h/lambda) along either axis;
    * smoothed, the pointwise variance is sum(Lambda~)/s at every vertex
      (the mask keeps tie groups whole, so the field stays stationary) and
      the relative increment variance E[(Z(x+h) - Z(x))^2] / E[Z(x)^2] falls
      below the unsmoothed 2 (1 - exp(-h/lambda)): the sample is smoother."""
    m, lam = 32, 0.1
    e = em.setup_embedding(cv.SEP_EXP, 0.5, lam, 1.0, m, em.PAD_NONE)
    assert e.P == 2 * m
    keep = e.s - 7 * e.s // 8
    mk = em.smoothing_mask(e.Lam, keep)
    assert keep - 16 <= mk.sum() <= keep          # a straddling tie group is dropped whole
    Lt = em.masked_eigenvalues(e.Lam, mk)
    rho = math.exp(-(1.0 / m) / lam)
    # a vertex away from the boundary and its two axis neighbours
    i, j = 10, 13
    rows = [i + (m + 1) * j, i + 1 + (m + 1) * j, i + (m + 1) * (j + 1)]
    for L_, smoothed in ((e.Lam, False), (Lt, True)):
        M = _field_matrix(L_, m)[rows]
        C = M @ M.T
        if not smoothed:
            assert abs(C[0, 0] - 1.0) < 1e-12
            assert abs(C[0, 1] - rho) < 1e-12 and abs(C[0, 2] - rho) < 1e-12
            rough = [2 * (C[0, 0] - C[0, 1]) / C[0, 0], 2 * (C[0, 0] - C[0, 2]) / C[0, 0]]
        else:
            assert np.allclose(np.diag(C), Lt.sum() / e.s, rtol=0, atol=1e-12)
            smooth = [2 * (C[0, 0] - C[0, 1]) / C[0, 0], 2 * (C[0, 0] - C[0, 2]) / C[0, 0]]
    assert rough[0] == pytest.approx(2 * (1 - rho), rel=1e-10)
    assert smooth[0] < 0.5 * rough[0] and smooth[1] < 0.5 * rough[1]

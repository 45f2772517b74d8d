"""Pins for the oracle's three-dimensional embedding, field and Darcy solve.

Each check is fixed by the mathematics or by the paper's d-dimensional
definitions, not by re-running the oracle's own formulas: brute-force
matrices on tiny grids, closed-form solutions, conservation and energy
identities, and the Kronecker structure of the separable covariance.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import covariance as cv
from oracle import darcy3d as d3
from oracle import embedding as em
from oracle import field3d as f3
from oracle import rng


# ------------------------------------------------------------------ helpers
def _grid3(m, P):
    """Embedding indices (i1 + P i2 + P^2 i3) and coordinates of the (m+1)^3 grid, x-fastest."""
    k, j, i = np.meshgrid(np.arange(m + 1), np.arange(m + 1), np.arange(m + 1), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    return i + P * j + P * P * k, np.stack([i / m, j / m, k / m], axis=1)


def _brute_R3(kind, nu, lam, sigma2, m):
    """Covariance matrix of the grid, entry by entry, from the covariance function."""
    _, X = _grid3(m, 2 * m)
    d = X[:, None, :] - X[None, :, :]
    if kind == cv.MATERN:
        return cv.matern(np.linalg.norm(d, axis=2), nu, lam, sigma2)
    return sigma2 * np.exp(-np.abs(d).sum(axis=2) / lam)


def _circulant_3d(c):
    P = c.shape[0]
    idx = np.arange(P ** 3)
    i3, r = np.divmod(idx, P * P)
    i2, i1 = np.divmod(r, P)
    return c[(i3[:, None] - i3[None, :]) % P, (i2[:, None] - i2[None, :]) % P,
             (i1[:, None] - i1[None, :]) % P]


def _hartley_matrix3(P):
    """G = Re F + Im F for the unitary three-dimensional F (exponent +2 pi i)."""
    idx = np.arange(P ** 3)
    i3, r = np.divmod(idx, P * P)
    i2, i1 = np.divmod(r, P)
    th = 2 * np.pi * (np.outer(i1, i1) + np.outer(i2, i2) + np.outer(i3, i3)) / P
    return (np.cos(th) + np.sin(th)) / P ** 1.5


def _field_matrix3(lam_masked, m):
    P = lam_masked.shape[0]
    cols = []
    for j in range(P ** 3):
        e = np.zeros(P ** 3)
        e[j] = 1.0
        cols.append(f3.hartley_field3(lam_masked, e, m).ravel())
    return np.array(cols).T


# ------------------------------------------------------------------ covariance
def test_cov3_closed_forms():
    r = np.random.default_rng(1).uniform(-1, 1, size=(3, 200))
    lam, s2 = 0.3, 1.7
    dist = np.sqrt((r ** 2).sum(axis=0))
    got = f3.cov3(cv.MATERN, r[0], r[1], r[2], 0.5, lam, s2)
    assert np.max(np.abs(got - s2 * np.exp(-dist / lam))) < 1e-13
    z = math.sqrt(3.0) * dist / lam
    got = f3.cov3(cv.MATERN, r[0], r[1], r[2], 1.5, lam, s2)
    assert np.max(np.abs(got - s2 * (1 + z) * np.exp(-z))) < 1e-13
    got = f3.cov3(cv.SEP_EXP, r[0], r[1], r[2], 0.0, lam, s2)
    want = s2 * np.exp(-np.abs(r[0]) / lam) * np.exp(-np.abs(r[1]) / lam) * np.exp(-np.abs(r[2]) / lam)
    assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("kind,nu", [(cv.MATERN, 0.5), (cv.MATERN, 2.5), (cv.SEP_EXP, 0.0)])
def test_c_ext3_equals_c_on_unit_cube_periodic_and_even(kind, nu):
    """Eq. (2.7): C_ext = C where |x|_inf <= 1 (the cutoff is 1 and every
    other shift leaves the support), 2l-periodic in each direction, even."""
    ell = 1.5
    g = np.random.default_rng(2)
    x = g.uniform(0, 1, size=(3, 60))
    assert np.max(np.abs(f3.c_ext3(kind, *x, nu, 0.2, 1.0, ell)
                         - f3.cov3(kind, *x, nu, 0.2, 1.0))) < 1e-15
    y = g.uniform(-ell, ell, size=(3, 60))
    a = f3.c_ext3(kind, *y, nu, 0.2, 1.0, ell)
    for ax in range(3):
        ys = y.copy()
        ys[ax] += 2 * ell
        assert np.max(np.abs(a - f3.c_ext3(kind, *ys, nu, 0.2, 1.0, ell))) < 1e-15
    assert np.max(np.abs(a - f3.c_ext3(kind, *(-y), nu, 0.2, 1.0, ell))) < 1e-15


# ------------------------------------------------------------------ embedding
@pytest.mark.parametrize("m,J,mode", [(2, 0, em.PAD_NONE), (2, 2, em.PAD_DOUBLING),
                                      (2, 2, em.PAD_SMOOTH)])
def test_embedding3_identity_against_brute_force(m, J, mode):
    """S = G Lambda G^T with the three-dimensional Hartley matrix, S circulant
    with first column c, and S restricted to the grid = R point by point."""
    kind, nu, lam, s2 = cv.MATERN, 1.5, 0.4, 1.3
    c = f3.first_column3(kind, nu, lam, s2, m, J, mode)
    P = c.shape[0]
    L = f3.dft3(c)
    assert np.max(np.abs(L.imag)) < 1e-12 * np.max(np.abs(L.real))
    S = _circulant_3d(c)
    G = _hartley_matrix3(P)
    assert np.max(np.abs(G @ G.T - np.eye(P ** 3))) < 1e-12
    assert np.max(np.abs(G @ np.diag(L.real.ravel()) @ G.T - S)) < 1e-12
    idx, _ = _grid3(m, P)
    R = _brute_R3(kind, nu, lam, s2, m)
    assert np.max(np.abs(S[np.ix_(idx, idx)] - R)) < 1e-14
    assert abs(L.real.sum() - P ** 3 * s2) < 1e-10 * P ** 3


@pytest.mark.parametrize("m,J", [(2, 2), (4, 1), (4, 4)])
def test_smooth_first_column3_is_c_ext_on_the_grid_period(m, J):
    """As in two dimensions: C_ext's period 2l must be the grid's period P/m,
    so the first column at every raw lag (i1, i2, i3)/m is C_ext there (a
    wrong l keeps S restricted to R equal to R)."""
    kind, nu, lam, sigma2 = cv.MATERN, 0.5, 0.3, 1.0
    c = f3.first_column3(kind, nu, lam, sigma2, m, J, em.PAD_SMOOTH)
    P = c.shape[0]
    t = np.arange(P) / m
    want = f3.c_ext3(kind, t[None, None, :], t[None, :, None], t[:, None, None], nu, lam,
                     sigma2, P / (2.0 * m))
    assert np.max(np.abs(c - want)) < 1e-14


def test_naive_dft3_matches_fft():
    c = f3.first_column3(cv.MATERN, 0.5, 0.2, 1.0, 8, 8, em.PAD_SMOOTH)
    a = f3.dft3_naive(c)
    b = np.fft.ifftn(c) * c.size
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("m,lam,s2", [(4, 0.3, 1.0), (8, 0.1, 2.0)])
def test_separable_exponential_kronecker3(m, lam, s2):
    """The separable covariance's eigenvalues are the threefold Kronecker
    product of the one-dimensional ones, divided by sigma^(2(d-1)) = sigma^4,
    and positive without padding (Lemma 2)."""
    c = f3.first_column3(cv.SEP_EXP, 0.0, lam, s2, m, 0, em.PAD_NONE)
    L = f3.dft3(c).real
    P = 2 * m
    s1 = s2 * np.exp(-em.lag_index(P) / m / lam)
    L1 = (em.dft_matrix(P) @ s1).real
    want = L1[:, None, None] * L1[None, :, None] * L1[None, None, :] / s2 ** 2
    assert np.max(np.abs(L - want)) < 1e-11 * L.max()
    assert L.min() > 0
    assert f3.setup_embedding3(cv.SEP_EXP, 0.0, lam, s2, m, em.PAD_NONE).P == P


def test_padding_loop3():
    """Matern nu = 0.5, lambda = 0.5 on the 9^3 grid: the 16^3 embedding has
    negative eigenvalues; classical padding doubles until the check passes,
    and the smooth periodisation is positive at its default J = m."""
    c = f3.first_column3(cv.MATERN, 0.5, 0.5, 1.0, 8, 0, em.PAD_DOUBLING)
    assert f3.dft3(c).real.min() < -1e-6
    e = f3.setup_embedding3(cv.MATERN, 0.5, 0.5, 1.0, 8, em.PAD_DOUBLING)
    assert e.P > 16 and e.Lam.min() >= 0
    with pytest.raises(em.NotPSD):
        f3.setup_embedding3(cv.MATERN, 0.5, 0.5, 1.0, 8, em.PAD_NONE)
    s = f3.setup_embedding3(cv.MATERN, 0.5, 0.05, 1.0, 8, em.PAD_SMOOTH)
    assert (s.P, s.J) == (32, 8) and s.lambda_min > 0


# ------------------------------------------------------------------ field
def test_sampler3_covariance_exact_and_sign():
    """Z = (G Lambda^(1/2) xi)_R has covariance R exactly; with a mask the
    covariance is (G Lambda~ G^T)_R; and the transform has the +i sign."""
    m = 2
    e = f3.setup_embedding3(cv.MATERN, 0.5, 0.5, 1.0, m, em.PAD_DOUBLING)
    P = e.P
    Mz = _field_matrix3(e.Lam, m)
    R = _brute_R3(cv.MATERN, 0.5, 0.5, 1.0, m)
    assert np.max(np.abs(Mz @ Mz.T - R)) < 1e-13
    mk = em.smoothing_mask(e.Lam, e.Lam.size - 40)
    Lt = em.masked_eigenvalues(e.Lam, mk)
    Mt = _field_matrix3(Lt, m)
    G = _hartley_matrix3(P)
    idx, _ = _grid3(m, P)
    full = G @ np.diag(Lt.ravel()) @ G.T
    assert np.max(np.abs(Mt @ Mt.T - full[np.ix_(idx, idx)])) < 1e-13
    q = (1, 2, 3)
    xi = np.zeros(P ** 3)
    xi[q[0] + P * q[1] + P * P * q[2]] = 1.0
    u = f3.hartley_field3(e.Lam, xi, m)
    k, j, i = np.meshgrid(np.arange(m + 1), np.arange(m + 1), np.arange(m + 1), indexing="ij")
    th = 2 * np.pi * (i * q[0] + j * q[1] + k * q[2]) / P
    want = math.sqrt(e.Lam[q[2], q[1], q[0]] / P ** 3) * (np.cos(th) + np.sin(th))
    assert np.max(np.abs(u - want)) < 1e-14


def test_mask3_symmetric_and_coarse_field():
    """Masks of a real even spectrum are invariant under k -> -k; with equal
    masks the coarse field is the fine field at the even vertices; a distinct
    coarse mask changes it."""
    m = 4
    e = f3.setup_embedding3(cv.MATERN, 0.5, 0.2, 1.0, m, em.PAD_SMOOTH)
    P = e.P
    mk = em.smoothing_mask(e.Lam, e.Lam.size - int(math.isqrt(e.Lam.size)))
    neg = (-np.arange(P)) % P
    assert np.array_equal(mk, mk[neg][:, neg][:, :, neg])
    xi = rng.normals(5, 1, 3, P ** 3, 32).astype(np.float64)
    kf, kc = f3.k_from_normals3(e, mk, mk, xi)
    assert np.array_equal(kc, kf[::2, ::2, ::2])
    full = np.ones_like(mk)
    kf2, kc2 = f3.k_from_normals3(e, full, mk, xi)
    assert np.max(np.abs(kc2 - kf[::2, ::2, ::2])) < 1e-14
    assert np.max(np.abs(kf2 - kf)) > 1e-6


# ------------------------------------------------------------------ Darcy
def _tet_count(m):
    """Tetrahedra per vertex, counted by hand: a vertex is corner a + delta of
    the cell a (delta in {0,1}^3); the Kuhn split puts corners a and a + 1 in
    all six tetrahedra of the cell and every other corner in two."""
    N = np.zeros((m + 1,) * 3)
    for dk, dj, di in itertools.product((0, 1), repeat=3):
        w = 6 if (di, dj, dk) in ((0, 0, 0), (1, 1, 1)) else 2
        N[dk:dk + m, dj:dj + m, di:di + m] += w
    return N


def test_mesh3_volume_counts_and_seven_point_pattern():
    m = 3
    T, K, M, vol = d3._element_matrices(m)
    assert T.shape == (6 * m ** 3, 4)
    assert np.max(np.abs(vol - 1.0 / (6 * m ** 3))) < 1e-15
    counts = np.bincount(T.ravel(), minlength=(m + 1) ** 3)
    assert np.array_equal(counts, _tet_count(m).ravel().astype(int))
    # only axis-parallel edges couple (the Kuhn split's stiffness is seven-point)
    A, F, _ = d3.assemble3(np.exp(np.random.default_rng(3).standard_normal((m + 1,) * 3)), 1.0)
    X = d3.coordinates3(m)
    r, c = A.nonzero()
    off = r != c
    dx = np.abs(X[r[off]] - X[c[off]]) * m
    big = np.abs(np.asarray(A[r[off], c[off]]).ravel()) > 1e-13
    assert np.all(np.isclose(dx[big].sum(axis=1), 1.0))
    assert abs(F.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("m", [2, 4, 8])
def test_constant_k_closed_forms3(m):
    """k = 2: f = 0 gives u = 1 - x (flux k, u(x*) = 8/15, ||u|| = 1/sqrt 3);
    f = 1 gives the one-dimensional parabola at the vertices, flux k + f/2."""
    k = np.full((m + 1,) * 3, 2.0)
    u, (A, F, M) = d3.solve3(k, 0.0)
    x = np.arange(m + 1) / m
    assert np.max(np.abs(u - (1 - x)[None, None, :])) < 1e-12
    q = d3.qois3(u, A, F, M)
    assert abs(q[0] - 2.0) < 1e-11
    assert abs(q[1] - 8.0 / 15.0) < 1e-12
    assert abs(q[2] - math.sqrt(1.0 / 3.0)) < 1e-12
    u, (A, F, M) = d3.solve3(k, 1.0)
    exact = 1 - x + x * (1 - x) / (2 * 2.0)
    assert np.max(np.abs(u - exact[None, None, :])) < 1e-12
    q = d3.qois3(u, A, F, M)
    assert abs(q[0] - (2.0 + 0.5)) < 1e-11
    a = int(np.floor(7 * m / 15))
    t = 7 * m / 15 - a
    assert abs(q[1] - ((1 - t) * exact[a] + t * exact[a + 1])) < 1e-12


def test_layered_k3_flux_is_energy():
    """k independent of x: u = 1 - x solves the discrete problem, and the
    outflow equals the energy sum_T |T| kbar_T = (h^3/24) sum_v N_T(v) k_v."""
    m = 4
    g = np.random.default_rng(4)
    kyz = np.exp(g.standard_normal((m + 1, m + 1)))
    k = np.repeat(kyz[:, :, None], m + 1, axis=2)
    u, (A, F, M) = d3.solve3(k, 0.0)
    x = np.arange(m + 1) / m
    assert np.max(np.abs(u - (1 - x)[None, None, :])) < 1e-12
    want = (_tet_count(m) * k).sum() / (24.0 * m ** 3)
    assert abs(d3.qois3(u, A, F, M)[0] - want) < 1e-12


def test_random_k3_conservation_symmetry_and_solvers():
    import scipy.sparse.linalg as spla
    m = 4
    g = np.random.default_rng(5)
    k = np.exp(0.8 * g.standard_normal((m + 1,) * 3))
    f = 1.3
    u, (A, F, M) = d3.solve3(k, f)
    assert abs(A - A.T).max() < 1e-15
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-13
    q = d3.qois3(u, A, F, M)
    assert abs(q[0] - (d3.inflow3(u, A, F) + f)) < 1e-12
    left, right = d3.dirichlet_nodes3(m)
    free = np.ones(A.shape[0], dtype=bool)
    free[left] = False
    free[right] = False
    Aff = A[free][:, free]
    assert np.linalg.eigvalsh(Aff.toarray()).min() > 0
    rhs = F[free] - A[free][:, left] @ np.ones(left.size)
    x, info = spla.cg(Aff, rhs, rtol=1e-14, maxiter=2000)
    assert info == 0
    assert np.max(np.abs(x - u.ravel()[free])) < 1e-10


def test_point_value3_and_mass_exact_on_linear_functions():
    m = 5
    X = d3.coordinates3(m)
    a, b = 0.3, np.array([1.1, -0.7, 0.45])
    u = (a + X @ b).reshape((m + 1,) * 3)
    _, _, M = d3.assemble3(np.ones((m + 1,) * 3))
    for x in [(d3.X_STAR,) * 3, (0.11, 0.93, 0.52), (1.0, 0.0, 0.5)]:
        assert abs(d3.point_value3(u, x) - (a + np.dot(b, x))) < 1e-13
    # int (a + b.x)^2 over the unit cube
    want = a * a + a * b.sum() + (b ** 2).sum() / 3 + (b[0] * b[1] + b[0] * b[2] + b[1] * b[2]) / 2
    uf = u.ravel()
    assert abs(uf @ (M @ uf) - want) < 1e-13


@pytest.mark.parametrize("m,seed", [(4, 0), (6, 1)])
def test_k_of_x3_outflow_below_the_series_bound(m, seed):
    """k varying along the flow only, f = 0.  Every Kuhn tetrahedron spans one
    x-layer [a, a+1] and has one, two or three of its four vertices on the far
    plane (two permutations each), so its vertex mean of k averages to
    (k_a + k_a+1)/2 over a cell.  The energy of u = x equals both
    sum_T kbar_T |T| and h^2 times the summed conductance of the layer's
    x-edges (only they see a potential difference), so with |T| = h^3/6 and
    6 m^2 tetrahedra per layer that conductance is
    m^2 h^3 (k_a + k_a+1)/2 / h^2 = m (k_a + k_a+1)/2.
    Shorting every y- and z-edge (Rayleigh's monotonicity law) can only raise
    the outflow, so it is at most the series formula
    1 / sum_a h / ((k_a + k_a+1)/2), with equality for constant k."""
    kx = np.exp(np.random.default_rng(seed).standard_normal(m + 1))
    k = np.broadcast_to(kx[None, None, :], (m + 1, m + 1, m + 1)).copy()
    q = d3.solve_qois3(k, 0.0)[0]
    upper = 1.0 / np.sum((1.0 / m) / ((kx[:-1] + kx[1:]) / 2.0))
    assert q <= upper * (1 + 1e-12)
    assert q > 0.9 * upper
    c = 1.7 * np.ones((m + 1, m + 1, m + 1))
    assert abs(d3.solve_qois3(c, 0.0)[0] - 1.7) < 1e-11

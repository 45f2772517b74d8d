"""Darcy problem, P1 finite elements with nodal quadrature (§3.1-3.2, Eq. (3.1)).

    -div(k grad u) = f on D = (0,1)^2,  u = 1 on x1 = 0,  u = 0 on x1 = 1,
    du/dn = 0 on x2 = 0 and x2 = 1.

Discretisation (§3.2: piecewise-linear elements, quadrature that uses k only
at the grid points).  Readings taken where the paper is silent:
* mesh: the (m+1)^2 vertex grid of the field, each cell [a, a+1] x [b, b+1]
  split by its diagonal (a, b)-(a+1, b+1) into
      T1 = {(a,b), (a+1,b), (a+1,b+1)},  T2 = {(a,b), (a,b+1), (a+1,b+1)};
* quadrature: k is replaced on each triangle by the mean of its three vertex
  values (the exact integral of k's P1 interpolant), so
      A_pq = sum_T kbar_T int_T grad phi_p . grad phi_q,
      F_p  = f sum_{T containing p} |T| / 3;
* Dirichlet values are imposed nodally and eliminated.

This module assembles A generically, element by element, from the vertex
coordinates (it does not use the five-point structure the GPU path relies on).

Quantities of interest (§3.1 and §4), index order of `qois`:
  0  outflow through x1 = 1: Q_out = -sum_{p on x1=1} (A u - F)_p, the
     variationally consistent boundary flux of q = -k grad u;
  1  point value u(7/15, 7/15) from the P1 interpolant;
  2  ||u_h||_{L2(D)} = sqrt(u^T M u) with the consistent P1 mass matrix M.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

X_STAR = 7.0 / 15.0


def node(i, j, m):
    return j * (m + 1) + i


def triangles(m):
    """(2 m^2, 3) vertex ids of the triangulation described above."""
    a, b = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    a = a.ravel()
    b = b.ravel()
    t1 = np.stack([node(a, b, m), node(a + 1, b, m), node(a + 1, b + 1, m)], axis=1)
    t2 = np.stack([node(a, b, m), node(a, b + 1, m), node(a + 1, b + 1, m)], axis=1)
    return np.concatenate([t1, t2])


def coordinates(m):
    j, i = np.divmod(np.arange((m + 1) ** 2), m + 1)
    return np.stack([i / m, j / m], axis=1)


def _element_matrices(m):
    """Per-triangle stiffness G G^T |T|, mass |T|/12 (1 + delta), areas."""
    T = triangles(m)
    X = coordinates(m)[T]                     # (nT, 3, 2)
    B = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)   # columns = edges
    det = B[:, 0, 0] * B[:, 1, 1] - B[:, 0, 1] * B[:, 1, 0]
    area = 0.5 * np.abs(det)
    Binv = np.linalg.inv(B)                   # rows = grad of barycentric 1, 2
    g12 = Binv                                # (nT, 2, 2): g12[t, r, :] = grad lambda_{r+1}
    g0 = -g12.sum(axis=1, keepdims=True)
    G = np.concatenate([g0, g12], axis=1)     # (nT, 3, 2)
    K = area[:, None, None] * np.einsum("tad,tbd->tab", G, G)
    M = area[:, None, None] / 12.0 * (np.ones((3, 3)) + np.eye(3))[None]
    return T, K, M, area


def assemble(k, f=0.0):
    """Full (Dirichlet rows included) stiffness A, load F and mass M for k on the grid."""
    k = np.asarray(k, dtype=np.float64)
    m = k.shape[0] - 1
    N = (m + 1) ** 2
    T, K, M, area = _element_matrices(m)
    kbar = k.ravel()[T].mean(axis=1)
    rows = np.repeat(T, 3, axis=1).ravel()
    cols = np.tile(T, (1, 3)).ravel()
    A = sp.coo_matrix(((kbar[:, None, None] * K).ravel(), (rows, cols)), shape=(N, N)).tocsr()
    Mm = sp.coo_matrix((M.ravel(), (rows, cols)), shape=(N, N)).tocsr()
    F = np.zeros(N)
    np.add.at(F, T.ravel(), np.repeat(f * area / 3.0, 3))
    return A, F, Mm


def dirichlet_nodes(m):
    j = np.arange(m + 1)
    return node(0, j, m), node(m, j, m)


def solve(k, f=0.0, dense=None):
    """Nodal solution u ((m+1) x (m+1), [j, i]) and (A, F, M)."""
    k = np.asarray(k, dtype=np.float64)
    m = k.shape[0] - 1
    N = (m + 1) ** 2
    A, F, M = assemble(k, f)
    left, right = dirichlet_nodes(m)
    u = np.zeros(N)
    u[left] = 1.0
    fixed = np.zeros(N, dtype=bool)
    fixed[left] = True
    fixed[right] = True
    free = ~fixed
    rhs = F[free] - A[free][:, fixed] @ u[fixed]
    Aff = A[free][:, free]
    if dense is None:
        dense = N <= 1200
    if dense:
        u[free] = np.linalg.solve(Aff.toarray(), rhs)
    else:
        u[free] = spla.spsolve(Aff.tocsc(), rhs)
    return u.reshape(m + 1, m + 1), (A, F, M)


def point_value(u, x=X_STAR, y=X_STAR):
    """P1 interpolant at (x, y): barycentric coordinates on the containing triangle."""
    m = u.shape[0] - 1
    a = min(int(np.floor(x * m)), m - 1)
    b = min(int(np.floor(y * m)), m - 1)
    X = coordinates(m)
    uf = u.ravel()
    for tri in ([node(a, b, m), node(a + 1, b, m), node(a + 1, b + 1, m)],
                [node(a, b, m), node(a, b + 1, m), node(a + 1, b + 1, m)]):
        P0, P1, P2 = X[tri]
        Bm = np.array([[P1[0] - P0[0], P2[0] - P0[0]], [P1[1] - P0[1], P2[1] - P0[1]]])
        l12 = np.linalg.solve(Bm, np.array([x - P0[0], y - P0[1]]))
        lam = np.array([1.0 - l12.sum(), l12[0], l12[1]])
        if np.all(lam >= -1e-12):
            return float(lam @ uf[tri])
    raise AssertionError("point not located")


def qois(u, A, F, M):
    m = u.shape[0] - 1
    uf = u.ravel()
    r = A @ uf - F
    _, right = dirichlet_nodes(m)
    q_out = -float(r[right].sum())
    q_pt = point_value(u)
    q_l2 = float(np.sqrt(uf @ (M @ uf)))
    return np.array([q_out, q_pt, q_l2])


def inflow(u, A, F):
    """sum over x1 = 0 of (A u - F): the flux entering through x1 = 0."""
    m = u.shape[0] - 1
    left, _ = dirichlet_nodes(m)
    return float((A @ u.ravel() - F)[left].sum())


def solve_qois(k, f=0.0):
    u, (A, F, M) = solve(k, f)
    return qois(u, A, F, M)

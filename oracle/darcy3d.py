"""Darcy problem on the unit cube, P1 elements with nodal quadrature (§3.1-3.2 in d = 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

    -div(k grad u) = f on D = (0,1)^3,  u = 1 on x1 = 0,  u = 0 on x1 = 1,
    du/dn = 0 on the other four faces.

The paper's model problem (Eq. (3.1)) and its P1 discretisation (§3.2) are
written for d <= 2; this is their d = 3 instance, read as follows:
* mesh: the (m+1)^3 vertex grid of the field; each cell a + [0,1]^3 (in grid
  units) is split into the six Kuhn tetrahedra
      T_pi = {a, a + e_pi1, a + e_pi1 + e_pi2, a + e1 + e2 + e3},
  one per permutation pi of the three axes (the two-dimensional mesh, cells
  split by the diagonal (a)-(a + e1 + e2), is the d = 2 case of the same rule);
* quadrature: k is replaced on each tetrahedron by the mean of its four vertex
  values, so A_pq = sum_T kbar_T int_T grad phi_p . grad phi_q and
  F_p = f sum_{T containing p} |T| / 4;
* Dirichlet values imposed nodally and eliminated.

A is assembled element by element from vertex coordinates (no use of the
seven-point structure the GPU path relies on).

Quantities of interest, index order of `qois3` (as in two dimensions):
  0  outflow through x1 = 1: Q_out = -sum_{p on x1=1} (A u - F)_p;
  1  point value u(7/15, 7/15, 7/15) of the P1 interpolant;
  2  ||u_h||_{L2(D)} = sqrt(u^T M u), consistent P1 mass matrix.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

X_STAR = 7.0 / 15.0
PERMS = list(itertools.permutations(range(3)))
UNIT = np.eye(3, dtype=np.int64)


def node3(i, j, k, m):
    return (k * (m + 1) + j) * (m + 1) + i


def tetrahedra(m):
    """(6 m^3, 4) vertex ids of the Kuhn tetrahedra described above."""
    c = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                 axis=-1).reshape(-1, 3)                      # cell corners (i, j, k)
    out = []
    for pi in PERMS:
        v0 = c
        v1 = v0 + UNIT[pi[0]]
        v2 = v1 + UNIT[pi[1]]
        v3 = c + 1
        out.append(np.stack([node3(v[:, 0], v[:, 1], v[:, 2], m) for v in (v0, v1, v2, v3)],
                            axis=1))
    return np.concatenate(out)


def coordinates3(m):
    idx = np.arange((m + 1) ** 3)
    k, r = np.divmod(idx, (m + 1) ** 2)
    j, i = np.divmod(r, m + 1)
    return np.stack([i / m, j / m, k / m], axis=1)


def _element_matrices(m):
    """Per-tetrahedron stiffness |T| G G^T, mass |T|/20 (1 + delta), volumes."""
    T = tetrahedra(m)
    X = coordinates3(m)[T]                                   # (nT, 4, 3)
    B = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    vol = np.abs(np.linalg.det(B)) / 6.0
    g123 = np.linalg.inv(B)                                  # rows = grad lambda_1..3
    g0 = -g123.sum(axis=1, keepdims=True)
    G = np.concatenate([g0, g123], axis=1)                   # (nT, 4, 3)
    K = vol[:, None, None] * np.einsum("tad,tbd->tab", G, G)
    M = vol[:, None, None] / 20.0 * (np.ones((4, 4)) + np.eye(4))[None]
    return T, K, M, vol


def assemble3(k, f=0.0):
    """Full stiffness A, load F and mass M for vertex values k ((m+1)^3, [k, j, i])."""
    k = np.asarray(k, dtype=np.float64)
    m = k.shape[0] - 1
    N = (m + 1) ** 3
    T, K, M, vol = _element_matrices(m)
    kbar = k.ravel()[T].mean(axis=1)
    rows = np.repeat(T, 4, axis=1).ravel()
    cols = np.tile(T, (1, 4)).ravel()
    A = sp.coo_matrix(((kbar[:, None, None] * K).ravel(), (rows, cols)), shape=(N, N)).tocsr()
    Mm = sp.coo_matrix((M.ravel(), (rows, cols)), shape=(N, N)).tocsr()
    F = np.zeros(N)
    np.add.at(F, T.ravel(), np.repeat(f * vol / 4.0, 4))
    return A, F, Mm


def dirichlet_nodes3(m):
    j, k = np.meshgrid(np.arange(m + 1), np.arange(m + 1), indexing="ij")
    return node3(0, j.ravel(), k.ravel(), m), node3(m, j.ravel(), k.ravel(), m)


def solve3(k, f=0.0):
    """Nodal solution u ((m+1)^3, [k, j, i]) and (A, F, M)."""
    k = np.asarray(k, dtype=np.float64)
    m = k.shape[0] - 1
    N = (m + 1) ** 3
    A, F, M = assemble3(k, f)
    left, right = dirichlet_nodes3(m)
    u = np.zeros(N)
    u[left] = 1.0
    fixed = np.zeros(N, dtype=bool)
    fixed[left] = True
    fixed[right] = True
    free = ~fixed
    rhs = F[free] - A[free][:, fixed] @ u[fixed]
    Aff = A[free][:, free]
    if N <= 1500:
        u[free] = np.linalg.solve(Aff.toarray(), rhs)
    else:
        u[free] = spla.spsolve(Aff.tocsc(), rhs)
    return u.reshape(m + 1, m + 1, m + 1), (A, F, M)


def point_value3(u, x=(X_STAR, X_STAR, X_STAR)):
    """P1 interpolant at x: barycentric coordinates on a tetrahedron that contains it."""
    m = u.shape[0] - 1
    a = [min(int(np.floor(t * m)), m - 1) for t in x]
    X = coordinates3(m)
    uf = u.ravel()
    for pi in PERMS:
        v0 = np.array(a)
        v1 = v0 + UNIT[pi[0]]
        v2 = v1 + UNIT[pi[1]]
        v3 = v0 + 1
        ids = [node3(v[0], v[1], v[2], m) for v in (v0, v1, v2, v3)]
        P0 = X[ids[0]]
        Bm = np.stack([X[ids[1]] - P0, X[ids[2]] - P0, X[ids[3]] - P0], axis=1)
        l123 = np.linalg.solve(Bm, np.asarray(x) - P0)
        lam = np.concatenate([[1.0 - l123.sum()], l123])
        if np.all(lam >= -1e-12):
            return float(lam @ uf[ids])
    raise AssertionError("point not located")


def qois3(u, A, F, M):
    m = u.shape[0] - 1
    uf = u.ravel()
    r = A @ uf - F
    _, right = dirichlet_nodes3(m)
    return np.array([-float(r[right].sum()), point_value3(u), float(np.sqrt(uf @ (M @ uf)))])


def inflow3(u, A, F):
    """sum over x1 = 0 of (A u - F): the flux entering through x1 = 0."""
    m = u.shape[0] - 1
    left, _ = dirichlet_nodes3(m)
    return float((A @ u.ravel() - F)[left].sum())


def solve_qois3(k, f=0.0):
    u, (A, F, M) = solve3(k, f)
    return qois3(u, A, F, M)

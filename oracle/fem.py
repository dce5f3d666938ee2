"""P1 finite elements for -div(kappa grad p) = f on (0,1)^2, p = 0 on the boundary (oracle).

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle; never imported by the
product library.

Follows Sec. 5 (zero-boundary examples): piecewise-linear continuous elements on
a uniform mesh of 2*N^2 triangles (N = 1/h). Each square cell (i, j) is split
by the diagonal (i,j)-(i+1,j+1) (the paper does not state the orientation).
kappa is piecewise constant, one value per triangle. The stiffness matrix is
assembled element by element with the generic P1 formula
    A_T[a, b] = kappa_T * area_T * grad(lambda_a) . grad(lambda_b)
(lambda the barycentric coordinates); the load is b_i = integral of f*phi_i,
computed with the edge-midpoint rule (exact for f constant). Dirichlet nodes
are eliminated and the interior system is solved by a sparse direct
factorisation (scipy SuperLU), so the only error is FP64 rounding.
"""
import functools

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def node_index(N, i, j):
    return j * (N + 1) + i


@functools.lru_cache(maxsize=16)
def mesh(N):
    """Node coordinates ((N+1)^2, 2) and triangles (2N^2, 3), element order e = 2*(j*N+i)+t."""
    h = 1.0 / N
    xs = np.arange(N + 1) * h
    X, Y = np.meshgrid(xs, xs)          # X[j, i] = i*h, Y[j, i] = j*h
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    J, I = np.meshgrid(np.arange(N), np.arange(N), indexing='ij')   # cell (i, j), row-major in j
    v00 = (J * (N + 1) + I).ravel()
    v10 = v00 + 1
    v01 = v00 + (N + 1)
    v11 = v01 + 1
    tris = np.empty((2 * N * N, 3), dtype=np.int64)
    tris[0::2] = np.stack([v00, v10, v11], axis=1)    # lower triangle of cell (i, j)
    tris[1::2] = np.stack([v00, v11, v01], axis=1)    # upper triangle
    return nodes, tris


def _barycentric_gradients(P):
    """P: (3, 2) vertex coordinates -> (grads (3, 2), area)."""
    M = np.array([[1.0, 1.0, 1.0],
                  [P[0, 0], P[1, 0], P[2, 0]],
                  [P[0, 1], P[1, 1], P[2, 1]]])
    Minv = np.linalg.inv(M)              # lambda = Minv @ [1, x, y]
    grads = Minv[:, 1:3]
    area = 0.5 * abs(np.linalg.det(M))
    return grads, area


@functools.lru_cache(maxsize=16)
def _unit_elements(N):
    """Per-triangle area * grad(lambda) grad(lambda)^T (kappa = 1), shape (2N^2, 3, 3).

    The same generic formula as _barycentric_gradients, applied to all triangles at once.
    """
    nodes, tris = mesh(N)
    P = nodes[tris]                                   # (E, 3 vertices, 2)
    M = np.ones((tris.shape[0], 3, 3))
    M[:, 1, :] = P[:, :, 0]
    M[:, 2, :] = P[:, :, 1]
    Minv = np.linalg.inv(M)
    G = Minv[:, :, 1:3]                               # (E, 3, 2) barycentric gradients
    area = 0.5 * np.abs(np.linalg.det(M))
    return area[:, None, None] * np.einsum('eaq,ebq->eab', G, G)


def assemble(N, kappa):
    """Global stiffness matrix (all (N+1)^2 nodes, CSR) for per-triangle kappa.

    Element by element: A = sum_T kappa_T * area_T * G_T G_T^T scattered to the
    triangle's three vertices.
    """
    nodes, tris = mesh(N)
    kappa = np.asarray(kappa, dtype=np.float64)
    assert kappa.shape == (tris.shape[0],)
    Ke = kappa[:, None, None] * _unit_elements(N)
    rows = np.repeat(tris, 3, axis=1).ravel()      # tri[a] for (a, b) row-major
    cols = np.tile(tris, (1, 3)).ravel()           # tri[b]
    n = nodes.shape[0]
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def _areas(N):
    nodes, tris = mesh(N)
    P = nodes[tris]
    d1 = P[:, 1] - P[:, 0]
    d2 = P[:, 2] - P[:, 0]
    return tris, 0.5 * np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])


def load_vector(N, f=None):
    """b_i = integral of f*phi_i; f=None means f == 1. Edge-midpoint quadrature per triangle."""
    nodes, tris = mesh(N)
    b = np.zeros(nodes.shape[0])
    if f is None:
        _, area = _areas(N)
        for a in range(3):
            np.add.at(b, tris[:, a], area / 3.0)
        return b
    for tri in tris:
        P = nodes[tri]
        _, area = _barycentric_gradients(P)
        # midpoints m_01, m_12, m_20; phi_a(m) = 1/2 on the two edges touching a, 0 otherwise
        mids = [(P[0] + P[1]) / 2, (P[1] + P[2]) / 2, (P[2] + P[0]) / 2]
        fm = [f(m[0], m[1]) for m in mids]
        touching = {0: (0, 2), 1: (0, 1), 2: (1, 2)}
        for a in range(3):
            b[tri[a]] += area / 3.0 * sum(0.5 * fm[q] for q in touching[a])
    return b


def nine_sources(x, y):
    """Source term of Example 5.1 (Sec. 5): nine smoothed point sources, the products of 1-D
    Gaussian densities N(x1; 0.25 n, 0.001) N(x2; 0.25 m, 0.001), n, m = 1..3."""
    var = 0.001
    norm = 1.0 / math.sqrt(2.0 * math.pi * var)
    gx = sum(norm * math.exp(-(x - 0.25 * n) ** 2 / (2.0 * var)) for n in (1, 2, 3))
    gy = sum(norm * math.exp(-(y - 0.25 * m) ** 2 / (2.0 * var)) for m in (1, 2, 3))
    return gx * gy


def interior_nodes(N):
    J, I = np.meshgrid(np.arange(1, N), np.arange(1, N), indexing='ij')
    return (J * (N + 1) + I).ravel()


def solve(N, kappa, f=None, A=None):
    """Nodal P1 solution on all (N+1)^2 nodes (zeros on the boundary)."""
    if A is None:
        A = assemble(N, kappa)
    b = load_vector(N, f)
    I = interior_nodes(N)
    Aii = A[I][:, I].tocsc()
    p = np.zeros(A.shape[0])
    p[I] = spla.spsolve(Aii, b[I])
    return p


def solve_flow_cell(N, kappa, A=None):
    """Nodal P1 solution of the flow cell of Example 5.3 (Sec. 5): -div(kappa grad p) = 0 with
    p = 0 on x = 0, p = 1 on x = 1 and no flow (homogeneous Neumann) on y = 0 and y = 1. The
    unknowns are the nodes with 0 < x < 1, boundary rows included; the Dirichlet values enter the
    right-hand side as -A_UD p_D."""
    if A is None:
        A = assemble(N, kappa)
    nodes = np.arange((N + 1) ** 2)
    i = nodes % (N + 1)
    U = nodes[(i > 0) & (i < N)]
    D = nodes[(i == 0) | (i == N)]
    pD = np.where(i[D] == N, 1.0, 0.0)
    A = A.tocsr()
    p = np.zeros((N + 1) ** 2)
    p[D] = pD
    p[U] = spla.spsolve(A[U][:, U].tocsc(), -(A[U][:, D] @ pD))
    return p


def observation_operator(N, obs_xy):
    """Sparse (n_obs, (N+1)^2) matrix of P1 interpolation weights at the points obs_xy.

    A point is located in cell (floor(x/h), floor(y/h)) (clamped to the mesh); it
    lies in the lower triangle when its local offset satisfies dx >= dy. A point on
    an edge gets the same value from either neighbour (P1 continuity).
    """
    nodes, tris = mesh(N)
    h = 1.0 / N
    obs_xy = np.asarray(obs_xy, dtype=np.float64)
    rows, cols, vals = [], [], []
    for r, (x, y) in enumerate(obs_xy):
        i = min(max(int(np.floor(x / h)), 0), N - 1)
        j = min(max(int(np.floor(y / h)), 0), N - 1)
        t = 0 if (x - i * h) >= (y - j * h) else 1
        tri = tris[2 * (j * N + i) + t]
        P = nodes[tri]
        M = np.array([[1.0, 1.0, 1.0], [P[0, 0], P[1, 0], P[2, 0]], [P[0, 1], P[1, 1], P[2, 1]]])
        lam = np.linalg.solve(M, np.array([1.0, x, y]))
        for a in range(3):
            rows.append(r)
            cols.append(tri[a])
            vals.append(lam[a])
    return sp.coo_matrix((vals, (rows, cols)), shape=(obs_xy.shape[0], nodes.shape[0])).tocsr()

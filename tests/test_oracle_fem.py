"""Pins of the oracle's P1 FEM against closed forms and invariants (Sec. 5 forward problem)."""
import math

import numpy as np
import pytest

from oracle import fem


def _kappa_at_centroids(N, fn):
    h = 1.0 / N
    k = np.empty(2 * N * N)
    for j in range(N):
        for i in range(N):
            e = 2 * (j * N + i)
            k[e] = fn((i + 2 / 3) * h, (j + 1 / 3) * h)
            k[e + 1] = fn((i + 1 / 3) * h, (j + 2 / 3) * h)
    return k


def test_manufactured_solution_second_order():
    """p = sin(pi x) sin(pi y), kappa = exp(0.5 sin(2 pi x) cos(pi y)): nodal max error falls ~4x per halving."""
    pi = math.pi
    kap = lambda x, y: math.exp(0.5 * math.sin(2 * pi * x) * math.cos(pi * y))

    def f(x, y):
        k = kap(x, y)
        ux = 0.5 * 2 * pi * math.cos(2 * pi * x) * math.cos(pi * y)      # d(log kappa)/dx
        uy = -0.5 * pi * math.sin(2 * pi * x) * math.sin(pi * y)         # d(log kappa)/dy
        px = pi * math.cos(pi * x) * math.sin(pi * y)
        py = pi * math.sin(pi * x) * math.cos(pi * y)
        lap = -2 * pi * pi * math.sin(pi * x) * math.sin(pi * y)
        return -k * (ux * px + uy * py + lap)

    errs = []
    for N in (8, 16, 32, 64):
        nodes, _ = fem.mesh(N)
        p = fem.solve(N, _kappa_at_centroids(N, kap), f)
        exact = np.sin(pi * nodes[:, 0]) * np.sin(pi * nodes[:, 1])
        errs.append(np.abs(p - exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.7 < r < 2.4 for r in rates), (errs, rates)


def torsion_centre(terms=400):
    s = 0.0
    for m in range(1, terms, 2):
        for n in range(1, terms, 2):
            s += 16.0 / (math.pi ** 4 * m * n * (m * m + n * n)) * math.sin(m * math.pi / 2) * math.sin(n * math.pi / 2)
    return s


def test_torsion_problem_centre_value():
    """kappa = 1, f = 1: centre value converges at O(h^2) to the double Fourier series (~0.07367)."""
    ref = torsion_centre()
    assert ref == pytest.approx(0.0736713, abs=2e-7)
    errs = []
    for N in (8, 16, 32, 64):
        p = fem.solve(N, np.ones(2 * N * N))
        errs.append(abs(p[fem.node_index(N, N // 2, N // 2)] - ref))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.8 < r < 2.2 for r in rates), (errs, rates)


def test_constant_kappa_scaling():
    N = 16
    k = np.random.default_rng(0).uniform(0.2, 5.0, 2 * N * N)
    p1 = fem.solve(N, k)
    p3 = fem.solve(N, 3.0 * k)
    assert np.allclose(p3 * 3.0, p1, rtol=1e-13, atol=0)


def test_reflection_symmetry():
    """The mesh maps to itself under x <-> y (lower <-> upper triangles): symmetric kappa gives p(x,y) = p(y,x)."""
    N = 16
    rng = np.random.default_rng(1)
    k = np.empty(2 * N * N)
    for j in range(N):
        for i in range(N):
            if i <= j:
                v_low, v_up = rng.uniform(0.3, 3.0, 2)
                k[2 * (j * N + i)] = v_low            # lower of (i, j)
                k[2 * (i * N + j) + 1] = v_low        # upper of (j, i) is its mirror image
                if i != j:
                    k[2 * (j * N + i) + 1] = v_up
                    k[2 * (i * N + j)] = v_up
    p = fem.solve(N, k).reshape(N + 1, N + 1)
    assert np.allclose(p, p.T, rtol=1e-12, atol=1e-16)


def test_element_assembly_is_five_point_stencil():
    """Diagonal-edge couplings vanish; edge (i,j)-(i+1,j) has weight (kappa_low(i,j) + kappa_up(i,j-1))/2."""
    N = 6
    k = np.random.default_rng(2).uniform(0.5, 2.0, 2 * N * N)
    A = fem.assemble(N, k).toarray()
    low = lambda i, j: k[2 * (j * N + i)] if (0 <= i < N and 0 <= j < N) else 0.0
    up = lambda i, j: k[2 * (j * N + i) + 1] if (0 <= i < N and 0 <= j < N) else 0.0
    n = (N + 1) ** 2
    B = np.zeros((n, n))
    for j in range(N + 1):
        for i in range(N + 1):
            a = fem.node_index(N, i, j)
            if i < N:   # horizontal edge to (i+1, j)
                w = 0.5 * (low(i, j) + up(i, j - 1))
                b = fem.node_index(N, i + 1, j)
                B[a, b] -= w; B[b, a] -= w; B[a, a] += w; B[b, b] += w
            if j < N:   # vertical edge to (i, j+1)
                w = 0.5 * (low(i - 1, j) + up(i, j))
                b = fem.node_index(N, i, j + 1)
                B[a, b] -= w; B[b, a] -= w; B[a, a] += w; B[b, b] += w
    assert np.abs(A - B).max() < 1e-14
    I = fem.interior_nodes(N)
    assert np.linalg.eigvalsh(A[np.ix_(I, I)]).min() > 0


def test_load_vector_constant_f():
    N = 8
    b = fem.load_vector(N)
    I = fem.interior_nodes(N)
    assert np.allclose(b[I], 1.0 / N ** 2, rtol=1e-14)
    assert b.sum() == pytest.approx(1.0, rel=1e-14)


def test_observation_operator():
    # at h = 1/8 the 7 x 7 grid (i/8, j/8) is exactly the interior nodes
    N = 8
    pts = np.array([((i + 1) / 8, (j + 1) / 8) for j in range(7) for i in range(7)])
    O = fem.observation_operator(N, pts).toarray()
    I = fem.interior_nodes(N)
    assert np.allclose(O[:, I], np.eye(49), atol=1e-15)
    # P1 interpolation reproduces linear functions at arbitrary points, and values on finer levels
    nodes, _ = fem.mesh(16)
    lin = 0.3 + 1.7 * nodes[:, 0] - 0.4 * nodes[:, 1]
    q = np.random.default_rng(3).uniform(0, 1, (50, 2))
    O = fem.observation_operator(16, q)
    assert np.allclose(O @ lin, 0.3 + 1.7 * q[:, 0] - 0.4 * q[:, 1], atol=1e-14)
    assert np.allclose(O.sum(axis=1), 1.0)


def _column_kappa(N, k):
    """kappa constant in each column of cells (both triangles of cell (i, j) take k[i])."""
    kap = np.empty(2 * N * N)
    for j in range(N):
        for i in range(N):
            kap[2 * (j * N + i)] = kap[2 * (j * N + i) + 1] = k[i]
    return kap


def test_flow_cell_linear_solution_for_constant_kappa():
    """Example 5.3's boundary conditions with kappa = c: p(x, y) = x at every node (P1 reproduces
    the exact linear solution)."""
    N = 16
    p = fem.solve_flow_cell(N, np.full(2 * N * N, 3.7))
    x = np.tile(np.arange(N + 1) / N, N + 1)
    assert np.max(np.abs(p - x)) < 1e-12


def test_flow_cell_series_conductances():
    """kappa constant in each column of cells: the flow is one-dimensional and the nodal pressure
    is the series-resistance formula p(x_i) = sum_{m<i} 1/k_m / sum_m 1/k_m on every row, the
    boundary rows (half conductances) included."""
    N = 16
    k = np.exp(np.random.default_rng(3).normal(0, 1, N))
    p = fem.solve_flow_cell(N, _column_kappa(N, k)).reshape(N + 1, N + 1)
    r = np.concatenate([[0.0], np.cumsum(1.0 / k)]) / np.sum(1.0 / k)
    assert np.max(np.abs(p - r[None, :])) < 1e-12


def test_flow_cell_half_turn_and_maximum_principle():
    """For kappa invariant under the half turn (x, y) -> (1-x, 1-y), which maps the mesh and swaps
    the two Dirichlet sides, p(1-x, 1-y) = 1 - p(x, y); for any kappa 0 <= p <= 1."""
    N = 16
    rng = np.random.default_rng(8)
    kap = np.exp(rng.normal(0, 1, 2 * N * N))
    kap = 0.5 * (kap + kap[::-1])            # element e <-> 2N^2 - 1 - e is the half turn
    p = fem.solve_flow_cell(N, kap).reshape(N + 1, N + 1)
    assert np.max(np.abs(p[::-1, ::-1] - (1.0 - p))) < 1e-12
    q = fem.solve_flow_cell(N, np.exp(rng.normal(0, 1.5, 2 * N * N)))
    assert q.min() >= -1e-14 and q.max() <= 1 + 1e-14


def test_flow_cell_prior_mean_scales_out():
    """f = 0 and Dirichlet data: kappa -> c kappa leaves p unchanged, so the prior mean m0 = 2 of
    Example 5.3 does not change G (checked through the forward map with and without m0)."""
    from oracle import forward
    obs = np.array([[0.25, 0.5], [0.5, 0.125], [0.875, 0.75]])
    th = np.random.default_rng(1).normal(0, 1, 4)
    a = forward.Level(16, 0.3, 1.0, 4, obs, bc="flow_cell").G(th)
    b = forward.Level(16, 0.3, 1.0, 4, obs, bc="flow_cell", m0=2.0).G(th)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-14) and np.all((a > 0) & (a < 1))

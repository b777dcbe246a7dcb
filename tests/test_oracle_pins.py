"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Every check here is independent of the oracle's own loops: dense linear
algebra from numpy, closed-form spectra, a hand-worked example, level sets
from a graph library, and invariances the paper's tables show.  A dropped
term, a wrong sign, a transposed triangle or an in-place inner sweep in the
oracle fails at least one of them.
"""
import math
import os

import networkx as nx
import numpy as np
import pytest

import oracle
from paper_2104_01196_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_parts(A):
    M = P.csr_to_dense(A)
    D = np.diag(np.diag(M))
    L = np.tril(M, -1)
    U = np.triu(M, 1)
    return M, D, L, U


def tiny_nonsym(n=7, seed=5):
    rng = np.random.default_rng(seed)
    M = rng.uniform(-1, 1, (n, n)) * (rng.uniform(0, 1, (n, n)) < 0.5)
    np.fill_diagonal(M, np.abs(M).sum(1) + rng.uniform(0.5, 1.5, n))
    return P.dense_to_csr(M)


# ---------------------------------------------------------------------------
# A hand-worked example (Eq. 3-5 applied by hand to a 3x3 tridiagonal system)
# ---------------------------------------------------------------------------

def test_hand_worked_gs2_and_gs():
    M = np.array([[4.0, -1, 0], [-1, 4, -1], [0, -1, 4]])
    A = P.dense_to_csr(M)
    b = np.array([1.0, 2.0, 3.0])
    # g0 = D^-1 r = [1/4, 1/2, 3/4]; g1 = D^-1 (r - L g0) = [1/4, 9/16, 7/8]
    x1 = oracle.gs2(A, b, np.zeros(3), outer=1, inner=1)
    assert x1.tolist() == [0.25, 0.5625, 0.875]
    # g2 = D^-1 (r - L g1) = [1/4, 9/16, 57/64] = exact forward GS (depth 2)
    x2 = oracle.gs2(A, b, np.zeros(3), outer=1, inner=2)
    assert x2.tolist() == [0.25, 0.5625, 0.890625]
    xg = oracle.gs(A, b, np.zeros(3), sweeps=1)
    assert xg.tolist() == [0.25, 0.5625, 0.890625]
    # zero inner sweeps = Jacobi-Richardson: D^-1 b
    x0 = oracle.gs2(A, b, np.zeros(3), outer=1, inner=0)
    assert x0.tolist() == [0.25, 0.5, 0.75]


# ---------------------------------------------------------------------------
# Exact GS / SOR against a dense triangular solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("omega", [1.0, 0.7, 1.3])
def test_gs_equals_dense_sor(omega):
    A = tiny_nonsym()
    M, D, L, U = dense_parts(A)
    rng = np.random.default_rng(1)
    b, x0 = rng.standard_normal(7), rng.standard_normal(7)
    # non-compact SOR form of the damping paragraph: x + w (D + w L)^-1 (b - A x)
    fwd = x0 + omega * np.linalg.solve(D + omega * L, b - M @ x0)
    assert np.allclose(oracle.gs(A, b, x0, 1, omega, oracle.FORWARD), fwd,
                       rtol=1e-13, atol=1e-13)
    # compact form of the same paragraph: w (D + w L)^-1 (b - [U + (1 - 1/w) D] x)
    cmp_ = omega * np.linalg.solve(D + omega * L, b - (U + (1 - 1 / omega) * D) @ x0)
    assert np.allclose(fwd, cmp_, rtol=1e-12, atol=1e-12)
    bwd = x0 + omega * np.linalg.solve(D + omega * U, b - M @ x0)
    assert np.allclose(oracle.gs(A, b, x0, 1, omega, oracle.BACKWARD), bwd,
                       rtol=1e-13, atol=1e-13)
    sym = fwd + omega * np.linalg.solve(D + omega * U, b - M @ fwd)
    assert np.allclose(oracle.gs(A, b, x0, 1, omega, oracle.SYMMETRIC), sym,
                       rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# GS2 against the closed forms of Sec. 4
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("inner", [0, 1, 2, 3])
@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_gs2_equals_neumann_series(inner, omega):
    """x + w sum_{j<=s} (-w D^-1 L)^j D^-1 r  (degree-s Neumann expansion)."""
    A = tiny_nonsym()
    M, D, L, U = dense_parts(A)
    rng = np.random.default_rng(2)
    b, x0 = rng.standard_normal(7), rng.standard_normal(7)
    Di = np.diag(1 / np.diag(M))
    r = b - M @ x0
    for T, d in ((L, oracle.FORWARD), (U, oracle.BACKWARD)):
        S = sum(np.linalg.matrix_power(-omega * Di @ T, j) for j in range(inner + 1))
        expect = x0 + omega * S @ Di @ r
        got = oracle.gs2(A, b, x0, 1, inner, omega, 1.0, d)
        assert np.allclose(got, expect, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("gamma", [0.5, 0.9, 1.2])
def test_gs2_inner_damping_closed_form(gamma):
    """Damped inner JR: g_s = g* + T^s (g_0 - g*), T = (1-gamma) I - gamma w D^-1 L,
    g* = (D + w L)^-1 r, g_0 = D^-1 r."""
    A = tiny_nonsym(6, 9)
    M, D, L, U = dense_parts(A)
    rng = np.random.default_rng(3)
    b, x0 = rng.standard_normal(6), rng.standard_normal(6)
    omega = 0.9
    Di = np.diag(1 / np.diag(M))
    r = b - M @ x0
    gstar = np.linalg.solve(D + omega * L, r)
    T = (1 - gamma) * np.eye(6) - gamma * omega * Di @ L
    for s in (1, 2, 4):
        g = gstar + np.linalg.matrix_power(T, s) @ (Di @ r - gstar)
        got = oracle.gs2(A, b, x0, 1, s, omega, gamma, oracle.FORWARD)
        assert np.allclose(got, x0 + omega * g, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", [6, 16])
def test_gs2_with_depth_inner_sweeps_is_exact_gs(N):
    """D^-1 L is nilpotent: with inner sweeps >= depth(L) GS2 is exact GS,
    with one fewer it is not (checked where the missing Neumann term,
    (1/4)^depth times a path count, is far above rounding)."""
    A = P.poisson2d_matrix(N)
    _, nlev = oracle.levels(A, lower=True)
    depth = nlev - 1
    assert depth == 2 * N - 2
    rng = np.random.default_rng(4)
    b, x0 = rng.standard_normal(N * N), rng.standard_normal(N * N)
    for d in (oracle.FORWARD, oracle.BACKWARD, oracle.SYMMETRIC):
        for omega in (1.0, 0.8):
            ex = oracle.gs(A, b, x0, 1, omega, d)
            got = oracle.gs2(A, b, x0, 1, depth, omega, 1.0, d)
            assert np.linalg.norm(got - ex) <= 1e-13 * np.linalg.norm(ex)
            if N <= 8 and d != oracle.SYMMETRIC:
                # (in a symmetric sweep the backward half absorbs most of it)
                short = oracle.gs2(A, b, x0, 1, depth - 1, omega, 1.0, d)
                assert np.linalg.norm(short - ex) > 1e-6 * np.linalg.norm(ex)


def test_gs2_zero_inner_is_jacobi_richardson():
    pr = P.random_system(300, 17)
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(pr.n)
    for omega in (1.0, 0.6):
        a = oracle.gs2(pr.A, pr.b, x0, 3, 0, omega, 1.0, oracle.FORWARD)
        j = oracle.jr(pr.A, pr.b, x0, 3, omega)
        assert np.allclose(a, j, rtol=1e-14, atol=1e-14)


def test_diagonal_matrix_collapses_everything():
    n = 40
    d = 1.0 + np.arange(n) % 7
    A = (np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d.copy())
    b = np.linspace(-1, 1, n)
    for omega in (1.0, 0.7):
        expect = omega * b / d
        for got in (oracle.gs2(A, b, np.zeros(n), 1, 3, omega, 1.0, oracle.SYMMETRIC * 0),
                    oracle.gs(A, b, np.zeros(n), 1, omega),
                    oracle.jr(A, b, np.zeros(n), 1, omega)):
            assert np.allclose(got, expect, rtol=1e-15, atol=0)
    # omega = 1: one sweep solves the system exactly
    assert np.array_equal(oracle.gs2(A, b, np.zeros(n), 1, 1), b / d)


def test_residual_propagators_of_sec4():
    """Sec. 5.3: one GS2(1) sweep maps r to (I - A D^-1 [I - L D^-1]) r, two JR
    sweeps to (I - A D^-1)^2 r = (I - A D^-1 [I - (L+U) D^-1]) r, SGS2(1) to
    (I - A D^-1 [I - U D^-1])(I - A D^-1 [I - L D^-1]) r."""
    A = tiny_nonsym(8, 13)
    M, D, L, U = dense_parts(A)
    Di = np.diag(1 / np.diag(M))
    I = np.eye(8)
    rng = np.random.default_rng(6)
    b, x0 = rng.standard_normal(8), rng.standard_normal(8)
    r0 = b - M @ x0
    Pg = I - M @ Di @ (I - L @ Di)
    Pb = I - M @ Di @ (I - U @ Di)
    Pj = I - M @ Di
    x = oracle.gs2(A, b, x0, 1, 1, 1.0, 1.0, oracle.FORWARD)
    assert np.allclose(b - M @ x, Pg @ r0, rtol=1e-12, atol=1e-12)
    x = oracle.gs2(A, b, x0, 1, 1, 1.0, 1.0, oracle.SYMMETRIC)
    assert np.allclose(b - M @ x, Pb @ Pg @ r0, rtol=1e-12, atol=1e-12)
    x = oracle.jr(A, b, x0, 2, 1.0)
    assert np.allclose(b - M @ x, Pj @ Pj @ r0, rtol=1e-12, atol=1e-12)
    assert np.allclose(Pj @ Pj, I - M @ Di @ (I - (L + U) @ Di), atol=1e-13)
    x = oracle.jr(A, b, x0, 3, 1.0)
    assert np.allclose(b - M @ x, Pj @ Pj @ Pj @ r0, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# Closed-form spectra of the 2D Dirichlet Laplacian (textbook)
# ---------------------------------------------------------------------------

def iteration_matrix(step, n):
    """Columns T e_i of a stationary iteration x -> T x (b = 0)."""
    return np.stack([step(np.eye(n)[:, i]) for i in range(n)], axis=1)


@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_jacobi_spectrum_2d_laplacian(omega):
    N = 8
    A = P.poisson2d_matrix(N)
    n = N * N
    T = iteration_matrix(lambda e: oracle.jr(A, np.zeros(n), e, 1, omega), n)
    ev = np.sort(np.linalg.eigvals(T).real)
    k = np.arange(1, N + 1)
    mu = (np.cos(np.pi * k / (N + 1))[:, None] + np.cos(np.pi * k / (N + 1))[None, :]) / 2
    expect = np.sort((1 - omega * (1 - mu)).ravel())
    assert np.allclose(ev, expect, atol=1e-12)
    rho = np.abs(ev).max()
    rho_cf = max(abs(1 - omega * (1 - math.cos(math.pi / (N + 1)))),
                 abs(1 - omega * (1 + math.cos(math.pi / (N + 1)))))
    assert abs(rho - rho_cf) < 1e-12


def test_jacobi_rho_for_64_grid_closed_form():
    # rho_J = cos(pi/65) for the 64 x 64 grid of the small workload
    assert abs(math.cos(math.pi / 65) - 0.998832) < 5e-7


def test_gs_and_sor_spectral_radius_young():
    """Lexicographic 5-point Laplacian is consistently ordered: rho(GS) =
    rho_J^2 and rho(SOR at w_opt) = w_opt - 1 (Young)."""
    N = 8
    A = P.poisson2d_matrix(N)
    n = N * N
    muJ = math.cos(math.pi / (N + 1))
    Tgs = iteration_matrix(lambda e: oracle.gs(A, np.zeros(n), e, 1, 1.0), n)
    assert abs(np.abs(np.linalg.eigvals(Tgs)).max() - muJ ** 2) < 1e-10
    wopt = 2 / (1 + math.sqrt(1 - muJ ** 2))
    Tsor = iteration_matrix(lambda e: oracle.gs(A, np.zeros(n), e, 1, wopt), n)
    # a 2x2 Jordan block sits at w_opt - 1: eigenvalues move by ~sqrt(eps)
    assert abs(np.abs(np.linalg.eigvals(Tsor)).max() - (wopt - 1)) < 1e-6
    # GS2 with inner sweeps >= depth has the same iteration matrix as GS
    Tgs2 = iteration_matrix(lambda e: oracle.gs2(A, np.zeros(n), e, 1, 2 * N - 2), n)
    assert np.allclose(Tgs2, Tgs, atol=1e-13)


# ---------------------------------------------------------------------------
# Level sets
# ---------------------------------------------------------------------------

def test_levels_of_structured_grids():
    N = 9
    lev, nlev = oracle.levels(P.poisson2d_matrix(N), lower=True)
    i = np.arange(N * N)
    assert nlev == 2 * N - 1
    assert np.array_equal(lev, (i % N) + (i // N))
    lev, nlev = oracle.levels(P.poisson2d_matrix(N), lower=False)
    assert np.array_equal(lev, (N - 1 - i % N) + (N - 1 - i // N))
    N = 6
    lev, nlev = oracle.levels(P.poisson3d_matrix(N), lower=True)
    i = np.arange(N ** 3)
    assert nlev == 3 * N - 2
    assert np.array_equal(lev, i % N + (i // N) % N + i // (N * N))


def test_levels_equal_longest_path_brute_force():
    A = P.random_csr(120, 21, mean_offdiag=3.0)
    rp, ci, _ = A
    G = nx.DiGraph()
    G.add_nodes_from(range(120))
    for i in range(120):
        for k in range(rp[i], rp[i + 1]):
            if ci[k] < i:
                G.add_edge(int(ci[k]), i)
    lev, nlev = oracle.levels(A, lower=True)
    longest = {v: 0 for v in G.nodes}
    for v in nx.topological_sort(G):
        for w in G.successors(v):
            longest[w] = max(longest[w], longest[v] + 1)
    assert [longest[v] for v in range(120)] == lev.tolist()
    assert nlev - 1 == nx.dag_longest_path_length(G)


# ---------------------------------------------------------------------------
# Multicolour GS (Sec. 6.1.2) against a dense solve in the colour ordering
# ---------------------------------------------------------------------------

def test_coloring_red_black_on_stencils_and_valid_on_random():
    N = 7
    col, nc = oracle.coloring(P.poisson2d_matrix(N))
    i = np.arange(N * N)
    assert nc == 2 and np.array_equal(col, (i % N + i // N) % 2)
    col, nc = oracle.coloring(P.poisson3d_matrix(5))
    i = np.arange(125)
    assert nc == 2 and np.array_equal(col, (i % 5 + (i // 5) % 5 + i // 25) % 2)
    A = P.random_csr(150, 9, mean_offdiag=4.0)
    rp, ci, _ = A
    col, nc = oracle.coloring(A)
    G = nx.Graph()
    G.add_nodes_from(range(150))
    for r in range(150):
        for k in range(rp[r], rp[r + 1]):
            if ci[k] != r:
                G.add_edge(r, int(ci[k]))
    assert all(col[u] != col[v] for u, v in G.edges)
    # first fit in natural order: every colour c > 0 of row i has an earlier
    # neighbour of each smaller colour, and the count equals the largest + 1
    for v in range(150):
        seen = {int(col[u]) for u in G.neighbors(v) if u < v}
        assert set(range(col[v])) <= seen
    assert nc == col.max() + 1
    greedy = nx.greedy_color(G, strategy=lambda g, c: range(150))
    assert [greedy[v] for v in range(150)] == col.tolist()


@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_mtgs_equals_dense_sor_in_colour_order(omega):
    """MT-GS is SOR on P A P^T with rows sorted (stably) by colour."""
    A = P.random_csr(60, 4, mean_offdiag=3.0)
    M = P.csr_to_dense(A)
    col, nc = oracle.coloring(A)
    assert nc >= 3
    perm = np.argsort(col, kind="stable")
    Mp = M[np.ix_(perm, perm)]
    D, L, U = np.diag(np.diag(Mp)), np.tril(Mp, -1), np.triu(Mp, 1)
    rng = np.random.default_rng(3)
    b, x0 = rng.standard_normal(60), rng.standard_normal(60)
    bp, xp = b[perm], x0[perm]
    fwd = xp + omega * np.linalg.solve(D + omega * L, bp - Mp @ xp)
    bwd = xp + omega * np.linalg.solve(D + omega * U, bp - Mp @ xp)
    sym = fwd + omega * np.linalg.solve(D + omega * U, bp - Mp @ fwd)
    for d, want in ((oracle.FORWARD, fwd), (oracle.BACKWARD, bwd),
                    (oracle.SYMMETRIC, sym)):
        got = oracle.mtgs(A, b, x0, 1, omega, d)
        assert np.allclose(got[perm], want, rtol=1e-12, atol=1e-12)


def test_mtgs_red_black_poisson_is_two_jacobi_half_steps():
    """On a red-black grid each colour's rows see only the other colour."""
    N = 6
    A = P.poisson2d_matrix(N)
    M = P.csr_to_dense(A)
    col, _ = oracle.coloring(A)
    rng = np.random.default_rng(8)
    b, x = rng.standard_normal(N * N), rng.standard_normal(N * N)
    y = x.copy()
    for c in (0, 1):
        m = col == c
        y[m] = (b[m] - (M[m] @ y - np.diag(M)[m] * y[m])) / np.diag(M)[m]
    assert np.allclose(oracle.mtgs(A, b, x, 1, 1.0, oracle.FORWARD), y,
                       rtol=1e-13, atol=1e-13)
    # a multicolour preconditioner from zero equals one sweep from zero
    z = oracle.precond(A, b, kind=oracle.PC_MTGS, outer=1, omega=1.0)
    assert np.allclose(z, oracle.mtgs(A, b, np.zeros(N * N), 1, 1.0), atol=0)


# ---------------------------------------------------------------------------
# Smoothed-aggregation AMG with a GS2 smoother
# ---------------------------------------------------------------------------

def _amg_golden():
    out = {}
    for line in open(os.path.join(GOLDEN, "amg_aggregates.txt")):
        if line.strip() and not line.startswith("#"):
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


def test_amg_aggregates_hand_worked():
    g = _amg_golden()
    n = 10
    L1 = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    M = oracle.AMG(P.dense_to_csr(L1), coarse_size=2, max_levels=2)
    assert M.aggregates(0).tolist() == g["laplace1d_10"]
    M = oracle.AMG(P.poisson2d_matrix(4), coarse_size=2, max_levels=2)
    assert M.aggregates(0).tolist() == g["laplace2d_4x4"]


def test_amg_aggregates_are_connected_partitions():
    A = P.random_csr(400, 12, mean_offdiag=4.0)
    M = oracle.AMG(A, coarse_size=8, max_levels=3)
    rp, ci, va = A
    agg = M.aggregates(0)
    na = M.level(1)[0]
    assert sorted(set(agg.tolist())) == list(range(na))
    # every aggregate is connected in the symmetrised strength graph
    G = nx.Graph()
    G.add_nodes_from(range(400))
    for i in range(400):
        row = slice(rp[i], rp[i + 1])
        off = [(int(j), abs(v)) for j, v in zip(ci[row], va[row]) if j != i]
        mx = max((v for _, v in off), default=0.0)
        for j, v in off:
            if mx > 0 and v >= 0.25 * mx:
                G.add_edge(i, j)
    for a in range(na):
        assert nx.is_connected(G.subgraph(np.flatnonzero(agg == a).tolist()))


def test_amg_prolongator_maps_aggregate_sizes_to_smoothed_ones():
    """P0 s = 1 with s_a = sqrt(|aggregate a|), so P s = (I - w D^-1 A) 1 =
    1 - w (row sums of A) / a_ii with w = 4 / (3 max_i sum_j |a_ij| / |a_ii|)."""
    for A in (P.poisson2d_matrix(9), P.random_csr(300, 13, mean_offdiag=5.0)):
        Md = P.csr_to_dense(A)
        d = np.diag(Md)
        w = 4.0 / (3.0 * np.max(np.abs(Md).sum(1) / np.abs(d)))
        M = oracle.AMG(A, coarse_size=4, max_levels=2)
        agg = M.aggregates(0)
        s = np.sqrt(np.bincount(agg).astype(float))
        Pd = _dense(M.prolongator(0), M.level(1)[0])
        assert np.allclose(Pd @ s, 1.0 - w * Md.sum(1) / d, rtol=0, atol=1e-13)


def _dense(csr, ncols):
    rp, ci, va = csr
    n = len(rp) - 1
    D = np.zeros((n, ncols))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            D[i, ci[k]] += va[k]
    return D


def test_amg_coarse_correction_is_a_projection():
    """Two levels, no smoothing: C = I - P A_c^-1 P^T A is idempotent and
    A-self-adjoint exactly when A_c is the Galerkin product and the cycle
    restricts with P^T and prolongs with P."""
    A = P.poisson2d_matrix(7)
    Md = P.csr_to_dense(A)
    M = oracle.AMG(A, coarse_size=30, max_levels=2)
    assert M.levels == 2
    n = Md.shape[0]
    Minv = np.column_stack([M.vcycle(e, outer=0) for e in np.eye(n)])
    C = np.eye(n) - Minv @ Md
    assert np.allclose(C @ C, C, atol=1e-12)
    assert np.allclose(Md @ C, (Md @ C).T, atol=1e-12)
    # rank of the correction = number of aggregates
    assert np.linalg.matrix_rank(Minv, tol=1e-10) == M.level(1)[0]


def test_amg_symmetric_vcycle_is_spd_and_contracts():
    """Forward pre- and backward post-smoothing give a symmetric positive
    definite preconditioner for SPD A; a forward-forward cycle does not, and
    the error propagator I - M^-1 A contracts in the A-norm."""
    A = P.poisson2d_matrix(8)
    Md = P.csr_to_dense(A)
    n = Md.shape[0]
    M = oracle.AMG(A, coarse_size=10, max_levels=3)
    assert M.levels == 3
    for kw in (dict(kind=oracle.PC_GS2, inner=1, omega=0.9),
               dict(kind=oracle.PC_GS2, inner=3),
               dict(kind=oracle.PC_JR, outer=2, omega=0.7)):
        Minv = np.column_stack([M.vcycle(e, direction=oracle.SYMMETRIC, **kw)
                                for e in np.eye(n)])
        assert np.allclose(Minv, Minv.T, atol=1e-12), kw
        assert np.linalg.eigvalsh((Minv + Minv.T) / 2).min() > 0
        E = np.eye(n) - Minv @ Md
        Lc = np.linalg.cholesky(Md)
        assert np.linalg.norm(Lc.T @ E @ np.linalg.inv(Lc.T), 2) < 1.0
    Mff = np.column_stack([M.vcycle(e, direction=oracle.FORWARD, inner=1) for e in np.eye(n)])
    assert not np.allclose(Mff, Mff.T, atol=1e-6)


def test_amg_preconditioned_cg_converges_like_gmres():
    """The symmetric V-cycle is SPD (pinned above), so CG with it converges on
    an SPD system, in about as many iterations as GMRES with the same cycle."""
    pr = P.poisson3d(16)
    M = oracle.AMG(pr.A)
    xc, ic = M.cg(pr.A, pr.b, tol=1e-8, max_iters=200)
    _, ig = M.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=200)
    assert ic.status == 0 and ic.true_relres <= 1e-8
    assert abs(ic.iters - ig.iters) <= 3 and ic.iters <= 15
    r = np.linalg.norm(pr.b - oracle.spmv(pr.A, xc)) / np.linalg.norm(pr.b)
    assert r <= 1e-8


def test_amg_iterations_grid_independent():
    """Multigrid: GMRES iterations stay flat as the grid is refined, while
    the one-level SGS2 preconditioner's grow with it."""
    amg, one = [], []
    for N in (32, 64, 128):
        pr = P.poisson2d(N)
        M = oracle.AMG(pr.A)
        _, info = M.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=500)
        assert info.status == 0
        amg.append(info.iters)
        _, info = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=5000,
                               pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC)
        one.append(info.iters)
    assert max(amg) - min(amg) <= 3 and max(amg) <= 14, amg
    assert one[2] > 2 * one[0], one


# ---------------------------------------------------------------------------
# GMRES against the Krylov least-squares minimiser
# ---------------------------------------------------------------------------

def precond_matrix(A, n, **kw):
    return iteration_matrix(lambda e: oracle.precond(A, e, **kw), n)


@pytest.mark.parametrize("pc", [dict(kind=oracle.PC_NONE),
                                dict(kind=oracle.PC_GS2, inner=1, omega=0.9),
                                dict(kind=oracle.PC_GS2, inner=2,
                                     direction=oracle.SYMMETRIC),
                                dict(kind=oracle.PC_JR, outer=2, omega=0.7)])
def test_gmres_residuals_are_krylov_minima(pc):
    n = 7
    A = tiny_nonsym(n, 31)
    M = P.csr_to_dense(A)
    b = np.random.default_rng(7).standard_normal(n)
    Minv = precond_matrix(A, n, **pc)
    AM = M @ Minv
    x, info, hist = oracle.gmres(A, b, restart=n, tol=1e-14, max_iters=n,
                                 pc_kind=pc["kind"], pc_outer=pc.get("outer", 1),
                                 pc_inner=pc.get("inner", 1),
                                 pc_omega=pc.get("omega", 1.0),
                                 pc_direction=pc.get("direction", 0), history=True)
    K = np.stack([np.linalg.matrix_power(AM, j) @ b for j in range(n)], axis=1)
    for k in range(1, info.iters + 1):
        y, *_ = np.linalg.lstsq(AM @ K[:, :k], b, rcond=None)
        best = np.linalg.norm(b - AM @ K[:, :k] @ y) / np.linalg.norm(b)
        # the power basis K is ill-conditioned, hence the absolute floor
        assert abs(hist[k - 1] - best) <= max(1e-9 * best, 1e-10), (k, hist[k - 1], best)
    assert info.iters <= n
    assert info.status == 0
    assert np.allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)


def test_gmres_restart_and_true_residual():
    pr = P.poisson2d(24, seed=P.SEED_BASE)
    x, info = oracle.gmres(pr.A, pr.b, restart=5, tol=1e-8, max_iters=5000,
                           pc_kind=oracle.PC_GS2, pc_inner=1)
    assert info.status == 0 and info.cycles > 1
    r = pr.b - P.csr_matvec(pr.A, x)
    assert np.linalg.norm(r) / np.linalg.norm(pr.b) == pytest.approx(info.true_relres, rel=1e-6)
    assert info.true_relres <= 1e-8


def test_gmres_small_workload_converges():
    """2D 5-point Poisson 64x64, GMRES(30), one forward GS2 sweep with one
    inner sweep, rel. residual 1e-8."""
    pr = P.poisson2d(64)
    x, info = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=2000,
                           pc_kind=oracle.PC_GS2, pc_inner=1)
    assert info.status == 0 and info.true_relres <= 1e-8
    assert np.linalg.norm(x - pr.x_true) / np.linalg.norm(pr.x_true) < 1e-4
    # unpreconditioned GMRES(30) needs more iterations, symmetric GS2 fewer
    _, info0 = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=20000,
                            pc_kind=oracle.PC_NONE)
    _, info2 = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=20000,
                            pc_kind=oracle.PC_GS2, pc_inner=1,
                            pc_direction=oracle.SYMMETRIC)
    assert info0.iters > info.iters > info2.iters


def _golden(key):
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as f:
        for line in f:
            if line.startswith(key + " "):
                return dict(kv.split("=") for kv in line.split()[1:])
    raise KeyError(key)


def test_jr1_iteration_count_independent_of_omega():
    """Table ela3d-omega prints 213 GMRES iterations for JR(1) at every omega:
    one JR sweep from zero is omega D^-1, and GMRES does not see a scalar
    factor on the preconditioner."""
    g = _golden("jr1_vs_omega")
    assert len(set(g["iters"].split(","))) == 1
    A, clamped = P.elasticity_matrix(5)
    b = P.elasticity_body_load(5, clamped)
    counts = []
    for om in [float(w) for w in g["omega"].split(",")]:
        _, info = oracle.gmres(A, b, restart=30, tol=1e-8, max_iters=3000,
                               pc_kind=oracle.PC_JR, pc_outer=1, pc_omega=om)
        assert info.status == 0
        counts.append(info.iters)
    assert len(set(counts)) == 1, counts


def test_sgs2_enough_inner_sweeps_matches_sgs_iterations():
    """Table ela3d-omega: SGS2(1,10) takes the SGS count (61 = 61 at omega=1)."""
    g = _golden("sgs_vs_sgs2_1_10")
    assert g["sgs"] == g["sgs2_1_10"]
    A = P.poisson3d_matrix(6)
    b = P.csr_matvec(A, P.uniform_pm1(3, 216))
    _, nlev = oracle.levels(A)
    _, i_gs = oracle.gmres(A, b, restart=30, tol=1e-10, pc_kind=oracle.PC_GS,
                           pc_direction=oracle.SYMMETRIC)
    _, i_gs2 = oracle.gmres(A, b, restart=30, tol=1e-10, pc_kind=oracle.PC_GS2,
                            pc_inner=nlev - 1, pc_direction=oracle.SYMMETRIC)
    assert i_gs.iters == i_gs2.iters


# ---------------------------------------------------------------------------
# CG and compact GS2
# ---------------------------------------------------------------------------

def test_cg_iterates_minimise_energy_norm():
    M = P.csr_to_dense(P.poisson2d_matrix(3))
    A = P.dense_to_csr(M)
    b = np.arange(1.0, 10.0)
    xs = np.linalg.solve(M, b)
    K = np.stack([np.linalg.matrix_power(M, j) @ b for j in range(9)], axis=1)
    for k in range(1, 4):
        x, info = oracle.cg(A, b, tol=1e-300, max_iters=k, pc_kind=oracle.PC_NONE)
        # min over y of ||K y - x*||_A
        Q = K[:, :k]
        y = np.linalg.solve(Q.T @ M @ Q, Q.T @ M @ xs)
        assert np.allclose(x, Q @ y, rtol=1e-9, atol=1e-11)


def test_cg_with_sgs2_converges_and_sgs2_is_symmetric():
    pr = P.poisson2d(20)
    x, info = oracle.cg(pr.A, pr.b, tol=1e-8, pc_kind=oracle.PC_GS2, pc_inner=1,
                        pc_direction=oracle.SYMMETRIC)
    assert info.status == 0 and info.true_relres <= 1e-8
    Minv = precond_matrix(P.poisson2d_matrix(6), 36, kind=oracle.PC_GS2, inner=1,
                          direction=oracle.SYMMETRIC)
    assert np.allclose(Minv, Minv.T, atol=1e-14)


def test_compact_gs2_closed_form_and_exact_limit():
    A = tiny_nonsym(7, 41)
    M, D, L, U = dense_parts(A)
    Di = np.diag(1 / np.diag(M))
    rng = np.random.default_rng(8)
    b, x0 = rng.standard_normal(7), rng.standard_normal(7)
    for s in (0, 1, 2):
        S = sum(np.linalg.matrix_power(-Di @ L, j) for j in range(s + 1))
        expect = S @ Di @ (b - U @ x0)
        got = oracle.gs2_compact(A, b, x0, 1, s, oracle.FORWARD)
        assert np.allclose(got, expect, rtol=1e-13, atol=1e-13)
    # exact inner solve: compact and non-compact GS coincide (Eq. 1 vs Eq. 8)
    Ap = P.poisson2d_matrix(7)
    bb, xx = rng.standard_normal(49), rng.standard_normal(49)
    assert np.allclose(oracle.gs2_compact(Ap, bb, xx, 1, 12), oracle.gs(Ap, bb, xx, 1),
                       rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# Error statuses
# ---------------------------------------------------------------------------

def test_statuses():
    A = P.dense_to_csr(np.array([[1.0, 2.0], [3.0, 0.0]]))
    with pytest.raises(oracle.OracleError):
        oracle.gs2(A, np.ones(2), np.zeros(2))
    pr = P.poisson2d(16)
    _, info = oracle.gmres(pr.A, pr.b, restart=10, tol=1e-12, max_iters=3,
                           pc_kind=oracle.PC_NONE)
    assert info.status == 5 and info.iters == 3
    b = pr.b.copy()
    b[3] = np.nan
    _, info = oracle.gmres(pr.A, b, restart=10, tol=1e-8, max_iters=30)
    assert info.status == 7


# ---------------------------------------------------------------------------
# Hybrid (block-Jacobi) relaxation, Sec. 3 with the local sweeps of the
# two-stage listing: dense block computations, and the special cases that
# reduce it to the global methods
# ---------------------------------------------------------------------------

def _blocks(n, parts):
    blk = np.empty(n, dtype=int)
    for p in range(parts):
        blk[p * n // parts:(p + 1) * n // parts] = p
    return blk


def _dense_hybrid(M, b, x, parts, outer, local, sweep):
    """Dense reference: per exchange c = b - E x (E the couplings between
    blocks), then `local` sweeps x <- sweep(A_loc, c, x)."""
    n = len(b)
    blk = _blocks(n, parts)
    same = blk[:, None] == blk[None, :]
    Aloc, E = np.where(same, M, 0.0), np.where(same, 0.0, M)
    for _ in range(outer):
        c = b - E @ x
        for _ in range(local):
            x = sweep(Aloc, c, x)
    return x


def test_hybrid_gs_is_block_jacobi_with_sor_blocks():
    """Local exact GS = x + omega (D + omega L_loc)^{-1} (c - A_loc x) per
    half sweep, with the other blocks' values frozen at the exchange."""
    A = tiny_nonsym(9, seed=11)
    M, _, _, _ = dense_parts(A)
    b = np.linspace(-1.0, 2.0, 9)
    x0 = np.linspace(0.5, -0.5, 9)
    om = 0.8

    def fwd(Al, c, x):
        Dl, Ll = np.diag(np.diag(Al)), np.tril(Al, -1)
        return x + om * np.linalg.solve(Dl + om * Ll, c - Al @ x)

    def bwd(Al, c, x):
        Dl, Ul = np.diag(np.diag(Al)), np.triu(Al, 1)
        return x + om * np.linalg.solve(Dl + om * Ul, c - Al @ x)

    for parts, outer, local in ((3, 1, 1), (3, 2, 3), (4, 1, 2)):
        want = _dense_hybrid(M, b, x0.copy(), parts, outer, local, lambda Al, c, x: bwd(Al, c, fwd(Al, c, x)))
        got = oracle.hybrid(A, b, x0, oracle.PC_GS, parts=parts, outer=outer, local=local,
                            omega=om, direction=oracle.SYMMETRIC)
        assert np.allclose(got, want, rtol=0, atol=1e-13), (parts, outer, local)


def test_hybrid_gs2_is_block_neumann_with_local_triangles():
    """Local GS2 half sweep: g0 = D^{-1} r, n_j damped JR sweeps with the
    local triangle, x += omega g (dense, per exchange)."""
    A = tiny_nonsym(10, seed=12)
    M, _, _, _ = dense_parts(A)
    b = np.linspace(1.0, -1.0, 10)
    x0 = np.cos(np.arange(10.0))
    om, ga, nj = 0.9, 0.7, 2

    def half(Al, c, x, tri):
        Dl = np.diag(np.diag(Al))
        T = tri(Al, -1) if tri is np.tril else tri(Al, 1)
        r = c - Al @ x
        g = np.linalg.solve(Dl, r)
        for _ in range(nj):
            g = (1 - ga) * g + ga * np.linalg.solve(Dl, r - om * T @ g)
        return x + om * g

    want = _dense_hybrid(M, b, x0.copy(), 3, 2, 2,
                         lambda Al, c, x: half(Al, c, half(Al, c, x, np.tril), np.triu))
    got = oracle.hybrid(A, b, x0, oracle.PC_GS2, parts=3, outer=2, local=2, inner=nj, omega=om,
                        gamma=ga, direction=oracle.SYMMETRIC)
    assert np.allclose(got, want, rtol=0, atol=1e-13)


def test_hybrid_reduces_to_the_global_methods():
    pr = P.poisson2d(12)
    x0 = P.uniform_pm1(3, pr.n)
    # one block: the global sweeps, n_t * n_k of them
    for kind, glob in ((oracle.PC_GS2, lambda x: oracle.gs2(pr.A, pr.b, x, outer=6, inner=2,
                                                             omega=0.9, direction=2)),
                       (oracle.PC_JR, lambda x: oracle.jr(pr.A, pr.b, x, sweeps=6, omega=0.9)),
                       (oracle.PC_GS, lambda x: oracle.gs(pr.A, pr.b, x, sweeps=6, omega=0.9,
                                                          direction=2))):
        got = oracle.hybrid(pr.A, pr.b, x0, kind, parts=1, outer=2, local=3, inner=2, omega=0.9,
                            direction=oracle.SYMMETRIC)
        assert np.abs(got - glob(x0)).max() <= 1e-14 * np.abs(got).max(), kind
    # one local sweep of JR per exchange is global JR, whatever the blocks
    for parts in (2, 5, 144):
        got = oracle.hybrid(pr.A, pr.b, x0, oracle.PC_JR, parts=parts, outer=4, local=1,
                            omega=0.7)
        want = oracle.jr(pr.A, pr.b, x0, sweeps=4, omega=0.7)
        assert np.allclose(got, want, rtol=0, atol=1e-14)
    # every row its own block: no local triangle, GS2 (and exact GS) is JR
    for kind in (oracle.PC_GS2, oracle.PC_GS):
        got = oracle.hybrid(pr.A, pr.b, x0, kind, parts=pr.n, outer=3, local=1, inner=2)
        want = oracle.jr(pr.A, pr.b, x0, sweeps=3, omega=1.0)
        assert np.allclose(got, want, rtol=0, atol=1e-14), kind


def test_hybrid_on_uncoupled_blocks_is_global():
    """Two uncoupled systems split exactly at their boundary: no couplings
    between blocks, so the hybrid sweep is the global one."""
    a, c = P.poisson2d(8), P.convdiff3d(4)
    Ma, Mc = P.csr_to_dense(a.A), P.csr_to_dense(c.A)
    M = np.zeros((a.n + c.n,) * 2)
    M[:a.n, :a.n], M[a.n:, a.n:] = Ma, Mc
    A = P.dense_to_csr(M)
    assert a.n == c.n  # 64 + 64 rows: two equal blocks
    b = np.concatenate([a.b, c.b])
    got = oracle.hybrid(A, b, np.zeros(len(b)), oracle.PC_GS2, parts=2, outer=2, local=1,
                        inner=3, direction=oracle.SYMMETRIC)
    want = oracle.gs2(A, b, np.zeros(len(b)), outer=2, inner=3, direction=oracle.SYMMETRIC)
    assert np.array_equal(got, want)


def test_hybrid_gs2_reaches_local_exact_gs_at_the_local_depth():
    """D_loc^{-1} L_loc is nilpotent: n_j at least the depth of the local
    triangles gives the local exact GS (the nilpotency limit of Sec. 4,
    block by block)."""
    pr = P.poisson2d(10)
    parts = 4
    depth = max(oracle.levels(P.dense_to_csr(np.where(
        _blocks(pr.n, parts)[:, None] == _blocks(pr.n, parts)[None, :],
        P.csr_to_dense(pr.A), 0.0)))[1], 1)
    x0 = P.uniform_pm1(9, pr.n)
    got = oracle.hybrid(pr.A, pr.b, x0, oracle.PC_GS2, parts=parts, outer=2, local=2,
                        inner=depth, direction=oracle.SYMMETRIC)
    want = oracle.hybrid(pr.A, pr.b, x0, oracle.PC_GS, parts=parts, outer=2, local=2,
                         direction=oracle.SYMMETRIC)
    assert np.allclose(got, want, rtol=0, atol=1e-13)
    less = oracle.hybrid(pr.A, pr.b, x0, oracle.PC_GS2, parts=parts, outer=2, local=2,
                         inner=depth - 3, direction=oracle.SYMMETRIC)
    assert np.abs(less - want).max() > 1e-8


def test_local_jr_iterations_grow_with_the_blocks_global_stay():
    """Sec. 8 strong scaling: GMRES with the global JR(4,1) takes the same
    iterations on any number of blocks; with the local JR(1,4) the count
    grows with the number of blocks."""
    pr = P.poisson2d(32)
    glob, loc = [], []
    for parts in (1, 4, 16):
        glob.append(oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, pc_kind=oracle.PC_HYBRID_JR,
                                 pc_outer=4, pc_parts=parts, pc_local=1)[1].iters)
        loc.append(oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, pc_kind=oracle.PC_HYBRID_JR,
                                pc_outer=1, pc_parts=parts, pc_local=4)[1].iters)
    assert glob[0] == glob[1] == glob[2]
    assert loc[0] == glob[0] and loc[0] < loc[1] < loc[2]


def test_openmp_build_is_bitwise_the_sequential_oracle():
    """The -fopenmp build of the oracle (the multi-core CPU timing) spreads
    only loops whose iterations write their own entry; it must give bitwise
    the results of the sequential build on a nonsymmetric system."""
    try:
        oracle.build(openmp=True)
    except Exception as e:  # a host compiler without OpenMP
        pytest.skip(f"no OpenMP build: {e}")
    pr = P.convdiff3d(12)
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-1, 1, pr.n)
    assert oracle.threads(openmp=False) == 1
    assert oracle.threads(openmp=True) >= 1
    for direction in (oracle.FORWARD, oracle.BACKWARD, oracle.SYMMETRIC):
        a = oracle.gs2(pr.A, pr.b, x0, 2, 2, 0.9, 0.8, direction)
        b = oracle.gs2(pr.A, pr.b, x0, 2, 2, 0.9, 0.8, direction, openmp=True)
        assert np.array_equal(a, b)
    assert np.array_equal(oracle.jr(pr.A, pr.b, x0, 3, 0.7),
                          oracle.jr(pr.A, pr.b, x0, 3, 0.7, openmp=True))
    assert np.array_equal(oracle.spmv(pr.A, x0), oracle.spmv(pr.A, x0, openmp=True))


# ---------------------------------------------------------------------------
# Lower-precision inner sweeps (Sec. 10; the FP16 row-scaled form of this
# library): IEEE binary16 rounding, exactness where every value is
# representable, the error bounds of the value precision, and the per-row
# scale that keeps FP16 in range
# ---------------------------------------------------------------------------

def test_round_half_is_ieee_binary16():
    rng = np.random.default_rng(3)
    v = np.concatenate([
        rng.choice([-1.0, 1.0], 4000) * 10.0 ** rng.uniform(-9, 5, 4000),
        [0.0, 1.0, 65504.0, 65519.99, 65520.0, 70000.0, 2.0 ** -24, 2.0 ** -25,
         3 * 2.0 ** -26, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25],
    ])
    # exact halfway points between consecutive binary16 values (ties to even)
    h = np.float16(rng.uniform(-1000, 1000, 2000))
    up = np.nextafter(h, np.float16(np.inf))
    mid = (h.astype(np.float64) + up.astype(np.float64)) / 2
    v = np.concatenate([v, mid])
    with np.errstate(over="ignore"):
        want = v.astype(np.float16).astype(np.float64)
    got = np.array([oracle.round_half(t) for t in v])
    assert np.array_equal(got, want)


def dyadic_nonsym_csr(N=6, seed=4):
    """A nonsymmetric 2D-pattern matrix with diagonal 16 and off-diagonals
    from {-1, -2, -4}: D^{-1}T entries are -1/16, -1/8, -1/4 and their ratio to
    the row maximum is a power of two, so every stored value is exact in
    FP32 and in row-scaled FP16."""
    rng = np.random.default_rng(seed)
    n = N * N
    M = np.zeros((n, n))
    for i in range(N):
        for j in range(N):
            r = i * N + j
            M[r, r] = 16.0
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                a, c = i + di, j + dj
                if 0 <= a < N and 0 <= c < N:
                    M[r, a * N + c] = -float(rng.choice([1, 2, 4]))
    return P.dense_to_csr(M), n


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_lowprec_gs2_exact_when_every_value_is_representable(prec):
    """With dyadic data whose every intermediate fits in 24 bits the
    lower-precision sweep performs exactly the FP64 sweep's arithmetic, so
    it must equal the FP64 oracle bitwise: a dropped row scale, a wrong
    triangle, sign or damping placement breaks the equality."""
    A, n = dyadic_nonsym_csr()
    rng = np.random.default_rng(8)
    b = rng.integers(-32, 33, n) / 16.0
    x0 = rng.integers(-64, 65, n) / 64.0
    for kw in (dict(outer=1, inner=2, omega=0.75, gamma=0.5, direction=oracle.FORWARD),
               dict(outer=1, inner=2, omega=1.0, gamma=1.0, direction=oracle.BACKWARD),
               dict(outer=1, inner=1, omega=1.0, gamma=1.0, direction=oracle.SYMMETRIC),
               dict(outer=1, inner=0, omega=0.5, gamma=1.0, direction=oracle.FORWARD)):
        ref = oracle.gs2(A, b, x0, **kw)
        got = oracle.gs2(A, b, x0, precision=prec, **kw)
        assert np.array_equal(got, ref), kw


def test_lowprec_gs2_error_within_the_value_precision():
    """Non-dyadic data: FP32 sweeps differ from FP64 by a few FP32 rounding
    units (u = 2^-24), FP16 values by a few FP16 units (2^-11), and both do
    differ (the rounding is really applied)."""
    A = tiny_nonsym(n=60, seed=12)
    rng = np.random.default_rng(2)
    b, x0 = rng.uniform(-1, 1, 60), rng.uniform(-1, 1, 60)
    for d in (oracle.FORWARD, oracle.SYMMETRIC):
        ref = oracle.gs2(A, b, x0, 1, 2, 0.9, 0.8, d)
        dx = np.linalg.norm(ref - x0)
        e32 = np.linalg.norm(oracle.gs2(A, b, x0, 1, 2, 0.9, 0.8, d, precision="fp32") - ref)
        e16 = np.linalg.norm(oracle.gs2(A, b, x0, 1, 2, 0.9, 0.8, d, precision="fp16") - ref)
        assert 1e-10 * dx < e32 < 40 * 2.0 ** -24 * dx
        assert 40 * 2.0 ** -24 * dx < e16 < 40 * 2.0 ** -11 * dx


def test_lowprec_fp16_row_scale_keeps_far_out_of_range_values():
    """A 10x10 grid whose rows alternate (checkerboard) between a diagonal
    of the off-diagonal size and one 2^28 times larger: the heavy rows have
    prescaled entries D^{-1}T near 2^-28 = 3.7e-9, below binary16's
    smallest subnormal (6e-8), and couple to light rows whose iterates are
    2^28 times their own, so those couplings decide the heavy rows' result.
    Stored unscaled they would vanish; the per-row scale keeps them, so the
    FP16 sweep matches the FP64 sweep to FP16 accuracy (errors measured in
    the balanced quantity D x) in a forward sweep, while dropping the
    couplings (zero inner sweeps) is far off."""
    N = 10
    rng = np.random.default_rng(5)
    n = N * N
    M = np.zeros((n, n))
    for i in range(N):
        for j in range(N):
            r = i * N + j
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                a, c = i + di, j + dj
                if 0 <= a < N and 0 <= c < N:
                    M[r, a * N + c] = -rng.uniform(0.2, 1.0)
            M[r, r] = (np.abs(M[r]).sum() + 1.0) * (2.0 ** 28 if (i + j) % 2 else 1.0)
    d = np.diag(M).copy()
    A = P.dense_to_csr(M)
    b = rng.uniform(-1, 1, n)
    ref = oracle.gs2(A, b, np.zeros(n), 1, 2, 1.0, 1.0, oracle.FORWARD)
    got = oracle.gs2(A, b, np.zeros(n), 1, 2, 1.0, 1.0, oracle.FORWARD, precision="fp16")
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(d * (got - ref)) <= 5e-3 * np.linalg.norm(d * ref)
    jr = oracle.gs2(A, b, np.zeros(n), 1, 0, 1.0, 1.0, oracle.FORWARD)
    assert np.linalg.norm(d * (jr - ref)) >= 0.1 * np.linalg.norm(d * ref)


def test_lowprec_gmres_keeps_the_iteration_count():
    """Sec. 10: a single-precision preconditioner leaves the GMRES iteration
    count of the double-precision solve essentially unchanged; the FP16
    row-scaled form stays close as well on a well-conditioned problem."""
    pr = P.poisson2d(48)
    _, i64 = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=3000,
                          pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC)
    for prec, slack in (("fp32", 1), ("fp16", 3)):
        x, i = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=3000,
                            pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC,
                            pc_precision=prec)
        assert i.status == 0 and abs(i.iters - i64.iters) <= slack, (prec, i, i64)
        r = np.linalg.norm(pr.b - oracle.spmv(pr.A, x)) / np.linalg.norm(pr.b)
        assert r <= 1e-8


# ---------------------------------------------------------------------------
# Whole-sweep single precision (Sec. 10: the outer GS iteration in single
# precision as well): residual, inner sweeps and iterate in FP32
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["fp32_sweep", "fp16_sweep"])
def test_sweep_precision_exact_when_every_value_is_representable(prec):
    """Dyadic data whose every intermediate (FP32 residual from the
    prescaled off-diagonal values, inner sweeps, FP32 iterate) fits in 24
    bits: the single-precision sweep performs the FP64 sweep's arithmetic
    exactly and must equal it bitwise; a dropped x or D^{-1}b term, a wrong
    sign, a wrong triangle or scale breaks the equality."""
    A, n = dyadic_nonsym_csr()
    rng = np.random.default_rng(8)
    b = rng.integers(-32, 33, n) / 16.0
    x0 = rng.integers(-64, 65, n) / 64.0
    for kw in (dict(outer=1, inner=2, omega=1.0, gamma=1.0, direction=oracle.BACKWARD),
               dict(outer=1, inner=1, omega=1.0, gamma=1.0, direction=oracle.SYMMETRIC),
               dict(outer=1, inner=0, omega=0.5, gamma=1.0, direction=oracle.FORWARD),
               dict(outer=2, inner=0, omega=1.0, gamma=1.0, direction=oracle.SYMMETRIC)):
        ref = oracle.gs2(A, b, x0, **kw)
        got = oracle.gs2(A, b, x0, precision=prec, **kw)
        assert np.array_equal(got, ref), kw


def test_sweep_precision_error_within_the_value_precision():
    """Non-dyadic data: the whole single-precision sweep differs from FP64
    by a few units of 2^-24 (FP32 values) or 2^-11 (FP16 values), and does
    differ."""
    A = tiny_nonsym(n=60, seed=12)
    rng = np.random.default_rng(2)
    b, x0 = rng.uniform(-1, 1, 60), rng.uniform(-1, 1, 60)
    for d in (oracle.FORWARD, oracle.SYMMETRIC):
        ref = oracle.gs2(A, b, x0, 1, 2, 0.9, 0.8, d)
        dx = np.linalg.norm(ref - x0)
        e32 = np.linalg.norm(oracle.gs2(A, b, x0, 1, 2, 0.9, 0.8, d, precision="fp32_sweep")
                             - ref)
        e16 = np.linalg.norm(oracle.gs2(A, b, x0, 1, 2, 0.9, 0.8, d, precision="fp16_sweep")
                             - ref)
        assert 1e-10 * dx < e32 < 40 * 2.0 ** -24 * dx
        assert 40 * 2.0 ** -24 * dx < e16 < 40 * 2.0 ** -11 * dx


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_sweep_precision_from_zero_equals_inner_only_form(prec):
    """One half sweep from x = 0 with omega = 1: the residual is b in both
    forms, the inner sweeps are the same FP32 ones, and x = 1 * g is exact in
    FP32 and FP64 alike, so the whole-sweep form equals the inner-only form
    of the same value precision bitwise."""
    pr = P.poisson2d(20)
    for d in (oracle.FORWARD, oracle.BACKWARD):
        a = oracle.gs2(pr.A, pr.b, np.zeros(pr.n), 1, 2, 1.0, 0.7, d, precision=prec)
        c = oracle.gs2(pr.A, pr.b, np.zeros(pr.n), 1, 2, 1.0, 0.7, d, precision=prec + "_sweep")
        assert np.array_equal(a, c)


def test_sweep_precision_gmres_keeps_the_iteration_count():
    """Sec. 10: the single-precision preconditioner keeps the count."""
    pr = P.poisson2d(48)
    _, i64 = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=3000,
                          pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC)
    for prec, slack in (("fp32_sweep", 1), ("fp16_sweep", 3)):
        x, i = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=3000,
                            pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC,
                            pc_precision=prec)
        assert i.status == 0 and abs(i.iters - i64.iters) <= slack, (prec, i, i64)
        r = np.linalg.norm(pr.b - oracle.spmv(pr.A, x)) / np.linalg.norm(pr.b)
        assert r <= 1e-8

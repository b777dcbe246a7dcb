"""Seeded synthetic inputs shaped like the paper's model problems.

This module is the one place both the GPU library's tests/benchmark and the
FP64 oracle take their inputs from.  It builds matrices and vectors only; it
holds none of the relaxation or Krylov arithmetic.

Random numbers come from SplitMix64 used as a counter-based generator
(Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): draw i of stream (seed) is mix(seed + (i + 1) * 0x9E3779B97F4A7C15)
with the published 64-bit finaliser; U[0,1) takes the top 53 bits.

Matrices are CSR tuples ``(rowptr int64[n+1], col int32[nnz], val float64[nnz])``
with ascending columns inside each row unless a builder says otherwise.

Model problems (the paper's Laplace and elasticity problems come from a
Galeri-style generator whose scaling and ordering it does not print):
  * 2D 5-point and 3D 7-point Laplacians, unscaled stencil (diagonal 4 or 6,
    off-diagonals -1), lexicographic ordering with x fastest, Dirichlet
    boundary nodes eliminated;
  * 3D trilinear (Q1) hexahedral linear elasticity, 3 dof per node
    interleaved, 2x2x2 Gauss quadrature, one face clamped;
  * 3D first-order upwind convection-diffusion with a rotating wind and a
    lognormal cell Peclet number, plus a mass term (a momentum-like system);
  * variable-coefficient Poisson / convection-diffusion for request streams.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20210403
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# --------------------------------------------------------------------------
# Counter-based random numbers
# --------------------------------------------------------------------------

def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+count-1 of the SplitMix64 stream for `seed`."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """U[-1, 1) from the seeded stream (the configs' x_true)."""
    return 2.0 * uniform01(seed, count) - 1.0


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on two interleaved uniform draws."""
    u = uniform01(seed, 2 * count)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------
# CSR helpers (input construction only)
# --------------------------------------------------------------------------

@dataclass
class Problem:
    """A linear system A x = b with the recipe that produced it."""
    name: str
    A: tuple
    b: np.ndarray
    x_true: np.ndarray | None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A[0].shape[0] - 1

    @property
    def nnz(self) -> int:
        return int(self.A[0][-1])


def csr_matvec(A, x):
    """b = A x, used only to form right-hand sides b = A x_true."""
    rp, ci, va = A
    n = rp.shape[0] - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    return np.bincount(rows, weights=va * x[ci], minlength=n)


def csr_to_dense(A):
    rp, ci, va = A
    n = rp.shape[0] - 1
    M = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(M, (rows, ci), va)
    return M


def dense_to_csr(M, keep_zero_diag=True):
    n = M.shape[0]
    rp = [0]
    ci, va = [], []
    for i in range(n):
        for j in range(n):
            if M[i, j] != 0.0 or (keep_zero_diag and i == j):
                ci.append(j)
                va.append(M[i, j])
        rp.append(len(ci))
    return (np.array(rp, dtype=np.int64), np.array(ci, dtype=np.int32),
            np.array(va, dtype=np.float64))


def _stencil_csr(dims, offsets, values):
    """Structured-grid operator in CSR.

    dims = (nx, ny, nz) with x fastest; offsets = list of (dx, dy, dz);
    values = list of scalars or per-row arrays, one per offset.  Neighbours
    outside the grid are dropped (Dirichlet elimination).  Offsets are sorted
    by linear distance so columns ascend inside each row.
    """
    nx, ny, nz = dims
    n = nx * ny * nz
    lin = [dz * nx * ny + dy * nx + dx for dx, dy, dz in offsets]
    order = np.argsort(lin, kind="stable")
    idx = np.arange(n, dtype=np.int64)
    ix = idx % nx
    iy = (idx // nx) % ny
    iz = idx // (nx * ny)
    S = len(offsets)
    mask = np.empty((n, S), dtype=bool)
    cols = np.empty((n, S), dtype=np.int64)
    vals = np.empty((n, S), dtype=np.float64)
    for s, o in enumerate(order):
        dx, dy, dz = offsets[o]
        m = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
             & (iz + dz >= 0) & (iz + dz < nz))
        mask[:, s] = m
        cols[:, s] = idx + lin[o]
        v = values[o]
        vals[:, s] = v if np.isscalar(v) else np.asarray(v, dtype=np.float64)
    counts = mask.sum(axis=1)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    ci = cols[mask].astype(np.int32)
    va = vals[mask]
    return rp, ci, va


def _rhs_problem(name, A, seed, meta):
    n = A[0].shape[0] - 1
    x_true = uniform_pm1(seed, n)
    return Problem(name, A, csr_matvec(A, x_true), x_true, dict(meta, seed=seed))


# --------------------------------------------------------------------------
# Laplacians
# --------------------------------------------------------------------------

def poisson2d_matrix(N: int):
    offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    vals = [-1.0, -1.0, 4.0, -1.0, -1.0]
    return _stencil_csr((N, N, 1), offs, vals)


def poisson3d_matrix(N: int):
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0),
            (0, 0, 1)]
    vals = [-1.0, -1.0, -1.0, 6.0, -1.0, -1.0, -1.0]
    return _stencil_csr((N, N, N), offs, vals)


def poisson2d(N: int = 64, seed: int = SEED_BASE) -> Problem:
    """2D 5-point Poisson on an N x N interior grid, b = A x_true."""
    return _rhs_problem(f"poisson2d_{N}", poisson2d_matrix(N), seed,
                        dict(kind="poisson2d", N=N))


def poisson3d(N: int = 128, seed: int = SEED_BASE) -> Problem:
    """3D 7-point Laplacian on an N^3 interior grid, b = A x_true."""
    return _rhs_problem(f"poisson3d_{N}", poisson3d_matrix(N), seed,
                        dict(kind="poisson3d", N=N))


# --------------------------------------------------------------------------
# Convection-diffusion (nonsymmetric)
# --------------------------------------------------------------------------

def _cell_centres(dims):
    nx, ny, nz = dims
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = ((idx % nx) + 0.5) / nx
    y = (((idx // nx) % ny) + 0.5) / ny
    z = ((idx // (nx * ny)) + 0.5) / nz
    return x, y, z


def _face_kappa(kappa, dims):
    """Harmonic-mean face coefficients per direction and side.

    Returns dict (axis, side) -> per-row face coefficient, with the missing
    neighbour at a Dirichlet boundary taking the cell's own kappa.
    """
    nx, ny, nz = dims
    K = kappa.reshape(nz, ny, nx)
    out = {}
    for axis, arr_axis in ((0, 2), (1, 1), (2, 0)):
        for side in (-1, 1):
            nb = np.roll(K, -side, axis=arr_axis)
            # boundary: neighbour wraps around -> replace with own value
            sl = [slice(None)] * 3
            sl[arr_axis] = slice(-1, None) if side == 1 else slice(0, 1)
            nb = nb.copy()
            nb[tuple(sl)] = K[tuple(sl)]
            out[(axis, side)] = (2.0 * K * nb / (K + nb)).reshape(-1)
    return out


def convdiff_matrix(dims, pe, wind, kappa=None, mass=1.0):
    """First-order upwind convection-diffusion, h^2-scaled.

    Row i: diagonal = sum of diffusion face coefficients + sum_d |p_d| + mass;
    the upwind neighbour in direction d gets -k_face - |p_d|, the downwind one
    -k_face, with p_d = 2 Pe_i w_d (h |w| = 2 Pe for unit viscosity).
    """
    nx, ny, nz = dims
    n = nx * ny * nz
    kap = np.ones(n) if kappa is None else kappa
    fk = _face_kappa(kap, dims)
    p = [2.0 * pe * wind[d] for d in range(3)]
    offs, vals = [], []
    diag = np.full(n, float(mass))
    for d in range(3):
        if dims[d] == 1:
            continue
        for side in (-1, 1):
            o = [0, 0, 0]
            o[d] = side
            # flow in +d (p_d > 0): upwind neighbour is side -1
            upwind = (p[d] > 0) if side == -1 else (p[d] < 0)
            v = -fk[(d, side)] - np.where(upwind, np.abs(p[d]), 0.0)
            offs.append(tuple(o))
            vals.append(v)
            diag += fk[(d, side)]
        diag += np.abs(p[d])
    offs.append((0, 0, 0))
    vals.append(diag)
    return _stencil_csr(dims, offs, vals)


def rotating_wind(dims):
    """Unit wind w = normalise(-(y - 1/2), x - 1/2, 0.2) at cell centres."""
    x, y, _ = _cell_centres(dims)
    w = np.stack([-(y - 0.5), x - 0.5, np.full_like(x, 0.2)])
    return w / np.linalg.norm(w, axis=0)


def lognormal_peclet(seed, n, lo=0.1, hi=10.0):
    """Cell Peclet ~ lognormal(0, ln(10)/2) clipped to [lo, hi]."""
    return np.clip(np.exp(normal(seed, n) * (math.log(10.0) / 2.0)), lo, hi)


def convdiff3d(N: int = 192, seed: int = SEED_BASE, mass: float = 1.0) -> Problem:
    """3D upwind convection-diffusion, rotating wind, lognormal Peclet."""
    dims = (N, N, N)
    n = N ** 3
    pe = lognormal_peclet(seed + 7919, n)
    A = convdiff_matrix(dims, pe, rotating_wind(dims), None, mass)
    return _rhs_problem(f"convdiff3d_{N}", A, seed,
                        dict(kind="convdiff3d", N=N, mass=mass))


# --------------------------------------------------------------------------
# Q1 hexahedral linear elasticity
# --------------------------------------------------------------------------

def _elasticity_D(E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    return D


def q1_element_stiffness(h: float, E: float = 1.0, nu: float = 0.3):
    """24x24 stiffness of a cube of side h, trilinear shape functions,
    2x2x2 Gauss.  Local node a = ax + 2 ay + 4 az with corner (ax, ay, az);
    dof 3a + c for displacement component c."""
    D = _elasticity_D(E, nu)
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)],
                       dtype=np.float64)
    s = 2.0 * corners - 1.0  # sign of xi at each node
    g = 1.0 / math.sqrt(3.0)
    Ke = np.zeros((24, 24))
    jac = h / 2.0
    for gx in (-g, g):
        for gy in (-g, g):
            for gz in (-g, g):
                xi = np.array([gx, gy, gz])
                # dN_a/dxi_k
                dN = np.empty((8, 3))
                for a in range(8):
                    f = 1.0 + s[a] * xi
                    dN[a, 0] = s[a, 0] * f[1] * f[2] / 8.0
                    dN[a, 1] = f[0] * s[a, 1] * f[2] / 8.0
                    dN[a, 2] = f[0] * f[1] * s[a, 2] / 8.0
                dNx = dN / jac
                B = np.zeros((6, 24))
                for a in range(8):
                    bx, by, bz = dNx[a]
                    B[0, 3 * a + 0] = bx
                    B[1, 3 * a + 1] = by
                    B[2, 3 * a + 2] = bz
                    B[3, 3 * a + 0] = by
                    B[3, 3 * a + 1] = bx
                    B[4, 3 * a + 1] = bz
                    B[4, 3 * a + 2] = by
                    B[5, 3 * a + 0] = bz
                    B[5, 3 * a + 2] = bx
                Ke += B.T @ D @ B * (jac ** 3)
    return Ke


def elasticity_matrix(Nn: int, E: float = 1.0, nu: float = 0.3, clamp=True):
    """Assembled Q1 stiffness on an Nn^3-node unit cube, dofs interleaved.

    Assembly is done per node-pair offset: the 3x3 block coupling node p to
    node p + d sums, over the elements holding both, the element block
    Ke[c, c + d] where c is p's corner in that element.  With clamp=True the
    dofs of the x = 0 face become identity rows and their couplings are
    removed from every other row and column.
    """
    h = 1.0 / (Nn - 1)
    Ke = q1_element_stiffness(h, E, nu)
    nnode = Nn ** 3
    idx = np.arange(nnode, dtype=np.int64)
    ix, iy, iz = idx % Nn, (idx // Nn) % Nn, idx // (Nn * Nn)
    ne = Nn - 1
    offsets = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    blocks = np.zeros((nnode, 27, 3, 3))
    present = np.zeros((nnode, 27), dtype=bool)
    for s, (dx, dy, dz) in enumerate(offsets):
        for a in range(8):
            c = (a & 1, (a >> 1) & 1, (a >> 2) & 1)
            cd = (c[0] + dx, c[1] + dy, c[2] + dz)
            if min(cd) < 0 or max(cd) > 1:
                continue
            a2 = cd[0] + 2 * cd[1] + 4 * cd[2]
            ex, ey, ez = ix - c[0], iy - c[1], iz - c[2]
            m = (ex >= 0) & (ex < ne) & (ey >= 0) & (ey < ne) & (ez >= 0) & (ez < ne)
            blocks[m, s] += Ke[3 * a:3 * a + 3, 3 * a2:3 * a2 + 3]
            present[m, s] = True
    nb = idx[:, None] + np.array([dz * Nn * Nn + dy * Nn + dx for dx, dy, dz in offsets])
    clamped = (ix == 0)
    if clamp:
        # remove couplings to clamped nodes; clamped rows become identity
        nbc = np.where(present, nb, 0)
        present &= ~clamped[nbc]
        present[clamped] = False
        centre = offsets.index((0, 0, 0))
        present[clamped, centre] = True
        blocks[clamped, centre] = np.eye(3)
    # rows: dof 3p + r; entries over neighbours in ascending node order,
    # 3 columns each -> ascending columns
    n = 3 * nnode
    cnt_node = present.sum(axis=1) * 3
    counts = np.repeat(cnt_node, 3)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    # (node, r, s, c) ordering
    pres4 = np.broadcast_to(present[:, None, :, None], (nnode, 3, 27, 3))
    cols4 = (3 * nb[:, None, :, None] + np.arange(3)[None, None, None, :])
    cols4 = np.broadcast_to(cols4, (nnode, 3, 27, 3))
    vals4 = blocks.transpose(0, 2, 1, 3)  # (node, r, s, c)
    ci = cols4[pres4].astype(np.int32)
    va = vals4[pres4].astype(np.float64)
    return (rp, ci, va), clamped


def elasticity_body_load(Nn: int, clamped, f=(0.0, 0.0, -1.0)):
    """Consistent nodal load of a uniform body force: each element gives
    h^3/8 f to each of its 8 nodes; clamped dofs get 0."""
    h = 1.0 / (Nn - 1)
    idx = np.arange(Nn ** 3)
    ix, iy, iz = idx % Nn, (idx // Nn) % Nn, idx // (Nn * Nn)

    def cnt(i):
        return np.where((i == 0) | (i == Nn - 1), 1, 2)

    nel = cnt(ix) * cnt(iy) * cnt(iz)
    b = (nel[:, None] * (h ** 3 / 8.0) * np.asarray(f)[None, :]).reshape(-1)
    b[np.repeat(clamped, 3)] = 0.0
    return b


def elasticity3d(Nn: int = 64, E: float = 1.0, nu: float = 0.3) -> Problem:
    """Q1 elasticity, Nn^3 nodes, face x=0 clamped, uniform body load."""
    A, clamped = elasticity_matrix(Nn, E, nu)
    b = elasticity_body_load(Nn, clamped)
    return Problem(f"elasticity3d_{Nn}", A, b, None,
                   dict(kind="elasticity3d", Nn=Nn, E=E, nu=nu))


# --------------------------------------------------------------------------
# Random matrices for kernel edge cases
# --------------------------------------------------------------------------

def random_csr(n: int, seed: int, mean_offdiag: float = 4.0, long_rows=(),
               empty_frac: float = 0.1, shuffle: bool = True, dominance: float = 1.0,
               symmetric_pattern: bool = False):
    """Random nonsymmetric CSR with a nonzero diagonal.

    Row lengths are random (about `mean_offdiag` off-diagonals), a fraction
    `empty_frac` of rows has no off-diagonal at all, rows listed in
    `long_rows` as (row, length) get that many off-diagonals.  Diagonal =
    dominance * sum|offdiag| + 1, so dominance >= 1 gives a diagonally
    dominant matrix.  shuffle=True leaves columns unsorted inside rows.
    """
    u = uniform01(seed, 4 * n + 16)
    lens = np.floor(u[:n] * 2.0 * mean_offdiag).astype(np.int64)
    lens[u[n:2 * n] < empty_frac] = 0
    for r, L in long_rows:
        lens[r] = L
    lens = np.minimum(lens, max(n - 1, 0))
    total = int(lens.sum())
    draws = splitmix64(seed + 1, max(total, 1))
    vals_u = uniform01(seed + 2, max(total, 1))
    rows_c, rows_v = [], []
    pos = 0
    for i in range(n):
        L = int(lens[i])
        if L == 0:
            rows_c.append(np.empty(0, dtype=np.int64))
            rows_v.append(np.empty(0))
            continue
        c = (draws[pos:pos + L] % np.uint64(max(n - 1, 1))).astype(np.int64)
        c = np.where(c >= i, c + 1, c)
        c = np.unique(c)
        v = -(0.2 + vals_u[pos:pos + c.size])
        rows_c.append(c)
        rows_v.append(v)
        pos += L
    if symmetric_pattern:
        M = {}
        for i in range(n):
            for c, v in zip(rows_c[i], rows_v[i]):
                M[(i, int(c))] = v
                M.setdefault((int(c), i), v * 0.7)
        rows_c = [[] for _ in range(n)]
        rows_v = [[] for _ in range(n)]
        for (i, c), v in sorted(M.items()):
            rows_c[i].append(c)
            rows_v[i].append(v)
        rows_c = [np.array(c, dtype=np.int64) for c in rows_c]
        rows_v = [np.array(v) for v in rows_v]
    rp = np.zeros(n + 1, dtype=np.int64)
    ci_all, va_all = [], []
    perm_u = uniform01(seed + 3, n + total + 8)
    for i in range(n):
        c = np.append(rows_c[i], i)
        v = np.append(rows_v[i], dominance * np.abs(rows_v[i]).sum() + 1.0)
        if shuffle and c.size > 1:
            key = perm_u[i:i + c.size] + np.arange(c.size) * 1e-9
            o = np.argsort(key)
            c, v = c[o], v[o]
        ci_all.append(c)
        va_all.append(v)
        rp[i + 1] = rp[i] + c.size
    return (rp, np.concatenate(ci_all).astype(np.int32) if n else np.empty(0, np.int32),
            np.concatenate(va_all) if n else np.empty(0))


def random_system(n: int, seed: int, **kw) -> Problem:
    A = random_csr(n, seed, **kw)
    return _rhs_problem(f"random_{n}_{seed}", A, seed + 11, dict(kind="random", n=n))


# --------------------------------------------------------------------------
# Request streams for the solve server
# --------------------------------------------------------------------------

@dataclass
class Request:
    arrival_s: float
    problem: Problem


def variable_coefficient_problem(kind: str, N: int, seed: int) -> Problem:
    """Poisson (2D/3D) or 3D convection-diffusion with per-cell diffusion
    kappa ~ lognormal(0, 1), face values by harmonic mean."""
    if kind == "poisson2d":
        dims = (N, N, 1)
    else:
        dims = (N, N, N)
    n = dims[0] * dims[1] * dims[2]
    kappa = np.exp(normal(seed + 101, n))
    if kind == "convdiff3d":
        pe = lognormal_peclet(seed + 103, n)
        A = convdiff_matrix(dims, pe, rotating_wind(dims), kappa, mass=1.0)
    else:
        A = convdiff_matrix(dims, np.zeros(n), np.zeros((3, n)), kappa, mass=0.0)
    return _rhs_problem(f"{kind}_{N}_k", A, seed, dict(kind=kind, N=N, variable=True))


def request_stream(count: int = 2000, rate_hz: float = 200.0, seed: int = SEED_BASE,
                   n_lo: float = 1e3, n_hi: float = 2e6, build=True):
    """Poisson arrivals at `rate_hz`; type uniform over {2D Poisson, 3D
    Poisson, 3D convection-diffusion}; n log-uniform in [n_lo, n_hi], shaped
    to N = round(n^(1/2)) or round(n^(1/3)).  With build=False only the
    (arrival, kind, N, seed) recipe is returned."""
    u = uniform01(seed + 5, 3 * count)
    gaps = -np.log(1.0 - u[0::3]) / rate_hz
    arrivals = np.cumsum(gaps)
    kinds = np.array(["poisson2d", "poisson3d", "convdiff3d"])[
        np.minimum((u[1::3] * 3).astype(int), 2)]
    logn = math.log(n_lo) + u[2::3] * (math.log(n_hi) - math.log(n_lo))
    nn = np.exp(logn)
    out = []
    for i in range(count):
        kind = str(kinds[i])
        N = int(round(nn[i] ** (0.5 if kind == "poisson2d" else 1.0 / 3.0)))
        N = max(N, 4)
        rec = (float(arrivals[i]), kind, N, seed + i)
        if build:
            out.append(Request(rec[0], variable_coefficient_problem(kind, N, seed + i)))
        else:
            out.append(rec)
    return out


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

def workload(name: str) -> Problem:
    """Named configurations of the model problems at full size."""
    if name == "poisson2d_64":
        return poisson2d(64)
    if name == "poisson3d_128":
        return poisson3d(128)
    if name == "elasticity3d_64":
        return elasticity3d(64)
    if name == "convdiff3d_192":
        return convdiff3d(192)
    raise KeyError(name)

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Floating-point tolerance: the GPU reduces each row in a different order
than the oracle (segments, FMA) and multiplies by a precomputed D^{-1}
where the oracle divides, so a sweep differs by a few ulps per entry; one
FP64 sweep must agree to ||x_gpu - x_ora|| / ||x_ora|| <= 1e-12.  GMRES
iteration counts must agree to +-1 at the same tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2104_01196_gb300 import problems as P

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def g():
    import torch  # noqa: F401

    from paper_2104_01196_gb300 import build as B
    B.build()
    import paper_2104_01196_gb300 as gs2
    gs2.load()
    return gs2


def dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# matrices spanning the kernels' cases: several tiles and a ragged tail,
# unsorted columns, rows without off-diagonals, rows longer than 32, 128,
# 1024 entries, a row longer than one staged tile (6144 entries)
def case_matrices():
    out = {
        "poisson2d_37": P.poisson2d_matrix(37),
        "poisson3d_11": P.poisson3d_matrix(11),
        "random_5000": P.random_csr(5000, 3, mean_offdiag=5.0,
                                    long_rows=[(17, 40), (400, 200), (4999, 1500)]),
        # one row with ~9000 distinct entries: processed by the long-row path
        "random_long": P.random_csr(20000, 5, mean_offdiag=3.0, long_rows=[(15000, 12000)]),
        # mean row lengths that select 2, 4, 8 and 16 lanes per row
        "rows_35": P.random_csr(2000, 6, mean_offdiag=35.0, empty_frac=0.0),
        "wide_rows": P.random_csr(3000, 8, mean_offdiag=60.0, empty_frac=0.0),
        "rows_150": P.random_csr(1500, 9, mean_offdiag=150.0, empty_frac=0.0),
        "rows_300": P.random_csr(1200, 10, mean_offdiag=300.0, empty_frac=0.0),
        "n1": (np.array([0, 1]), np.array([0], np.int32), np.array([3.0])),
        "n7": P.random_csr(7, 2, mean_offdiag=2.0),
    }
    A, _ = P.elasticity_matrix(6)
    out["elasticity_6"] = A
    return out


MATS = case_matrices()


def rhs_and_x0(A, seed):
    n = len(A[0]) - 1
    return P.uniform_pm1(seed, n), P.uniform_pm1(seed + 1, n)


@pytest.mark.parametrize("name", list(MATS))
def test_spmv(g, name):
    A = MATS[name]
    x, _ = rhs_and_x0(A, 3)
    h = g.gs2_setup(A)
    y = dev(np.zeros(len(x)))
    g.gs2_spmv(h, dev(x), y)
    assert rel(host(y), oracle.spmv(A, x)) <= TOL


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_gs2_sweeps(g, name, direction):
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 11)
    h = g.gs2_setup(A)
    for outer, inner, omega in ((1, 1, 1.0), (2, 3, 0.8), (1, 0, 1.0), (1, 2, 1.2)):
        x = dev(x0)
        g.gs2_apply(h, dev(b), x, outer, inner, omega, direction)
        ref = oracle.gs2(A, b, x0, outer, inner, omega, 1.0, direction)
        assert rel(host(x), ref) <= TOL, (outer, inner, omega)


@pytest.mark.parametrize("gamma", [0.6, 1.3])
def test_gs2_inner_damping(g, gamma):
    A = MATS["random_5000"]
    b, x0 = rhs_and_x0(A, 12)
    h = g.gs2_setup(A)
    p = g.params("gs2", outer=2, inner=3, omega=0.9, gamma=gamma, direction="symmetric")
    x = dev(x0)
    g.gs2_apply_ex(h, dev(b), x, p)
    assert rel(host(x), oracle.gs2(A, b, x0, 2, 3, 0.9, gamma, oracle.SYMMETRIC)) <= TOL


@pytest.mark.parametrize("name", ["poisson2d_37", "random_5000", "elasticity_6"])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_compact_gs2(g, name, direction):
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 13)
    h = g.gs2_setup(A)
    p = g.params("gs2", outer=2, inner=2, direction=direction, form="compact")
    x = dev(x0)
    g.gs2_apply_ex(h, dev(b), x, p)
    assert rel(host(x), oracle.gs2_compact(A, b, x0, 2, 2, direction)) <= TOL


@pytest.mark.parametrize("name", ["poisson2d_37", "poisson3d_11", "random_5000", "n1", "n7",
                                  "elasticity_6"])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_level_scheduled_gs(g, name, direction):
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 17)
    h = g.gs2_setup(A)
    for omega in (1.0, 0.7):
        x = dev(x0)
        g.gs_apply(h, dev(b), x, 2, omega, direction)
        assert rel(host(x), oracle.gs(A, b, x0, 2, omega, direction)) <= TOL
    st = h.stats()
    _, nl = oracle.levels(A, True)
    _, nu = oracle.levels(A, False)
    assert (st["levels_lower"], st["levels_upper"]) == (nl, nu)


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_multicolor_gs(g, name, direction):
    """Multicolour GS/SOR (Sec. 6.1.2): same colouring as the oracle's first
    fit, sweeps equal to the oracle's colour-by-colour recurrence."""
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 29)
    h = g.gs2_setup(A)
    assert h.stats()["colors"] == 0
    for sweeps, omega in ((2, 1.0), (1, 0.7), (2, 1.2)):
        x = dev(x0)
        g.mtgs_apply(h, dev(b), x, sweeps, omega, direction)
        assert rel(host(x), oracle.mtgs(A, b, x0, sweeps, omega, direction)) <= TOL
    assert h.stats()["colors"] == oracle.coloring(A)[1]


@pytest.mark.parametrize("name", list(MATS))
def test_jr(g, name):
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 19)
    h = g.gs2_setup(A)
    for sweeps, omega in ((1, 1.0), (3, 0.8), (4, 0.6)):
        x = dev(x0)
        g.jr_apply(h, dev(b), x, sweeps, omega)
        assert rel(host(x), oracle.jr(A, b, x0, sweeps, omega)) <= TOL


def test_deep_inner_sweeps_reproduce_exact_gs_on_gpu(g):
    """With n_j = depth(L) the GPU's GS2 equals the oracle's exact GS."""
    A = P.poisson2d_matrix(16)
    b, x0 = rhs_and_x0(A, 23)
    h = g.gs2_setup(A)
    x = dev(x0)
    g.gs2_apply(h, dev(b), x, 1, 30, 1.0, 0)
    assert rel(host(x), oracle.gs(A, b, x0, 1, 1.0, 0)) <= TOL


def test_host_vectors_match_device_vectors(g):
    A = MATS["poisson3d_11"]
    b, x0 = rhs_and_x0(A, 29)
    h = g.gs2_setup(A)
    xd = dev(x0)
    g.gs2_apply(h, dev(b), xd, 1, 1, 1.0, 2)
    xh = x0.copy()
    g.gs2_apply(h, b.copy(), xh, 1, 1, 1.0, 2)
    assert np.array_equal(host(xd), xh)


def test_bitwise_reproducible(g):
    pr = P.poisson2d(64)
    h = g.gs2_setup(pr.A)
    outs = []
    for _ in range(2):
        x = dev(np.zeros(pr.n))
        g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 3000, g.params("gs2", 1, 1, direction=2))
        outs.append(host(x))
    assert np.array_equal(outs[0], outs[1])


# ---------------------------------------------------------------------------
# GMRES and CG
# ---------------------------------------------------------------------------

PCS = {
    "none": (None, dict(pc_kind=oracle.PC_NONE)),
    "gs2_fwd_1_1": (dict(kind="gs2", outer=1, inner=1), dict(pc_kind=oracle.PC_GS2)),
    "sgs2_1_2": (dict(kind="gs2", outer=1, inner=2, direction="symmetric"),
                 dict(pc_kind=oracle.PC_GS2, pc_inner=2, pc_direction=2)),
    "sgs2_damped": (dict(kind="gs2", outer=1, inner=1, omega=0.8, gamma=0.9,
                         direction="symmetric"),
                    dict(pc_kind=oracle.PC_GS2, pc_omega=0.8, pc_gamma=0.9, pc_direction=2)),
    "jr3": (dict(kind="jr", outer=3, omega=0.8), dict(pc_kind=oracle.PC_JR, pc_outer=3,
                                                      pc_omega=0.8)),
    "gs_sym": (dict(kind="gs", outer=1, direction="symmetric"),
               dict(pc_kind=oracle.PC_GS, pc_direction=2)),
    "mtsgs": (dict(kind="mtgs", outer=1, direction="symmetric"),
              dict(pc_kind=oracle.PC_MTGS, pc_direction=2)),
    "mtgs_2_w0.9": (dict(kind="mtgs", outer=2, omega=0.9),
                    dict(pc_kind=oracle.PC_MTGS, pc_outer=2, pc_omega=0.9)),
}


@pytest.mark.parametrize("pc", list(PCS))
def test_gmres_small_workload(g, pc):
    """2D 5-point Poisson 64x64, GMRES(30), rel. residual 1e-8."""
    pr = P.poisson2d(64)
    gp, op = PCS[pc]
    h = g.gs2_setup(pr.A)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, restart=30, tol=1e-8, max_iters=5000,
                         precond=g.params(**gp) if gp else None)
    xo, oinfo = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=5000, **op)
    assert info.status == 0 and oinfo.status == 0
    assert abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)
    assert info.true_relres <= 1e-8
    xg = host(x)
    # independent check of the reported residual
    assert np.linalg.norm(pr.b - oracle.spmv(pr.A, xg)) / np.linalg.norm(pr.b) <= 1e-8
    assert rel(xg, xo) <= 1e-6


@pytest.mark.parametrize("restart", [1, 5, 64])
def test_gmres_restarts(g, restart):
    pr = P.random_system(3000, 31, mean_offdiag=6.0, dominance=1.05)
    h = g.gs2_setup(pr.A)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, restart=restart, tol=1e-10, max_iters=3000,
                         precond=g.params("gs2", 1, 1))
    _, oinfo = oracle.gmres(pr.A, pr.b, restart=restart, tol=1e-10, max_iters=3000,
                            pc_kind=oracle.PC_GS2)
    assert info.status == oinfo.status == 0
    assert abs(info.iters - oinfo.iters) <= 1
    assert info.cycles == oinfo.cycles or abs(info.iters - oinfo.iters) == 1


def test_gmres_statuses(g):
    pr = P.poisson2d(32)
    h = g.gs2_setup(pr.A)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, restart=10, tol=1e-12, max_iters=7)
    assert info.status == 5 and info.iters == 7
    b = pr.b.copy()
    b[5] = np.nan
    info = g.gmres_solve(h, dev(b), dev(np.zeros(pr.n)), restart=10, tol=1e-8, max_iters=50)
    assert info.status == 7
    x = dev(np.ones(pr.n))
    info = g.gmres_solve(h, dev(np.zeros(pr.n)), x, restart=10, tol=1e-8, max_iters=50)
    assert info.status == 0 and np.all(host(x) == 0.0)
    # warm start at the solution: zero iterations
    x = dev(pr.x_true)
    info = g.gmres_solve(h, dev(pr.b), x, restart=10, tol=1e-8, max_iters=50)
    assert info.status == 0 and info.iters == 0


def test_gmres_jr1_count_independent_of_omega(g):
    """Table ela3d-omega: JR(1) iteration counts do not depend on omega."""
    A, cl = P.elasticity_matrix(6)
    b = P.elasticity_body_load(6, cl)
    h = g.gs2_setup(A)
    counts = set()
    for om in (0.5, 0.8, 1.0, 1.4):
        info = g.gmres_solve(h, dev(b), dev(np.zeros(len(b))), restart=30, tol=1e-8,
                             max_iters=5000, precond=g.params("jr", 1, omega=om))
        assert info.status == 0
        counts.add(info.iters)
    assert len(counts) == 1


def test_cg_matches_oracle(g):
    pr = P.poisson2d(48)
    h = g.gs2_setup(pr.A)
    for gp, op in ((dict(kind="gs2", outer=1, inner=1, direction="symmetric"),
                    dict(pc_kind=oracle.PC_GS2, pc_direction=2)),
                   (dict(kind="mtgs", outer=1, direction="symmetric"),
                    dict(pc_kind=oracle.PC_MTGS, pc_direction=2)),
                   (None, dict(pc_kind=oracle.PC_NONE))):
        x = dev(np.zeros(pr.n))
        info = g.cg_solve(h, dev(pr.b), x, tol=1e-8, max_iters=5000,
                          precond=g.params(**gp) if gp else None)
        _, oinfo = oracle.cg(pr.A, pr.b, tol=1e-8, max_iters=5000, **op)
        assert info.status == 0 and abs(info.iters - oinfo.iters) <= 1, (info, oinfo)
        assert info.true_relres <= 1e-8


def test_batch_results_equal_alone(g):
    probs = [P.poisson2d(20), P.poisson3d(9), P.random_system(700, 41, dominance=1.1),
             P.poisson2d(45)]
    hs = [g.gs2_setup(p.A) for p in probs]
    import torch
    streams = [torch.cuda.Stream() for _ in probs]
    for h, s in zip(hs, streams):
        h.set_stream(s.cuda_stream)
    pc = g.params("gs2", 1, 1, direction="symmetric")
    alone = []
    for h, p in zip(hs, probs):
        x = dev(np.zeros(p.n))
        torch.cuda.synchronize()
        h.set_graph_mode(1)  # the cycle-graph path a batch runs (not the one-launch solver)
        info = g.gmres_solve(h, dev(p.b), x, 30, 1e-8, 3000, pc)
        h.set_graph_mode(0)
        alone.append((info, host(x)))
    bs = [dev(p.b) for p in probs]
    xs = [dev(np.zeros(p.n)) for p in probs]
    torch.cuda.synchronize()
    infos = g.gs2_batch_solve(hs, bs, xs, 30, 1e-8, 3000, pc)
    for (ia, xa), ib, xb in zip(alone, infos, xs):
        assert ib.status == 0 and ib.iters == ia.iters
        assert np.array_equal(xa, host(xb))


# ---------------------------------------------------------------------------
# lower-precision inner sweeps (Sec. 10; FP16 row-scaled is an extension)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,bound", [("fp32", 2e-6), ("fp16", 2e-2)])
def test_lowprec_sweep_error_vs_fp64_oracle(g, prec, bound):
    A = P.poisson3d_matrix(12)
    b, x0 = rhs_and_x0(A, 37)
    h = g.gs2_setup(A, precisions=(prec,))
    p = g.params("gs2", 1, 2, direction="symmetric", precision=prec)
    x = dev(x0)
    g.gs2_apply_ex(h, dev(b), x, p)
    ref = oracle.gs2(A, b, x0, 1, 2, 1.0, 1.0, oracle.SYMMETRIC)
    e = rel(host(x), ref)
    assert e <= bound, e


LOWPREC_TOL = 1e-6


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp32_sweep", "fp16_sweep"])
def test_lowprec_sweeps_match_lowprec_oracle(g, name, prec):
    """FP32 and row-scaled FP16 inner sweeps (FP64 residual, r-hat rounded to
    FP32, values in the sweep precision, FP32 accumulation), and the whole
    sweep in single precision (FP32 residual on the prescaled off-diagonal
    values and FP32 iterate as well), against the oracle's definition of the
    same precision: the two differ only in FP32 rounding order (FMA, the
    order of a row's partial sums), a few units of 2^-24 per sweep, so 1e-6
    relative per vector; every kernel path, direction and damping."""
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 11)
    h = g.gs2_setup(A, precisions=(prec,))
    for d in (0, 1, 2):
        for outer, inner, omega, gamma in ((1, 1, 1.0, 1.0), (2, 3, 0.8, 0.7), (1, 0, 1.0, 1.0),
                                           (1, 2, 1.2, 1.0)):
            x = dev(x0)
            g.gs2_apply_ex(h, dev(b), x, g.params("gs2", outer, inner, omega=omega, gamma=gamma,
                                                  direction=d, precision=prec))
            ref = oracle.gs2(A, b, x0, outer, inner, omega, gamma, d, precision=prec)
            assert rel(host(x), ref) <= LOWPREC_TOL, (d, outer, inner, omega, gamma)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "fp32_sweep", "fp16_sweep"])
def test_lowprec_preconditioner_keeps_convergence(g, prec):
    """Sec. 10: the single-precision preconditioner keeps the GMRES
    iteration count (6,656 = 6,656 in the paper's table)."""
    pr = P.poisson2d(64)
    h = g.gs2_setup(pr.A, precisions=(prec,))
    i64 = g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 30, 1e-8, 5000,
                        g.params("gs2", 1, 1, direction="symmetric"))
    x = dev(np.zeros(pr.n))
    ilo = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 5000,
                        g.params("gs2", 1, 1, direction="symmetric", precision=prec))
    assert ilo.status == 0 and ilo.true_relres <= 1e-8
    assert abs(ilo.iters - i64.iters) <= (1 if prec.startswith("fp32") else 3), \
        (ilo.iters, i64.iters)
    # and the oracle's count for the same precision
    _, oi = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=5000,
                         pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC, pc_precision=prec)
    assert abs(ilo.iters - oi.iters) <= 1, (ilo.iters, oi.iters)


# ---------------------------------------------------------------------------
# full-size workload: 3D 7-point Laplacian 128^3
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big():
    return P.poisson3d(128)


def test_full_size_sweeps_match_oracle(g, big):
    """One symmetric GS2(1,1) sweep, one JR sweep and one SpMV at n = 2.1M,
    compared with the oracle on every entry."""
    A, b = big.A, big.b
    x0 = P.uniform_pm1(43, big.n)
    h = g.gs2_setup(A)
    x = dev(x0)
    g.gs2_apply(h, dev(b), x, 1, 1, 1.0, 2)
    assert rel(host(x), oracle.gs2(A, b, x0, 1, 1, 1.0, 1.0, 2)) <= TOL
    x = dev(x0)
    g.jr_apply(h, dev(b), x, 1, 0.8)
    assert rel(host(x), oracle.jr(A, b, x0, 1, 0.8)) <= TOL
    y = dev(np.zeros(big.n))
    g.gs2_spmv(h, dev(x0), y)
    assert rel(host(y), oracle.spmv(A, x0)) <= TOL


def test_full_size_gmres_true_residual(g, big):
    """GMRES(30) + SGS2(1,1) to 1e-8 at n = 2.1M: the true residual,
    recomputed by the oracle's SpMV on the returned x, meets the tolerance."""
    h = g.gs2_setup(big.A)
    x = dev(np.zeros(big.n))
    info = g.gmres_solve(h, dev(big.b), x, 30, 1e-8, 3000,
                         g.params("gs2", 1, 1, direction="symmetric"))
    assert info.status == 0
    xg = host(x)
    r = np.linalg.norm(big.b - oracle.spmv(big.A, xg)) / np.linalg.norm(big.b)
    assert r <= 1e-8 and abs(r - info.true_relres) <= 1e-12
    assert rel(xg, big.x_true) <= 1e-3


def _oracle_counts():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_counts.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *kv = line.split()
            out[key] = dict(x.split("=") for x in kv)
    return out


FULL_PCS = {
    "sgs2_1_1": dict(kind="gs2", outer=1, inner=1, direction="symmetric"),
    "sgs2_1_2": dict(kind="gs2", outer=1, inner=2, direction="symmetric"),
    "sgs2_1_3": dict(kind="gs2", outer=1, inner=3, direction="symmetric"),
    "sgs_exact": dict(kind="gs", outer=1, direction="symmetric"),
    "jr3_w1.0": dict(kind="jr", outer=3, omega=1.0),
    "jr3_w0.8": dict(kind="jr", outer=3, omega=0.8),
    "mtsgs": dict(kind="mtgs", outer=1, direction="symmetric"),
    "amg_sgs2_1_1": dict(kind="amg", outer=1, inner=1, direction="symmetric"),
}


@pytest.mark.parametrize("pc", list(FULL_PCS))
def test_full_size_iteration_counts_match_oracle(g, big, pc):
    """3D Laplacian 128^3, GMRES(30) to 1e-8: the GPU's iteration count is
    within +-1 of the oracle's (stored by tests/golden/make_oracle_counts.py)."""
    ref = _oracle_counts()[f"poisson3d_128_gmres30_{pc}"]
    h = g.gs2_setup(big.A)
    x = dev(np.zeros(big.n))
    info = g.gmres_solve(h, dev(big.b), x, 30, 1e-8, 5000, g.params(**FULL_PCS[pc]))
    assert info.status == 0 and info.true_relres <= 1e-8
    assert abs(info.iters - int(ref["iters"])) <= 1, (info.iters, ref)


@pytest.mark.parametrize("name", ["poisson3d_11", "random_5000", "rows_35", "elasticity_6"])
def test_autotuned_shapes_keep_parity(g, name):
    """After the autotuner re-tiles A and the triangles, sweeps still match
    the oracle to 1e-12 and the chosen shapes are valid."""
    A = MATS[name]
    b, x0 = rhs_and_x0(A, 51)
    h = g.gs2_setup(A)
    h.autotune()
    st = h.stats()
    assert st["tpr_a"] in (1, 2, 4, 8, 16) and st["rpt_a"] in (1, 2)
    assert st["rpt_a"] == 1 or st["tpr_a"] <= 2
    for d in (0, 1, 2):
        x = dev(x0)
        g.gs2_apply(h, dev(b), x, 1, 2, 0.9, d)
        assert rel(host(x), oracle.gs2(A, b, x0, 1, 2, 0.9, 1.0, d)) <= TOL
    y = dev(np.zeros(len(b)))
    g.gs2_spmv(h, dev(x0), y)
    assert rel(host(y), oracle.spmv(A, x0)) <= TOL


@pytest.mark.parametrize("pc", ["sgs2_1_2", "jr3", "gs_sym", "mtsgs", "none"])
def test_graph_and_eager_cycles_agree_bitwise(g, pc):
    """Arnoldi steps replayed as a captured CUDA graph give the same bits as
    separate launches, also when a cached graph is reused for a new b."""
    pr = P.poisson2d(64)
    b2 = P.csr_matvec(pr.A, P.uniform_pm1(77, pr.n))
    gp, _ = PCS[pc]
    prm = g.params(**gp) if gp else None
    res = {}
    for mode in (1, 2):
        h = g.gs2_setup(pr.A)
        h.set_graph_mode(mode)
        for k, b in enumerate((pr.b, b2)):
            x = dev(np.zeros(pr.n))
            info = g.gmres_solve(h, dev(b), x, 30, 1e-8, 5000, prm)
            assert info.status == 0
            res[(mode, k)] = (info.iters, host(x))
    for k in (0, 1):
        assert res[(1, k)][0] == res[(2, k)][0]
        assert np.array_equal(res[(1, k)][1], res[(2, k)][1])


@pytest.mark.parametrize("mode", [1, 2])
def test_profiled_launch_counts_in_graph_and_eager_cycles(g, mode):
    """Per-kernel profiling counts exactly the Arnoldi steps that ran, also
    when the steps replay as a graph whose trailing steps are no-ops."""
    pr = P.poisson2d(64)
    h = g.gs2_setup(pr.A)
    h.set_graph_mode(mode)
    h.profile(True)
    h.profile_reset()
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 5000,
                         g.params("gs2", 1, 1, direction="symmetric"))
    st = h.profile_read()
    h.profile(False)
    assert info.status == 0 and info.iters % 30 != 0  # the last cycle stops early
    assert st["spmv"]["launches"] == info.iters
    assert st["cgs2_upd_norm"]["launches"] == info.iters
    assert all(v["total_ms"] > 0 for v in st.values() if v["launches"])


def test_handles_release_all_device_memory(g):
    """Handles with every optional structure (lower-precision copies, level
    sets, colours, an AMG hierarchy, Krylov workspace, captured graphs) give
    all their device memory back when destroyed."""
    import torch
    pr = P.poisson3d(24)
    torch.cuda.synchronize()

    def cycle():
        h = g.gs2_setup(pr.A, precisions=("fp32", "fp16"))
        x = dev(np.zeros(pr.n))
        for prm in (g.params("gs2", 1, 1, direction="symmetric", precision="fp16"),
                    g.params("gs", 1, direction="symmetric"),
                    g.params("mtgs", 1, direction="symmetric"),
                    g.params("amg", 1, 1, direction="symmetric")):
            x.zero_()
            info = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 500, prm)
            assert info.status == 0
        h.close()
        torch.cuda.synchronize()

    cycle()  # first use: process-wide caches (pinned pool, kernel attributes)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        cycle()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < 4 << 20, (free0, free1)


def _long_row_stream_matrix(n=400_000, seed=29):
    """Rows of 25..32 entries, the length constant inside each 32-row chunk and
    cycling over chunks (every remainder mod 4 of the chunk length, no
    padding), CSR of ~137 MB: above the L2, so A takes the pipelined
    long-row sliced-ELL path.  Columns i + 997 k (mod n), diagonally dominant."""
    rng = np.random.default_rng(seed)
    lens = 25 + (np.arange(n) // 32) % 8
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    rows = np.repeat(np.arange(n), lens)
    k = np.arange(rp[-1]) - np.repeat(rp[:-1], lens)  # slot inside the row
    ci = np.where(k == 0, rows, (rows + 997 * k) % n).astype(np.int32)
    va = rng.uniform(-1.0, 1.0, rp[-1])
    off = np.abs(va)
    off[k == 0] = 0.0
    rowsum = np.add.reduceat(off, rp[:-1])
    va[k == 0] = rowsum + 1.0
    return rp, ci, va


def test_long_rows_streamed_from_hbm_match_oracle(g):
    A = _long_row_stream_matrix()
    n = len(A[0]) - 1
    assert 12 * len(A[1]) > 128 * (1 << 20)
    h = g.gs2_setup(A)
    assert h.stats()["sell_a"] == 1
    x0 = P.uniform_pm1(31, n)
    b = P.uniform_pm1(32, n)
    y = dev(np.zeros(n))
    g.gs2_spmv(h, dev(x0), y)
    assert rel(host(y), oracle.spmv(A, x0)) <= TOL
    for direction, dname in ((oracle.FORWARD, "forward"), (oracle.SYMMETRIC, "symmetric")):
        x = dev(x0)
        g.gs2_apply_ex(h, dev(b), x, g.params("gs2", 1, 2, omega=0.9, direction=dname))
        ref = oracle.gs2(A, b, x0, 1, 2, 0.9, 1.0, direction)
        assert rel(host(x), ref) <= TOL, dname
    h.close()

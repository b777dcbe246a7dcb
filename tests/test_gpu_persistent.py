"""GPU parity of the small-system GMRES solvers -- the one-launch solver
(the whole restarted solve in one cooperative launch, graph mode 3) and the
one-cluster solver (the whole solve inside one thread-block cluster, the
system in its CTAs' shared memory, graph mode 4): iteration counts within +-1
of the oracle and of the multi-kernel path for every preconditioner they
take, the solver statuses, run-to-run reproducibility, automatic selection,
and the bounded grid and cluster barriers giving up with GS2_ERR_TIMEOUT
instead of hanging.
"""
import numpy as np
import pytest

import oracle
from paper_2104_01196_gb300 import problems as P

pytestmark = pytest.mark.gpu


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


PROBS = {
    "poisson2d_64": P.poisson2d(64),
    "random_3000": P.random_system(3000, 61, mean_offdiag=6.0, dominance=1.1),
    "convdiff3d_12": P.convdiff3d(12),
    "elasticity3d_4": P.elasticity3d(4),
    "poisson3d_40": P.poisson3d(40),
}
PCS = {
    "none": (None, dict(pc_kind=oracle.PC_NONE)),
    "gs2_fwd_1_1": (dict(kind="gs2", outer=1, inner=1), dict(pc_kind=oracle.PC_GS2)),
    "sgs2_1_2_damped": (dict(kind="gs2", outer=1, inner=2, omega=0.9, gamma=0.8,
                             direction="symmetric"),
                        dict(pc_kind=oracle.PC_GS2, pc_inner=2, pc_omega=0.9, pc_gamma=0.8,
                             pc_direction=oracle.SYMMETRIC)),
    "gs2_bwd_2_0": (dict(kind="gs2", outer=2, inner=0, direction="backward"),
                    dict(pc_kind=oracle.PC_GS2, pc_outer=2, pc_inner=0,
                         pc_direction=oracle.BACKWARD)),
    "jr_3_w0.8": (dict(kind="jr", outer=3, omega=0.8),
                  dict(pc_kind=oracle.PC_JR, pc_outer=3, pc_omega=0.8)),
    # an even number of JR sweeps ends in the second buffer (a copy back)
    "jr_4": (dict(kind="jr", outer=4), dict(pc_kind=oracle.PC_JR, pc_outer=4)),
    "jr_2_w0.9": (dict(kind="jr", outer=2, omega=0.9),
                  dict(pc_kind=oracle.PC_JR, pc_outer=2, pc_omega=0.9)),
}


# Restarted GMRES with a 5-vector basis on the small Q1 elasticity problem is
# rounding-sensitive: perturbing b by one unit in the last place changes the
# oracle's own iteration count over a wide range (gs2_bwd_2_0: 301..681, jr_4:
# 287..489), because every restart keeps only a 5-dimensional Krylov space and
# the tiny differences between two runs grow by about 1e14 within 10 to 40
# steps.  There an iteration count agreeing to +-1 is not a property of the
# method but of one rounding sequence, so these cases assert instead that (1)
# the oracle itself is sensitive (a one-ulp ensemble spreads by more than 2),
# (2) the GPU tracks the oracle's true residual step by step to 1e-10 for as
# long as the oracle tracks itself to 1e-12, and (3) the GPU's count lies in
# the ensemble's range widened by 15%.  JR(2) with omega = 0.9 is sensitive in
# its outcome as well: 16 of 48 one-ulp perturbations converge (in 3,369 to
# 5,999 steps) and the others stop at the 6,000-step limit, so there the GPU
# must reach an outcome the ensemble shows.  Forward GS2(1,1) stagnates at
# restart 5 on elasticity in every run (relative residual 0.84 in all 48):
# both sides must return NOT_CONVERGED.
SENSITIVE = {("elasticity3d_4", 5, pc)
             for pc in ("none", "gs2_bwd_2_0", "jr_3_w0.8", "jr_4", "jr_2_w0.9")}
# the systems whose rows fit one cluster's shared memory (the 40^3 Laplacian,
# 64,000 rows, does not)
CLUSTER_FITS = {"poisson2d_64", "random_3000", "convdiff3d_12", "elasticity3d_4"}
STAGNATING = {("elasticity3d_4", 5, "gs2_fwd_1_1")}
ULP = 2.0 ** -52


_ENSEMBLES = {}


def oracle_ensemble(pr, restart, op, members=48, seed=7):
    """The oracle's solve of A x = b(1 + e), e_i ~ one ulp (seeded), for
    `members` perturbations: their iteration counts and statuses (computed
    once per case; every solver mode is checked against the same sample).
    The sample must be large enough to show the spread's tails: twelve
    members of backward GS2(2,0) at restart 5 spanned 334..484 iterations,
    while the spread of such perturbations reaches 301..681."""
    key = (pr.name, restart, tuple(sorted(op.items())), members, seed)
    if key not in _ENSEMBLES:
        rng = np.random.default_rng(seed)
        out = []
        for _ in range(members):
            bp = pr.b * (1.0 + ULP * rng.standard_normal(pr.n))
            _, oi = oracle.gmres(pr.A, bp, restart=restart, tol=1e-8, max_iters=6000, **op)
            out.append(oi)
        _ENSEMBLES[key] = out
    return _ENSEMBLES[key]


def tracking_horizon(pr, restart, op, kmax=40, members=4, seed=11):
    """Per step k <= kmax the oracle's true relative residual after k Arnoldi
    steps (a solve stopped by max_iters = k), and the largest k up to which
    one-ulp perturbations of b leave it within 1e-12 (the steps over which the
    oracle agrees with itself)."""
    rng = np.random.default_rng(seed)
    pert = [pr.b * (1.0 + ULP * rng.standard_normal(pr.n)) for _ in range(members)]
    base, horizon = [], 0
    for k in range(1, kmax + 1):
        _, oi = oracle.gmres(pr.A, pr.b, restart=restart, tol=1e-8, max_iters=k, **op)
        base.append(oi.true_relres)
        spread = max(abs(oracle.gmres(pr.A, bp, restart=restart, tol=1e-8, max_iters=k,
                                      **op)[1].true_relres - oi.true_relres) / oi.true_relres
                     for bp in pert)
        if spread <= 1e-12 and horizon == k - 1:
            horizon = k
    return base, horizon


def check_sensitive(g, h, pr, restart, prm, op, info):
    ens = oracle_ensemble(pr, restart, op)
    counts = [e.iters for e in ens if e.status == 0]
    stopped = [e for e in ens if e.status != 0]
    assert all(e.status in (0, 5) for e in ens)
    # the case is rounding-sensitive: both outcomes occur, or the counts spread
    if stopped:
        assert counts, "every perturbation stops: a stagnating case"
    else:
        assert max(counts) - min(counts) > 2, counts
    if info.status == 0:
        # a converged outcome, in the range of the ensemble's converged ones
        assert counts, "the GPU converged where no perturbation of the oracle does"
        lo, hi = 0.85 * min(counts), 1.15 * max(counts)
        assert lo <= info.iters <= hi, (info.iters, sorted(counts))
    else:
        assert info.status == 5 and stopped, (info, len(stopped))
    base, horizon = tracking_horizon(pr, restart, op)
    assert horizon >= 5, horizon  # at least one whole restart cycle
    for k in range(1, horizon + 1):
        x = dev(np.zeros(pr.n))
        ik = g.gmres_solve(h, dev(pr.b), x, restart, 1e-8, k, prm)
        assert abs(ik.true_relres - base[k - 1]) <= 1e-10 * base[k - 1], (k, ik, base[k - 1])


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("pc", list(PCS))
@pytest.mark.parametrize("restart", [5, 30])
def test_one_launch_matches_oracle_and_multi_kernel_path(g, name, pc, restart):
    pr = PROBS[name]
    gp, op = PCS[pc]
    case = (name, restart, pc)
    prm = g.params(**gp) if gp else None
    h = g.gs2_setup(pr.A)
    _, oinfo = oracle.gmres(pr.A, pr.b, restart=restart, tol=1e-8, max_iters=6000, **op)
    # the one-launch solver, the one-cluster solver, the multi-kernel path
    for mode in (3, 4, 1):
        if mode == 4 and name not in CLUSTER_FITS:
            h.set_graph_mode(4)
            with pytest.raises(g.GS2Error) as e:
                g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), restart, 1e-8, 10, prm)
            assert e.value.status == 1
            continue
        h.set_graph_mode(mode)
        x = dev(np.zeros(pr.n))
        info = g.gmres_solve(h, dev(pr.b), x, restart, 1e-8, 6000, prm)
        if case in STAGNATING:
            assert oinfo.status == 5 and info.status == 5, (info, oinfo)
            assert info.iters == oinfo.iters == 6000
            continue
        if case in SENSITIVE:
            check_sensitive(g, h, pr, restart, prm, op, info)
        else:
            assert info.status == 0 and oinfo.status == 0, (info, oinfo)
            assert abs(info.iters - oinfo.iters) <= 1, (mode, info.iters, oinfo.iters)
        r = np.linalg.norm(pr.b - oracle.spmv(pr.A, host(x))) / np.linalg.norm(pr.b)
        assert abs(info.true_relres - r) <= 1e-12
        assert info.status != 0 or r <= 1e-8


@pytest.mark.parametrize("mode", [3, 4])
def test_one_launch_statuses_and_reproducibility(g, mode):
    pr = P.poisson2d(40)
    h = g.gs2_setup(pr.A)
    h.set_graph_mode(mode)
    prm = g.params("gs2", 1, 1)
    x1, x2 = dev(np.zeros(pr.n)), dev(np.zeros(pr.n))
    i1 = g.gmres_solve(h, dev(pr.b), x1, 30, 1e-8, 3000, prm)
    i2 = g.gmres_solve(h, dev(pr.b), x2, 30, 1e-8, 3000, prm)
    assert i1.iters == i2.iters and i1.cycles == i2.cycles
    assert np.array_equal(host(x1), host(x2))
    # iteration limit
    info = g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 10, 1e-12, 7, prm)
    assert info.status == 5 and info.iters == 7
    # NaN in b
    b = pr.b.copy()
    b[3] = np.nan
    assert g.gmres_solve(h, dev(b), dev(np.zeros(pr.n)), 10, 1e-8, 50, prm).status == 7
    # zero right-hand side: x = 0, no step
    x = dev(np.ones(pr.n))
    info = g.gmres_solve(h, dev(np.zeros(pr.n)), x, 10, 1e-8, 50, prm)
    assert info.status == 0 and info.iters == 0 and np.all(host(x) == 0.0)
    # warm start at the solution: no step
    info = g.gmres_solve(h, dev(pr.b), dev(pr.x_true), 10, 1e-8, 50, prm)
    assert info.status == 0 and info.iters == 0
    # a diagonal matrix with JR(1): M^{-1} = D^{-1} = A^{-1}, so the first
    # step is a lucky breakdown (H(1,0) = 0) and the solve has converged
    n = 300
    d = 1.0 + P.uniform01(9, n)
    D = (np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d)
    hd = g.gs2_setup(D)
    hd.set_graph_mode(mode)
    v = P.uniform_pm1(10, n)
    x = dev(np.zeros(n))
    info = g.gmres_solve(hd, dev(v), x, 30, 1e-10, 100, g.params("jr", 1))
    assert info.status == 0 and info.iters == 1
    assert np.linalg.norm(host(x) - v / d) <= 1e-12 * np.linalg.norm(v / d)


def test_automatic_selection_uses_one_launch_for_small_systems(g):
    pr = P.poisson2d(64)
    h = g.gs2_setup(pr.A)
    b, x = dev(pr.b), dev(np.zeros(pr.n))
    g.gmres_solve(h, b, x, 30, 1e-8, 3000, g.params("gs2", 1, 1))  # warm
    c0 = g.launch_count()
    info = g.gmres_solve(h, b, dev(np.zeros(pr.n)), 30, 1e-8, 3000, g.params("gs2", 1, 1))
    assert info.status == 0 and info.iters > 100
    assert g.launch_count() - c0 <= 2, g.launch_count() - c0
    # not eligible: restart above 32, FP32 sweeps; mode 3 refuses them
    h.set_graph_mode(3)
    with pytest.raises(g.GS2Error):
        g.gmres_solve(h, b, x, 40, 1e-8, 100, g.params("gs2", 1, 1))
    with pytest.raises(g.GS2Error):
        g.gmres_solve(h, b, x, 30, 1e-8, 100, g.params("gs2", 1, 1, precision="fp32"))


@pytest.mark.parametrize("mode", [3, 4])
def test_stalled_barrier_times_out_and_the_handle_recovers(g, mode):
    """The grid and cluster barriers' waits are bounded: with an arrival
    count no block can complete (one launch) or a CTA that never arrives
    (one cluster), every block gives up (about two seconds), the solve
    reports GS2_ERR_TIMEOUT, and the next solve on the handle is normal."""
    pr = P.poisson2d(32)
    h = g.gs2_setup(pr.A)
    h.set_graph_mode(mode)
    h.test_stall_barrier()
    with pytest.raises(g.GS2Error) as e:
        g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 30, 1e-8, 500, g.params("gs2", 1, 1))
    assert e.value.status == 8
    info = g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 30, 1e-8, 500,
                         g.params("gs2", 1, 1))
    assert info.status == 0


@pytest.mark.parametrize("mode", [3, 4])
@pytest.mark.parametrize("restart", [1, 2, 8, 9, 32])
def test_one_launch_restart_edges(g, restart, mode):
    """Restart lengths at and around the register-block boundaries (the CGS2
    phases round the basis size up to a multiple of 8; m <= 32)."""
    pr = P.random_system(1500, 71, mean_offdiag=5.0, dominance=1.2)
    h = g.gs2_setup(pr.A)
    h.set_graph_mode(mode)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, restart, 1e-9, 4000, g.params("gs2", 1, 1))
    _, oinfo = oracle.gmres(pr.A, pr.b, restart=restart, tol=1e-9, max_iters=4000,
                            pc_kind=oracle.PC_GS2)
    assert info.status == 0 and oinfo.status == 0
    assert abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)


@pytest.mark.parametrize("mode", [3, 4])
def test_one_launch_tiny_systems(g, mode):
    """One row, two rows, and a system smaller than one block."""
    one = (np.array([0, 1]), np.array([0], np.int32), np.array([4.0]))
    h = g.gs2_setup(one)
    h.set_graph_mode(mode)
    x = dev(np.zeros(1))
    info = g.gmres_solve(h, dev(np.array([2.0])), x, 30, 1e-12, 10, g.params("gs2", 1, 1))
    assert info.status == 0 and host(x)[0] == pytest.approx(0.5, rel=1e-15)
    two = P.dense_to_csr(np.array([[3.0, 1.0], [-1.0, 2.0]]))
    h = g.gs2_setup(two)
    h.set_graph_mode(mode)
    x = dev(np.zeros(2))
    info = g.gmres_solve(h, dev(np.array([1.0, 1.0])), x, 30, 1e-12, 10, None)
    assert info.status == 0 and info.iters <= 2
    assert np.allclose(host(x), np.linalg.solve([[3.0, 1.0], [-1.0, 2.0]], [1.0, 1.0]),
                       rtol=1e-12)
    pr = P.poisson2d(9)  # 81 rows
    h = g.gs2_setup(pr.A)
    h.set_graph_mode(mode)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, 30, 1e-10, 500, g.params("gs2", 1, 2,
                                                                     direction="symmetric"))
    _, oinfo = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-10, max_iters=500,
                            pc_kind=oracle.PC_GS2, pc_inner=2, pc_direction=oracle.SYMMETRIC)
    assert info.status == 0 and abs(info.iters - oinfo.iters) <= 1


SPD = {
    "poisson2d_64": P.poisson2d(64),
    "poisson3d_24": P.poisson3d(24),
    "elasticity3d_4": P.elasticity3d(4),
}
CG_PCS = {
    "none": (None, dict(pc_kind=oracle.PC_NONE)),
    "sgs2_1_1": (dict(kind="gs2", outer=1, inner=1, direction="symmetric"),
                 dict(pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC)),
    "sgs2_1_2_w0.9": (dict(kind="gs2", outer=1, inner=2, omega=0.9, direction="symmetric"),
                      dict(pc_kind=oracle.PC_GS2, pc_inner=2, pc_omega=0.9,
                           pc_direction=oracle.SYMMETRIC)),
    "jr_2_w0.7": (dict(kind="jr", outer=2, omega=0.7),
                  dict(pc_kind=oracle.PC_JR, pc_outer=2, pc_omega=0.7)),
}


@pytest.mark.parametrize("mode", [3, 4])
@pytest.mark.parametrize("name", list(SPD))
@pytest.mark.parametrize("pc", list(CG_PCS))
def test_one_launch_cg_matches_oracle(g, name, pc, mode):
    pr = SPD[name]
    gp, op = CG_PCS[pc]
    prm = g.params(**gp) if gp else None
    h = g.gs2_setup(pr.A)
    h.set_graph_mode(mode)
    x = dev(np.zeros(pr.n))
    info = g.cg_solve(h, dev(pr.b), x, 1e-8, 5000, prm)
    _, oinfo = oracle.cg(pr.A, pr.b, tol=1e-8, max_iters=5000, **op)
    assert info.status == 0 and oinfo.status == 0, (info, oinfo)
    assert abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)
    r = np.linalg.norm(pr.b - oracle.spmv(pr.A, host(x))) / np.linalg.norm(pr.b)
    assert r <= 1e-8 and abs(info.true_relres - r) <= 1e-12
    h.set_graph_mode(1)
    ig = g.cg_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 1e-8, 5000, prm)
    assert abs(ig.iters - info.iters) <= 1


@pytest.mark.parametrize("mode", [3, 4])
def test_one_launch_cg_statuses_and_selection(g, mode):
    pr = P.poisson2d(40)
    h = g.gs2_setup(pr.A)
    prm = g.params("gs2", 1, 1, direction="symmetric")
    b = dev(pr.b)
    g.cg_solve(h, b, dev(np.zeros(pr.n)), 1e-8, 500, prm)  # warm
    c0 = g.launch_count()
    info = g.cg_solve(h, b, dev(np.zeros(pr.n)), 1e-8, 500, prm)
    assert info.status == 0 and g.launch_count() - c0 <= 2
    h.set_graph_mode(mode)
    info = g.cg_solve(h, b, dev(np.zeros(pr.n)), 1e-14, 9, prm)
    assert info.status == 5 and info.iters == 9
    x = dev(np.ones(pr.n))
    info = g.cg_solve(h, dev(np.zeros(pr.n)), x, 1e-8, 50, prm)
    assert info.status == 0 and info.iters == 0 and np.all(host(x) == 0.0)
    bn = pr.b.copy()
    bn[7] = np.nan
    assert g.cg_solve(h, dev(bn), dev(np.zeros(pr.n)), 1e-8, 50, prm).status == 7
    with pytest.raises(g.GS2Error):
        g.cg_solve(h, b, dev(np.zeros(pr.n)), 1e-8, 50,
                   g.params("gs2", 1, 1, direction="symmetric", precision="fp32"))


def test_autotune_gmres_picks_a_structure_and_keeps_the_results(g):
    """gs2_autotune_gmres times one restart cycle per solve structure
    (separate launches, cycle graphs, one launch or one cluster where
    eligible), makes the fastest the automatic choice for that restart and
    preconditioner, reports
    it in the handle's stats, and the tuned automatic solve keeps the
    oracle's count; a different preconditioner falls back to the size rule."""
    prm = g.params("gs2", 1, 1, direction="symmetric")
    # the 64^2 system also fits one cluster; the 40^3 one does not
    for pr, candidates in ((P.poisson2d(64), 4), (P.poisson3d(40), 3)):
        h = g.gs2_setup(pr.A)
        mode = h.autotune_gmres(30, prm)
        st = h.stats()
        assert mode in (1, 2, 3, 4) and st["solve_mode"] == mode
        assert st["solve_modes_timed"] == candidates
        x = dev(np.zeros(pr.n))
        info = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 3000, prm)
        _, oinfo = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=3000,
                                pc_kind=oracle.PC_GS2, pc_direction=oracle.SYMMETRIC)
        assert info.status == 0 and abs(info.iters - oinfo.iters) <= 1
        r = np.linalg.norm(pr.b - oracle.spmv(pr.A, host(x))) / np.linalg.norm(pr.b)
        assert r <= 1e-8
        # another preconditioner: untuned, the size rule applies
        info2 = g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 30, 1e-8, 3000,
                              g.params("jr", 3, omega=0.8))
        assert info2.status == 0
    # lower-precision sweeps: the one-launch solver does not take them
    pr = P.poisson2d(40)
    h = g.gs2_setup(pr.A, precisions=("fp32",))
    mode = h.autotune_gmres(30, g.params("gs2", 1, 1, precision="fp32"))
    assert mode in (1, 2) and h.stats()["solve_modes_timed"] == 2

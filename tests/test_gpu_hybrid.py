"""GPU parity of the hybrid (block-Jacobi) form of GS2 and JR (Sec. 3, with
the n_k local sweeps of the two-stage listing): the rows in P contiguous
blocks, the other blocks' values frozen at each exchange.  Every sweep must
match the oracle to 1e-12 per vector; GMRES and CG with the hybrid
preconditioners must take the oracle's iteration counts within +-1; and the
local-versus-global JR trend of the paper's strong-scaling runs must hold.
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


PROBS = {
    "poisson2d_37": P.poisson2d(37),
    "random_3000": P.random_system(3000, 71, mean_offdiag=6.0, dominance=1.1),
    "convdiff3d_12": P.convdiff3d(12),
    "elasticity3d_5": P.elasticity3d(5),
}
DIRS = {"forward": oracle.FORWARD, "backward": oracle.BACKWARD, "symmetric": oracle.SYMMETRIC}


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("parts", [2, 7, 64])
@pytest.mark.parametrize("direction", list(DIRS))
def test_hybrid_gs2_sweeps_match_oracle(g, name, parts, direction):
    pr = PROBS[name]
    b = P.uniform_pm1(81, pr.n)
    x0 = P.uniform_pm1(82, pr.n)
    for outer, local, inner, om, ga in ((1, 1, 1, 1.0, 1.0), (2, 3, 2, 0.9, 0.8)):
        h = g.gs2_setup(pr.A)
        x = dev(x0)
        g.gs2_apply_ex(h, dev(b), x, g.params("gs2", outer, inner, omega=om, gamma=ga,
                                            direction=direction, parts=parts, local=local))
        want = oracle.hybrid(pr.A, b, x0, oracle.PC_GS2, parts=parts, outer=outer, local=local,
                             inner=inner, omega=om, gamma=ga, direction=DIRS[direction])
        assert rel(host(x), want) <= TOL, (outer, local)


@pytest.mark.parametrize("name", list(PROBS))
def test_hybrid_jr_and_special_cases(g, name):
    pr = PROBS[name]
    b = P.uniform_pm1(83, pr.n)
    x0 = P.uniform_pm1(84, pr.n)
    h = g.gs2_setup(pr.A)
    # a local GS2 half sweep without inner sweeps is a local JR sweep
    for parts, outer, local in ((3, 2, 2), (16, 1, 4), (16, 4, 1)):
        x = dev(x0)
        g.gs2_apply_ex(h, dev(b), x, g.params("gs2", outer, 0, omega=0.7, parts=parts,
                                            local=local))
        want = oracle.hybrid(pr.A, b, x0, oracle.PC_JR, parts=parts, outer=outer, local=local,
                             omega=0.7)
        assert rel(host(x), want) <= TOL, (parts, outer, local)
    # one block with n_k local sweeps = n_t n_k global sweeps
    x = dev(x0)
    g.gs2_apply_ex(h, dev(b), x, g.params("gs2", 2, 2, direction="symmetric", parts=1, local=3))
    want = oracle.gs2(pr.A, b, x0, outer=6, inner=2, direction=oracle.SYMMETRIC)
    assert rel(host(x), want) <= TOL
    # more blocks than rows count as one block per row: GS2 becomes JR
    x = dev(x0)
    g.gs2_apply_ex(h, dev(b), x, g.params("gs2", 3, 2, parts=10 * pr.n))
    want = oracle.jr(pr.A, b, x0, sweeps=3, omega=1.0)
    assert rel(host(x), want) <= TOL


PCS = {
    "sgs2_1_1_p8": (dict(kind="gs2", outer=1, inner=1, direction="symmetric", parts=8),
                    dict(pc_kind=oracle.PC_HYBRID_GS2, pc_direction=oracle.SYMMETRIC,
                         pc_parts=8)),
    "gs2_2_2_p5_local2": (dict(kind="gs2", outer=2, inner=2, omega=0.9, parts=5, local=2),
                          dict(pc_kind=oracle.PC_HYBRID_GS2, pc_outer=2, pc_inner=2,
                               pc_omega=0.9, pc_parts=5, pc_local=2)),
    "jr_1_4_p16": (dict(kind="jr", outer=1, parts=16, local=4),
                   dict(pc_kind=oracle.PC_HYBRID_JR, pc_outer=1, pc_parts=16, pc_local=4)),
    "jr_4_1_p16": (dict(kind="jr", outer=4, parts=16, local=1),
                   dict(pc_kind=oracle.PC_HYBRID_JR, pc_outer=4, pc_parts=16, pc_local=1)),
}


@pytest.mark.parametrize("name", ["poisson2d_37", "random_3000", "convdiff3d_12"])
@pytest.mark.parametrize("pc", list(PCS))
def test_gmres_with_hybrid_preconditioners_matches_oracle(g, name, pc):
    pr = PROBS[name]
    gp, op = PCS[pc]
    h = g.gs2_setup(pr.A)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 4000, g.params(**gp))
    _, oinfo = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=4000, **op)
    assert info.status == 0 and oinfo.status == 0
    assert abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)
    r = np.linalg.norm(pr.b - oracle.spmv(pr.A, host(x))) / np.linalg.norm(pr.b)
    assert r <= 1e-8


def test_cg_with_hybrid_sgs2_matches_oracle(g):
    pr = P.poisson3d(14)
    h = g.gs2_setup(pr.A)
    x = dev(np.zeros(pr.n))
    info = g.cg_solve(h, dev(pr.b), x, 1e-8, 2000,
                      g.params("gs2", 1, 1, direction="symmetric", parts=6))
    _, oinfo = oracle.cg(pr.A, pr.b, tol=1e-8, max_iters=2000, pc_kind=oracle.PC_HYBRID_GS2,
                         pc_direction=oracle.SYMMETRIC, pc_parts=6)
    assert info.status == 0 and oinfo.status == 0
    assert abs(info.iters - oinfo.iters) <= 1


def test_local_jr_grows_with_the_blocks_global_jr_does_not(g):
    """Sec. 8 strong scaling: with the global JR(4,1) the GMRES count does
    not depend on the number of blocks (processes); with the local JR(1,4)
    it grows with them."""
    pr = P.poisson3d(24)
    h = g.gs2_setup(pr.A)
    glob, loc = [], []
    for parts in (1, 8, 64):
        for out, outer, local in ((glob, 4, 1), (loc, 1, 4)):
            info = g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 30, 1e-8, 4000,
                                 g.params("jr", outer, parts=parts, local=local))
            assert info.status == 0
            out.append(info.iters)
    assert max(glob) - min(glob) <= 1
    assert abs(loc[0] - glob[0]) <= 1 and loc[0] < loc[1] < loc[2]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_hybrid_lower_precision_inner_sweeps(g, prec):
    pr = PROBS["convdiff3d_12"]
    h = g.gs2_setup(pr.A)
    p64 = g.params("gs2", 1, 1, direction="symmetric", parts=8)
    plo = g.params("gs2", 1, 1, direction="symmetric", parts=8, precision=prec)
    i64 = g.gmres_solve(h, dev(pr.b), dev(np.zeros(pr.n)), 30, 1e-8, 4000, p64)
    x = dev(np.zeros(pr.n))
    ilo = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 4000, plo)
    assert ilo.status == 0 and abs(ilo.iters - i64.iters) <= 2
    r = np.linalg.norm(pr.b - oracle.spmv(pr.A, host(x))) / np.linalg.norm(pr.b)
    assert r <= 1e-8


def test_hybrid_refusals(g):
    pr = PROBS["poisson2d_37"]
    h = g.gs2_setup(pr.A)
    b, x = dev(pr.b), dev(np.zeros(pr.n))
    for bad in (g.params("gs2", 1, 1, form="compact", parts=4),
                g.params("mtgs", 1, parts=4), g.params("amg", 1, 1, parts=4),
                g.params("mtgs", 1, local=2), g.params("gs2", 1, 1, parts=-1)):
        with pytest.raises(g.GS2Error):
            g.gmres_solve(h, b, x, 30, 1e-8, 10, bad)
    pk = g.pack_setup([pr.A, pr.A])
    with pytest.raises(g.GS2Error):
        g.pack_gmres(pk, dev(np.concatenate([pr.b, pr.b])), dev(np.zeros(2 * pr.n)), 30, 1e-8,
                     10, g.params("gs2", 1, 1, parts=4))


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("parts", [1, 5, 40])
def test_relax_apply_every_kind_global_and_hybrid(g, name, parts):
    """relax_apply: JR, exact GS (the local triangles solved by their own
    level sets in the hybrid form) and GS2 against the oracle; multicolour
    GS (global only) against its oracle."""
    pr = PROBS[name]
    b = P.uniform_pm1(91, pr.n)
    x0 = P.uniform_pm1(92, pr.n)
    h = g.gs2_setup(pr.A)
    cases = [("jr", oracle.PC_JR, dict(outer=2, omega=0.8, local=2)),
             ("gs", oracle.PC_GS, dict(outer=2, omega=0.9, direction="symmetric", local=2)),
             ("gs", oracle.PC_GS, dict(outer=1, direction="backward")),
             ("gs2", oracle.PC_GS2, dict(outer=1, inner=3, direction="symmetric", local=2))]
    for kind, okind, kw in cases:
        x = dev(x0)
        g.relax_apply(h, dev(b), x, g.params(kind, parts=parts, **kw))
        want = oracle.hybrid(pr.A, b, x0, okind, parts=parts, outer=kw["outer"],
                             local=kw.get("local", 1), inner=kw.get("inner", 1),
                             omega=kw.get("omega", 1.0),
                             direction=DIRS[kw.get("direction", "forward")])
        assert rel(host(x), want) <= TOL, (kind, kw)
    if parts == 1:
        x = dev(x0)
        g.relax_apply(h, dev(b), x, g.params("mtgs", 2, omega=0.9, direction="symmetric"))
        want = oracle.mtgs(pr.A, b, x0, sweeps=2, omega=0.9, direction=oracle.SYMMETRIC)
        assert rel(host(x), want) <= TOL


@pytest.mark.parametrize("name", ["poisson2d_37", "convdiff3d_12"])
def test_gmres_with_hybrid_exact_sgs_matches_oracle(g, name):
    pr = PROBS[name]
    h = g.gs2_setup(pr.A)
    x = dev(np.zeros(pr.n))
    info = g.gmres_solve(h, dev(pr.b), x, 30, 1e-8, 4000,
                         g.params("gs", 1, direction="symmetric", parts=12))
    _, oinfo = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=4000,
                            pc_kind=oracle.PC_HYBRID_GS, pc_direction=oracle.SYMMETRIC,
                            pc_parts=12)
    assert info.status == 0 and oinfo.status == 0
    assert abs(info.iters - oinfo.iters) <= 1, (info.iters, oinfo.iters)

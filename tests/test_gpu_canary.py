"""Canary padding around the caller's vectors: every entry point that
writes a vector (relaxations of every kind, SpMV, GMRES and CG on the
multi-kernel and one-launch paths, packs, the AMG cycle, the server) must
leave the guard regions before and after it bit for bit untouched, and read
nothing beyond its n entries (a NaN planted in the guards would spread into
the result)."""
import numpy as np
import pytest

from paper_2104_01196_gb300 import problems as P

pytestmark = pytest.mark.gpu
G = 4099  # guard entries on each side (odd, so vectors start unaligned too)


@pytest.fixture(scope="module")
def g():
    import torch  # noqa: F401

    from paper_2104_01196_gb300 import build as B
    B.build()
    import paper_2104_01196_gb300 as gs2
    gs2.load()
    return gs2


def guarded(v, fill=np.nan):
    """A device buffer [guard | v | guard]; returns (buffer, view of v)."""
    import torch
    n = len(v)
    buf = torch.full((n + 2 * G,), fill, dtype=torch.float64, device="cuda")
    buf[G:G + n] = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()
    return buf, buf[G:G + n]


def guards_intact(buf, n, fill=np.nan):
    import torch
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    lo, hi = h[:G], h[G + n:]
    if np.isnan(fill):
        return bool(np.all(np.isnan(lo)) and np.all(np.isnan(hi)))
    return bool(np.all(lo == fill) and np.all(hi == fill))


PROBS = {"poisson3d_20": P.poisson3d(20),
         "random_5000": P.random_system(5000, 81, mean_offdiag=7.0, dominance=1.1,
                                        long_rows=((17, 40), (2500, 900)))}


@pytest.mark.parametrize("name", list(PROBS))
def test_relaxations_and_spmv_keep_guards(g, name):
    pr = PROBS[name]
    h = g.gs2_setup(pr.A, precisions=("fp32", "fp16"))
    for params in (g.params("gs2", 2, 2, omega=0.9, gamma=0.8, direction="symmetric"),
                   g.params("gs2", 1, 1, direction="symmetric", precision="fp16"),
                   g.params("gs2", 1, 2, direction="backward", form="compact"),
                   g.params("jr", 3, omega=0.7), g.params("gs", 1, direction="symmetric"),
                   g.params("mtgs", 1, direction="symmetric"),
                   g.params("gs2", 1, 1, direction="symmetric", parts=5, local=2)):
        bb, b = guarded(pr.b)
        xb, x = guarded(np.zeros(pr.n))
        g.relax_apply(h, b, x, params)
        out = x.cpu().numpy()
        assert np.all(np.isfinite(out)), params.kind
        assert guards_intact(bb, pr.n) and guards_intact(xb, pr.n), params.kind
    xb, x = guarded(P.uniform_pm1(3, pr.n))
    yb, y = guarded(np.zeros(pr.n))
    g.gs2_spmv(h, x, y)
    assert np.all(np.isfinite(y.cpu().numpy()))
    assert guards_intact(xb, pr.n) and guards_intact(yb, pr.n)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_solvers_keep_guards(g, mode):
    """mode 0 takes the one-launch solver for the small system."""
    for pr in (P.poisson2d(60), P.poisson3d(20)):
        h = g.gs2_setup(pr.A)
        h.set_graph_mode(mode)
        for solve in ("gmres", "cg"):
            bb, b = guarded(pr.b)
            xb, x = guarded(np.zeros(pr.n))
            prm = g.params("gs2", 1, 1, direction="symmetric")
            info = (g.gmres_solve(h, b, x, 30, 1e-8, 3000, prm) if solve == "gmres"
                    else g.cg_solve(h, b, x, 1e-8, 3000, prm))
            assert info.status == 0 and info.true_relres <= 1e-8, (solve, info)
            assert guards_intact(bb, pr.n) and guards_intact(xb, pr.n), solve


def test_pack_amg_and_server_keep_guards(g):
    probs = [P.poisson2d(30), P.convdiff3d(9), P.random_system(700, 41, dominance=1.1)]
    pk = g.pack_setup([p.A for p in probs])
    rhs = np.concatenate([p.b for p in probs])
    bb, b = guarded(rhs)
    xb, x = guarded(np.zeros(pk.n))
    infos = g.pack_gmres(pk, b, x, 30, 1e-8, 3000, g.params("gs2", 1, 1))
    assert all(i.status == 0 for i in infos)
    assert guards_intact(bb, pk.n) and guards_intact(xb, pk.n)
    pr = P.poisson3d(24)
    h = g.gs2_setup(pr.A)
    bb, b = guarded(pr.b)
    xb, x = guarded(np.zeros(pr.n))
    g.amg_vcycle(h, b, x, g.params("amg", 1, 1, direction="symmetric"))
    assert np.all(np.isfinite(x.cpu().numpy()))
    assert guards_intact(bb, pr.n) and guards_intact(xb, pr.n)

"""The solve server: continuous batching of independent systems.

GPU tests check that every result is the same, bit for bit, alone and in the
mix (small requests are solved in one cluster, the others with per-cycle
graphs, as gmres_solve does in those graph modes); that admission follows
the memory budget; and that a failure injected
on the host (a request whose allocation "fails") is reported for that
request while the others complete.  The CPU test checks the admission
estimate, which needs no GPU.
"""
import numpy as np
import pytest

import paper_2104_01196_gb300 as gs2
from paper_2104_01196_gb300 import build as B
from paper_2104_01196_gb300 import problems as P


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gs2.load()


def test_footprint_covers_matrix_triangles_and_basis(lib):
    n, nnz = 100_000, 700_000
    fp = gs2.server_footprint(n, nnz, restart=30)
    # A (12 B/entry), the two prescaled triangles, the 31-vector basis
    assert fp >= 12 * nnz + 12 * (nnz - n) + 8 * n * 31
    assert fp < 2 * (24 * nnz + 8 * n * 60)
    assert gs2.server_footprint(2 * n, 2 * nnz) > fp
    assert gs2.server_footprint(n, nnz, restart=60) > fp
    lowp = gs2.server_footprint(n, nnz, precond=gs2.params("gs2", precision="fp32"))
    assert lowp > gs2.server_footprint(n, nnz, precond=gs2.params("gs2"))
    # multicolour GS keeps a colour-ordered copy of the off-diagonal entries
    mc = gs2.server_footprint(n, nnz, precond=gs2.params("mtgs"))
    assert mc >= gs2.server_footprint(n, nnz, precond=gs2.params("gs2")) + 12 * (nnz - n)


def _mix():
    reqs = [P.variable_coefficient_problem("poisson2d", 30, 11),
            P.variable_coefficient_problem("poisson3d", 14, 12),
            P.variable_coefficient_problem("convdiff3d", 12, 13),
            P.poisson2d(50),
            P.variable_coefficient_problem("poisson3d", 22, 14),
            P.random_system(3000, 15, dominance=1.1),
            P.variable_coefficient_problem("convdiff3d", 18, 16),
            P.poisson3d(16)]
    return reqs


def _alone(pr, pc, max_iters=4000):
    """gmres_solve alone, on the path the server takes: one cluster where the
    system fits (graph mode 4), else the per-cycle graphs (mode 1)."""
    import torch
    h = gs2.gs2_setup(pr.A)
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    b = torch.from_numpy(pr.b).cuda()
    h.set_graph_mode(4)
    try:
        info = gs2.gmres_solve(h, b, x, 30, 1e-8, max_iters, pc)
    except gs2.GS2Error as e:
        assert e.status == 1  # does not fit one cluster: refused before any work
        h.set_graph_mode(1)
        info = gs2.gmres_solve(h, b, x, 30, 1e-8, max_iters, pc)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    h.close()
    return info, out


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_sweep", "mtsgs", "amg", "hybrid"])
def test_results_equal_alone_and_in_the_mix(lib, prec):
    if prec == "mtsgs":
        pc = gs2.params("mtgs", 1, direction="symmetric")
    elif prec == "amg":
        pc = gs2.params("amg", 1, 1, direction="symmetric")
    elif prec == "hybrid":
        pc = gs2.params("gs2", 1, 1, direction="symmetric", parts=6, local=2)
    else:
        pc = gs2.params("gs2", 1, 1, direction="symmetric", precision=prec)
    probs = _mix()
    srv = gs2.Server(restart=30, tol=1e-8, max_iters=4000, precond=pc, max_slots=3,
                     prep_threads=2)
    tickets = [srv.submit(p.A, p.b) for p in probs]
    got = [srv.wait(t, p.n) for t, p in zip(tickets, probs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(probs) and st["failed"] == 0
    assert 1 < st["max_active"] <= 3
    for p, (info, x, lat) in zip(probs, got):
        ainfo, ax = _alone(p, pc)
        assert info.status == 0 and info.true_relres <= 1e-8
        assert info.iters == ainfo.iters
        assert np.array_equal(x, ax), p.name
        assert lat > 0.0


@pytest.mark.gpu
def test_admission_follows_the_memory_budget(lib):
    probs = [P.poisson3d(20) for _ in range(6)]
    pc = gs2.params("gs2", 1, 1, direction="symmetric")
    probe = gs2.Server(precond=pc, max_slots=8)
    fp = probe.footprint(probs[0].n, probs[0].nnz)
    probe.close()
    # room for two requests at a time, although eight slots are free
    srv = gs2.Server(precond=pc, max_slots=8, hbm_budget_bytes=int(2.5 * fp))
    tickets = [srv.submit(p.A, p.b) for p in probs]
    for t, p in zip(tickets, probs):
        info, x, _ = srv.wait(t, p.n)
        assert info.status == 0
    st = srv.stats()
    srv.close()
    assert st["completed"] == 6 and st["max_active"] <= 2
    assert st["reserved_bytes"] == 0
    # a request that can never fit is refused at submission
    small = gs2.Server(precond=pc, hbm_budget_bytes=fp // 2)
    with pytest.raises(gs2.GS2Error) as e:
        small.submit(probs[0].A, probs[0].b)
    assert e.value.status == 3
    small.close()


@pytest.mark.gpu
def test_injected_allocation_failure_is_reported_and_others_complete(lib):
    probs = [P.poisson2d(40), P.poisson2d(41), P.poisson2d(42)]
    srv = gs2.Server(precond=gs2.params("gs2", 1, 1), max_slots=2, fail_ticket=2)
    tickets = [srv.submit(p.A, p.b) for p in probs]
    assert tickets == [1, 2, 3]
    out = [srv.wait(t, p.n) for t, p in zip(tickets, probs)]
    st = srv.stats()
    srv.close()
    assert out[1][0].status == 3
    assert out[0][0].status == 0 and out[2][0].status == 0
    assert st["failed"] == 1 and st["completed"] == 2


@pytest.mark.gpu
def test_poll_busy_unknown_and_invalid_requests(lib):
    pr = P.poisson3d(24)
    srv = gs2.Server(precond=gs2.params("gs2", 1, 1, direction="symmetric"))
    t = srv.submit(pr.A, pr.b)
    r = srv.poll(t, pr.n)
    while r is None:
        r = srv.poll(t, pr.n)
    assert r[0].status == 0
    with pytest.raises(gs2.GS2Error):
        srv.poll(t, pr.n)  # already collected
    # a zero diagonal fails in preparation and is reported for the request
    bad = P.dense_to_csr(np.array([[1.0, 2.0], [3.0, 0.0]]))
    tb = srv.submit(bad, np.ones(2))
    info, _, _ = srv.wait(tb, 2)
    assert info.status == 2
    srv.close()


def _pack_of_one(pr, pc):
    import torch
    pk = gs2.pack_setup([pr.A])
    pk.set_graph_mode(1)  # the cycle-graph path the server runs packs on
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    info = gs2.pack_gmres(pk, torch.from_numpy(pr.b).cuda(), x, 30, 1e-8, 4000, pc)[0]
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    pk.close()
    return info, out


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_sweep"])
def test_packed_requests_are_independent_of_their_pack_mates(lib, prec):
    """Requests up to pack_rows rows are admitted together and solved as one
    pack; each result is bitwise that of the request solved as a pack of
    one, agrees with gmres_solve alone (iterations +-1, x to 1e-6), and the
    larger requests still run alone, bitwise as gmres_solve."""
    pc = gs2.params("gs2", 1, 1, direction="symmetric", precision=prec)
    probs = _mix()
    limit = 5000
    srv = gs2.Server(restart=30, tol=1e-8, max_iters=4000, precond=pc, max_slots=2,
                     prep_threads=2, pack_rows=limit, pack_max=4)
    tickets = [srv.submit(p.A, p.b) for p in probs]
    got = [srv.wait(t, p.n) for t, p in zip(tickets, probs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(probs) and st["failed"] == 0 and st["max_active"] <= 2
    assert st["reserved_bytes"] == 0
    packed = [p.n <= limit for p in probs]
    assert 2 <= sum(packed) < len(probs)
    for p, small, (info, x, lat) in zip(probs, packed, got):
        assert info.status == 0 and info.true_relres <= 1e-8 and lat > 0.0
        ainfo, ax = _alone(p, pc)
        if small:
            oinfo, ox = _pack_of_one(p, pc)
            assert info.iters == oinfo.iters and np.array_equal(x, ox), p.name
            assert abs(info.iters - ainfo.iters) <= 1
            assert np.linalg.norm(x - ax) <= 1e-6 * np.linalg.norm(ax)
        else:
            assert info.iters == ainfo.iters and np.array_equal(x, ax), p.name


@pytest.mark.gpu
def test_a_bad_request_in_a_pack_fails_alone(lib):
    """Inside one pack: an injected allocation failure and a zero diagonal
    are reported for their own requests; the others converge."""
    good = [P.poisson2d(20), P.poisson2d(21), P.poisson2d(22)]
    bad = P.dense_to_csr(np.array([[1.0, 2.0], [3.0, 0.0]]))
    srv = gs2.Server(precond=gs2.params("gs2", 1, 1), max_slots=1, pack_rows=10_000,
                     fail_ticket=1)
    mats = [(good[0].A, good[0].b), (bad, np.ones(2)), (good[1].A, good[1].b),
            (good[2].A, good[2].b)]
    tickets = [srv.submit(A, b) for A, b in mats]
    out = [srv.wait(t, len(b)) for t, (A, b) in zip(tickets, mats)]
    st = srv.stats()
    srv.close()
    assert [o[0].status for o in out] == [3, 2, 0, 0]
    assert st["failed"] == 2 and st["completed"] == 2 and st["reserved_bytes"] == 0
    for (info, x, _), p in zip(out[2:], good[1:]):
        r = np.linalg.norm(p.b - P.csr_matvec(p.A, x)) / np.linalg.norm(p.b)
        assert r <= 1e-8


@pytest.mark.gpu
@pytest.mark.parametrize("pc_name", ["sgs2", "sgs2_fp32", "sgs2_fp16", "mtgs", "gs", "jr",
                                     "hybrid4", "amg"])
def test_footprint_bounds_what_a_handle_allocates(lib, pc_name):
    """The admission estimate is an upper bound of the device bytes a handle
    holds after solving with that preconditioner (matrix, triangles, their
    sliced-ELL and lower-precision copies, level sets or colours, the
    hierarchy, the Krylov workspace), on short- and long-row matrices."""
    import torch
    pcs = {
        "sgs2": gs2.params("gs2", 1, 1, direction="symmetric"),
        "sgs2_fp32": gs2.params("gs2", 1, 1, direction="symmetric", precision="fp32"),
        "sgs2_fp16": gs2.params("gs2", 1, 1, direction="symmetric", precision="fp16"),
        "mtgs": gs2.params("mtgs", 1, direction="symmetric"),
        "gs": gs2.params("gs", 1, direction="symmetric"),
        "jr": gs2.params("jr", 2, omega=0.7),
        "hybrid4": gs2.params("gs2", 1, 1, direction="symmetric", parts=4),
        "amg": gs2.params("amg", 1, 1, direction="symmetric"),
    }
    pc = pcs[pc_name]
    for pr in (P.poisson2d(40), P.poisson3d(16), P.convdiff3d(12), P.elasticity3d(6)):
        prec = {"sgs2_fp32": ("fp32",), "sgs2_fp16": ("fp16",)}.get(pc_name, ())
        h = gs2.gs2_setup(pr.A, precisions=prec)
        if pc_name == "amg":
            h.amg_setup()
        b = torch.from_numpy(pr.b).cuda()
        x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
        gs2.gmres_solve(h, b, x, 30, 1e-8, 60, pc)
        used = h.stats()["device_bytes"]
        h.close()
        fp = gs2.server_footprint(pr.n, pr.nnz, restart=30, precond=pc)
        assert used <= fp, (pr.name, pc_name, used, fp)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp16"])
def test_staggered_arrivals_equal_alone(lib, prec):
    """Requests submitted while earlier ones are on the GPU (each submitted
    after the previous one was admitted and has run for a while, and one
    large request keeps a slot busy throughout) are admitted into free slots
    as they arrive; every result is still bitwise the one it gets alone."""
    import time
    pc = gs2.params("gs2", 1, 1, direction="symmetric", precision=prec)
    big = P.variable_coefficient_problem("poisson2d", 1200, 21)  # a long solve
    probs = [big] + _mix()
    srv = gs2.Server(restart=30, tol=1e-8, max_iters=8000, precond=pc, max_slots=3,
                     prep_threads=2)
    t_sub = [time.perf_counter()]
    tickets = [srv.submit(big.A, big.b)]
    running_seen = 0
    for p in probs[1:]:
        time.sleep(0.01)
        running_seen = max(running_seen, srv.stats()["active"])
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(p.A, p.b))
    got = [srv.wait(t, p.n) for t, p in zip(tickets, probs)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(probs) and st["failed"] == 0
    assert running_seen >= 1 and st["max_active"] > 1
    # the large request was still running when the last one arrived
    assert t_sub[0] + got[0][2] / 1000.0 > t_sub[-1]
    for p, (info, x, lat) in zip(probs, got):
        ainfo, ax = _alone(p, pc, 8000)
        assert info.status == 0 and info.iters == ainfo.iters, p.name
        assert np.array_equal(x, ax), p.name


@pytest.mark.gpu
@pytest.mark.parametrize("pack_rows", [0, 5000])
def test_small_requests_pass_large_ones_waiting_for_a_slot(lib, pack_rows):
    """With one of two slots kept for requests of at most 5,000 rows, large
    requests run one at a time and the small requests submitted behind two
    large ones are admitted before the second: each finishes before the
    first large one does, the second large one only starts after the first
    ends, and every result is still bitwise the one it gets alone (or as a
    pack of one, when packed)."""
    import time
    pc = gs2.params("gs2", 1, 1, direction="symmetric")
    bigs = [P.variable_coefficient_problem("poisson2d", 1000, 31),
            P.variable_coefficient_problem("poisson2d", 1000, 32)]
    smalls = [p for p in _mix() if p.n <= 5000]
    assert len(smalls) >= 3
    srv = gs2.Server(restart=30, tol=1e-8, max_iters=8000, precond=pc, max_slots=2,
                     prep_threads=2, pack_rows=pack_rows, pack_max=4, small_rows=5000,
                     small_slots=1)
    t0 = time.perf_counter()
    subs, tickets = [], []
    for p in bigs + smalls:
        subs.append(time.perf_counter() - t0)
        tickets.append(srv.submit(p.A, p.b))
    got = [srv.wait(t, p.n) for t, p in zip(tickets, bigs + smalls)]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(tickets) and st["failed"] == 0 and st["reserved_bytes"] == 0
    done = [s + lat / 1000.0 for s, (_, _, lat) in zip(subs, got)]
    # the two large requests are alike: run one after the other, the second
    # ends about one solve after the first (side by side, both would end
    # at about the same time)
    assert done[1] - done[0] > 0.5 * (done[0] - subs[0]), "the large requests ran side by side"
    for d in done[2:]:
        assert d < done[0], "a small request waited behind the large ones"
    for p, (info, x, _) in zip(bigs + smalls, got):
        assert info.status == 0 and info.true_relres <= 1e-8
        if pack_rows and p.n <= pack_rows:
            oinfo, ox = _pack_of_one(p, pc)
        else:
            oinfo, ox = _alone(p, pc, 8000)
        assert info.iters == oinfo.iters and np.array_equal(x, ox), p.name


def test_server_refuses_reserving_every_slot(lib):
    """The configuration is checked before any device work."""
    with pytest.raises(gs2.GS2Error, match="bad server configuration"):
        gs2.Server(max_slots=2, small_rows=100, small_slots=2)
    with pytest.raises(gs2.GS2Error, match="bad server configuration"):
        gs2.Server(max_slots=2, small_rows=-1, small_slots=1)

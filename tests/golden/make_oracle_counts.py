"""Write oracle_counts.txt: full-size GMRES iteration counts of the FP64 CPU
oracle on the seeded synthetic workloads.

Only the oracle (and the input generators) run here.  The counts are the
expected values of the full-size parity tests (GPU count within +-1) and the
scale factor that turns a timed sample of oracle Arnoldi steps into solves/s.

    python tests/golden/make_oracle_counts.py            # every case
    python tests/golden/make_oracle_counts.py KEY ...    # recompute these keys only
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2104_01196_gb300 import problems as P  # noqa: E402

CASES = [
    # (key, problem builder, preconditioner keywords of oracle.gmres)
    ("poisson2d_64_gmres30_gs2_1_1", lambda: P.poisson2d(64),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.FORWARD)),
    ("poisson3d_128_gmres30_sgs2_1_1", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_gmres30_sgs2_1_2", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=2, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_gmres30_sgs2_1_3", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=3, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_gmres30_sgs_exact", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_gmres30_mtsgs", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_MTGS, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_gmres30_jr3_w1.0", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_JR, pc_outer=3, pc_omega=1.0)),
    ("poisson3d_128_gmres30_jr3_w0.8", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_JR, pc_outer=3, pc_omega=0.8)),
    ("poisson3d_128_gmres30_amg_sgs2_1_1", lambda: P.poisson3d(128),
     dict(amg=True, kind=oracle.PC_GS2, inner=1, direction=oracle.SYMMETRIC)),
    ("elasticity3d_64_gmres30_sgs2_1_2_w0.8", lambda: P.elasticity3d(64),
     dict(pc_kind=oracle.PC_GS2, pc_inner=2, pc_omega=0.8, pc_direction=oracle.SYMMETRIC)),
    ("convdiff3d_192_gmres30_sgs2_1_1", lambda: P.convdiff3d(192),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC)),
]


def main(only=(), out=os.path.join(HERE, "oracle_counts.txt")):
    oracle.build()
    header = ["# GMRES(30), x0 = 0, rel. residual 1e-8, max 5000 iterations; FP64 CPU oracle",
              "# written by tests/golden/make_oracle_counts.py"]
    kept = {}
    if only and os.path.exists(out):
        for line in open(out):
            if line.strip() and not line.startswith("#"):
                kept[line.split()[0]] = line.rstrip("\n")
    cache = {}
    for key, mk, pc in CASES:
        if only and key not in only:
            continue
        name = key.split("_gmres")[0]
        if name not in cache:
            cache = {name: mk()}
        pr = cache[name]
        t0 = time.time()
        if pc.get("amg"):
            # smoothed-aggregation hierarchy with the default settings
            # (theta 0.25, 10 levels, coarsest <= 64 rows), one V-cycle
            kw = {k: v for k, v in pc.items() if k != "amg"}
            _, info = oracle.AMG(pr.A).gmres(pr.A, pr.b, restart=30, tol=1e-8,
                                             max_iters=5000, **kw)
        else:
            _, info = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=5000, **pc)
        dt = time.time() - t0
        line = (f"{key} iters={info.iters} cycles={info.cycles} status={info.status} "
                f"true_relres={info.true_relres:.6e} seconds={dt:.1f}")
        print(line, flush=True)
        kept[key] = line
    order = [k for k, _, _ in CASES]
    lines = header + [kept[k] for k in order if k in kept]
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(tuple(sys.argv[1:]))

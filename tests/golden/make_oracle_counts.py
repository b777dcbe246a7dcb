"""Write oracle_counts.txt: full-size GMRES iteration counts of the FP64 CPU
oracle on the seeded synthetic workloads.

Only the oracle (and the input generators) run here.  The counts are the
expected values of the full-size parity tests (GPU count within +-1) and the
scale factor that turns a timed sample of oracle Arnoldi steps into solves/s.

    python tests/golden/make_oracle_counts.py            # every case
    python tests/golden/make_oracle_counts.py KEY ...    # recompute these keys only
    python tests/golden/make_oracle_counts.py --jobs 6 [KEY ...]   # cases in parallel

Keys ending in _fp32 / _fp16 run the GS2 preconditioner's inner sweeps in
that precision, _fp32_sweep / _fp16_sweep the whole sweep (the oracle's
lowprec.c definitions); everything else is FP64.
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
    # lower-precision inner sweeps (Sec. 10) and the second elasticity setting
    ("poisson3d_128_gmres30_sgs2_1_1_fp32", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp32")),
    ("poisson3d_128_gmres30_sgs2_1_1_fp16", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp16")),
    ("elasticity3d_64_gmres30_sgs2_1_2_w0.8_fp32", lambda: P.elasticity3d(64),
     dict(pc_kind=oracle.PC_GS2, pc_inner=2, pc_omega=0.8, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp32")),
    ("elasticity3d_64_gmres30_sgs2_1_3_w0.9", lambda: P.elasticity3d(64),
     dict(pc_kind=oracle.PC_GS2, pc_inner=3, pc_omega=0.9, pc_direction=oracle.SYMMETRIC)),
    ("elasticity3d_64_gmres30_sgs2_1_3_w0.9_fp32", lambda: P.elasticity3d(64),
     dict(pc_kind=oracle.PC_GS2, pc_inner=3, pc_omega=0.9, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp32")),
    ("convdiff3d_192_gmres30_sgs2_1_1_fp32", lambda: P.convdiff3d(192),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp32")),
    ("convdiff3d_192_gmres30_sgs2_1_1_fp16", lambda: P.convdiff3d(192),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp16")),
    # the whole sweep in single precision (residual and iterate too)
    ("poisson3d_128_gmres30_sgs2_1_1_fp32_sweep", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp32_sweep")),
    ("poisson3d_128_gmres30_sgs2_1_1_fp16_sweep", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp16_sweep")),
    ("convdiff3d_192_gmres30_sgs2_1_1_fp32_sweep", lambda: P.convdiff3d(192),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp32_sweep")),
    ("convdiff3d_192_gmres30_sgs2_1_1_fp16_sweep", lambda: P.convdiff3d(192),
     dict(pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
          pc_precision="fp16_sweep")),
    # compact GS2 of Eq. (9) as the GMRES preconditioner; CG (tol 1e-8) with
    # SGS2(1,1) and with the AMG V-cycle
    ("poisson3d_128_gmres30_compact_sgs2_1_2", lambda: P.poisson3d(128),
     dict(pc_kind=oracle.PC_GS2_COMPACT, pc_inner=2, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_cg_sgs2_1_1", lambda: P.poisson3d(128),
     dict(cg=True, pc_kind=oracle.PC_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC)),
    ("poisson3d_128_cg_amg_sgs2_1_1", lambda: P.poisson3d(128),
     dict(cg=True, amg=True, kind=oracle.PC_GS2, inner=1, direction=oracle.SYMMETRIC)),
]

# the hybrid (block-Jacobi) preconditioners of Sec. 3 on the 128^3 Laplacian,
# P contiguous row blocks: global JR(4,1), local JR(1,4), hybrid SGS2(1,1)
# and hybrid exact SGS
for _P in (1, 8, 64, 512):
    CASES += [
        (f"poisson3d_128_gmres30_hybrid_jr_4_1_P{_P}", lambda: P.poisson3d(128),
         dict(pc_kind=oracle.PC_HYBRID_JR, pc_outer=4, pc_parts=_P, pc_local=1)),
        (f"poisson3d_128_gmres30_hybrid_jr_1_4_P{_P}", lambda: P.poisson3d(128),
         dict(pc_kind=oracle.PC_HYBRID_JR, pc_outer=1, pc_parts=_P, pc_local=4)),
        (f"poisson3d_128_gmres30_hybrid_sgs2_1_1_P{_P}", lambda: P.poisson3d(128),
         dict(pc_kind=oracle.PC_HYBRID_GS2, pc_inner=1, pc_direction=oracle.SYMMETRIC,
              pc_parts=_P)),
        (f"poisson3d_128_gmres30_hybrid_sgs_P{_P}", lambda: P.poisson3d(128),
         dict(pc_kind=oracle.PC_HYBRID_GS, pc_direction=oracle.SYMMETRIC, pc_parts=_P)),
    ]
CASES.append(("poisson2d_64_cg_sgs2_1_1", lambda: P.poisson2d(64),
              dict(cg=True, pc_kind=oracle.PC_GS2, pc_inner=1,
                   pc_direction=oracle.SYMMETRIC)))

# One-ulp ensembles: the same solve with b multiplied entrywise by
# (1 + 2^-52 e), e ~ N(0, 1) from numpy's seeded generator (seed = member),
# where the count is sensitive to rounding (FP32 preconditioning of the 64^3
# elasticity problem): keys <case>_ens<member>.
ENSEMBLE_MEMBERS = 8
for _base in ("elasticity3d_64_gmres30_sgs2_1_2_w0.8_fp32",
              "elasticity3d_64_gmres30_sgs2_1_3_w0.9_fp32"):
    _, _mk, _pc = next(c for c in CASES if c[0] == _base)
    for _m in range(1, ENSEMBLE_MEMBERS + 1):
        CASES.append((f"{_base}_ens{_m}", _mk, dict(_pc, perturb=_m)))


def run_case(key):
    """One case through the oracle: its line of oracle_counts.txt."""
    oracle.build()
    _, mk, pc = next(c for c in CASES if c[0] == key)
    pr = mk()
    t0 = time.time()
    kw = {k: v for k, v in pc.items() if k not in ("amg", "cg", "perturb")}
    if pc.get("perturb"):
        import numpy as np
        rng = np.random.default_rng(pc["perturb"])
        pr.b = pr.b * (1.0 + 2.0 ** -52 * rng.standard_normal(pr.n))
    if pc.get("amg"):
        # smoothed-aggregation hierarchy with the default settings
        # (theta 0.25, 10 levels, coarsest <= 64 rows), one V-cycle
        M = oracle.AMG(pr.A)
        if pc.get("cg"):
            _, info = M.cg(pr.A, pr.b, tol=1e-8, max_iters=5000, **kw)
        else:
            _, info = M.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=5000, **kw)
    elif pc.get("cg"):
        _, info = oracle.cg(pr.A, pr.b, tol=1e-8, max_iters=5000, **kw)
    else:
        _, info = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=5000, **kw)
    dt = time.time() - t0
    line = (f"{key} iters={info.iters} cycles={info.cycles} status={info.status} "
            f"true_relres={info.true_relres:.6e} seconds={dt:.1f}")
    print(line, flush=True)
    return line


def main(only=(), out=os.path.join(HERE, "oracle_counts.txt"), jobs=1):
    oracle.build()
    header = ["# GMRES(30) (CG where the key says cg), x0 = 0, rel. residual 1e-8, "
              "max 5000 iterations; FP64 CPU oracle",
              "# (keys ending _fp32 / _fp16: GS2 inner sweeps in that precision)",
              "# written by tests/golden/make_oracle_counts.py"]
    kept = {}
    if only and os.path.exists(out):
        for line in open(out):
            if line.strip() and not line.startswith("#"):
                kept[line.split()[0]] = line.rstrip("\n")
    keys = [k for k, _, _ in CASES if not only or k in only]
    if jobs > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(jobs) as pool:
            lines = pool.map(run_case, keys, chunksize=1)
    else:
        lines = [run_case(k) for k in keys]
    for k, line in zip(keys, lines):
        kept[k] = line
    order = [k for k, _, _ in CASES]
    lines = header + [kept[k] for k in order if k in kept]
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    args = sys.argv[1:]
    jobs = 1
    if args[:1] == ["--jobs"]:
        jobs, args = int(args[1]), args[2:]
    main(tuple(args), jobs=jobs)

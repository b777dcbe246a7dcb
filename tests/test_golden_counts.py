"""The stored oracle counts (tests/golden/oracle_counts.txt, written by
tests/golden/make_oracle_counts.py from the oracle alone) cover every
iteration count the benchmark reports beside its own, every stored solve
converged, and the one-ulp ensembles behind the FP32 elasticity checks are
complete and do spread (the reason those checks use a range)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_counts.txt")


def _lines():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            key, *fields = line.split()
            out[key] = dict(f.split("=", 1) for f in fields)
    return out


def test_every_reported_count_is_stored():
    import bench
    have = _lines()
    want = set(bench.ORACLE_KEYS.values())
    want |= {"convdiff3d_192_gmres30_sgs2_1_1", "poisson3d_128_gmres30_sgs2_1_1",
             "poisson2d_64_gmres30_gs2_1_1", "poisson2d_64_cg_sgs2_1_1"}
    want |= {f"convdiff3d_192_gmres30_sgs2_1_1_{p}"
             for p in ("fp32", "fp16", "fp32_sweep", "fp16_sweep")}
    for stem in ("sgs2_1_2_w0.8", "sgs2_1_3_w0.9"):
        want |= {f"elasticity3d_64_gmres30_{stem}", f"elasticity3d_64_gmres30_{stem}_fp32"}
    for P in (1, 8, 64, 512):
        for k in ("jr_4_1", "jr_1_4", "sgs2_1_1", "sgs"):
            want.add(f"poisson3d_128_gmres30_hybrid_{k}_P{P}")
    missing = sorted(want - set(have))
    assert not missing, missing


def test_stored_solves_converged():
    for key, f in _lines().items():
        assert f["status"] == "0", key
        assert float(f["true_relres"]) <= 1e-8, key


@pytest.mark.parametrize("stem", ["sgs2_1_2_w0.8", "sgs2_1_3_w0.9"])
def test_fp32_elasticity_ensembles(stem):
    have = _lines()
    base = f"elasticity3d_64_gmres30_{stem}_fp32"
    members = [int(f["iters"]) for k, f in have.items() if k.startswith(base + "_ens")]
    assert len(members) == 8
    counts = members + [int(have[base]["iters"])]
    assert max(counts) - min(counts) > 2, counts

"""Host-side pieces of bench.py (no GPU): the FP64 work count of one stage that the
roofline uses, and the reference arm's JSON line (the oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_stage_flop_count_of_the_split_stage():
    import bench
    # Euler P2, counted by hand from the face pass and the cell pass (FMA = 2 flops):
    # face: two doubled traces 2 x 4 x 13 (normal sums 2 + 1 FMAs over psi_0, then one
    # FMA at the middle point and an FMA, a product and two additions for the pair), three
    # LLF points 3 x 53, projection 4 x 9;
    # cell: t_b 40, point values 84, fluxes 9 x 18, column sums and x weights 272,
    # scalings 38, lifting 144, stage combination 96 (mean over the three stages)
    fl = bench.stage_flops_per_cell(2, 1, 2)
    assert fl["face"] == 2 * 4 * 13 + 3 * 53 + 4 * 9 == 299
    assert fl["cell"] == 40 + 84 + 9 * 18 + 272 + 38 + 144 + 96 == 836
    assert fl["total"] == 2 * 299 + 836
    # more modes cost more; Burgers less than Euler
    for pde in (0, 1):
        c = [bench.stage_flops_per_cell(2, pde, N)["total"] for N in (1, 2, 3)]
        assert c[0] < c[1] < c[2]
    assert bench.stage_flops_per_cell(2, 0, 2)["total"] < bench.stage_flops_per_cell(2, 1, 2)["total"]


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--size", "96"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "DOF-updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]

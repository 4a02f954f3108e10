"""The reference arm of bench.py (the CPU oracle on a bounded sample) prints
one JSON line with the keys the benchmark contract asks for; no GPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_fp64_pipe_counts_the_smoothers_instructions():
    # FP64 instructions the bench line attributes to a level-0 launch: one FMA
    # per stored entry; none more a row for r = b - (A S) b (negated FMAs from
    # b_i down); b_i + r_i, the final FMA and the (r, z) term for the level-0
    # post-smoother (two a row on coarser levels)
    import argparse

    sys.path.insert(0, ROOT)
    import bench

    class StubHierarchy:
        def level_info(self, level):
            return (1000, 7000)

        def level_layout(self, level, ap=False):
            return {"slots": 5100 if ap else 7040}

    a = argparse.Namespace(precision="f64")
    H = StubHierarchy()
    assert bench.fp64_pipe(H, 0, "pre", 1.0, a)["ops_per_launch"] == 7040
    assert bench.fp64_pipe(H, 0, "post", 1.0, a)["ops_per_launch"] == 5100 + 3 * 1000
    assert bench.fp64_pipe(H, 2, "post", 1.0, a)["ops_per_launch"] == 5100 + 2 * 1000
    assert bench.fp64_pipe(H, 0, "restrict", 1.0, a) is None
    assert bench.fp64_pipe(H, 0, "pre", 1.0, argparse.Namespace(precision="f32")) is None

"""Host-side logic of bench.py that needs no GPU: the workload descriptions, the position cycle with its
model uploads, the padded-volume scaling of the oracle sample, and the reference arm's JSON line on
reduced models."""
import argparse
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_large_workload_cycles_positions_and_uploads_once_per_round():
    bw = bench.BenchWorkload("c5", 0, scale=8)
    assert len(bw.items) == bench.POSITIONS_C5 == 16
    assert [bw.uploads_model(k) for k in range(18)] == [k % 16 == 0 for k in range(18)]
    zs = [bw.item(k).sources[0].pos[2] for k in range(16)]
    assert zs == sorted(zs) and len(set(zs)) == 16
    assert bw.item(16).sources[0].pos == bw.item(0).sources[0].pos
    assert bw.split == [k * (bw.grid.nz // 8) for k in range(9)]
    assert bw.opts["concurrent_blocks"] and bw.opts["outer_krylov"] and bw.dd == "jacobi"
    # one model for all positions
    assert all(it.sigma6 is bw.items[0].sigma6 for it in bw.items)


def test_padded_volume():
    from paper_2306_17537_gb300 import inputs

    g = inputs.centred_grid(256, 256, 512, 0.25)
    assert bench.padded_volume(g, 64) == 512 * 512 * 128
    assert bench.padded_volume(g, 512) == 512 * 512 * 1024
    assert bench.padded_volume(g, 16) * 32 == bench.padded_volume(g, 512)


def _reference_line(workload, scale):
    args = argparse.Namespace(workload=workload, seed=0, scale=scale, operator="contraction", steps=1, warmup=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    return json.loads(buf.getvalue().strip().splitlines()[-1])


def test_reference_arm_line_on_reduced_models():
    for workload, scale in (("c5", 8), ("c2", 8)):
        line = _reference_line(workload, scale)
        assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
        assert line["value"] > 0 and line["higher_is_better"] is True
        assert line["cpu_baseline"]["kind"] == "oracle" and "extrapolation" in line["cpu_baseline"]["sample"]
        assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]

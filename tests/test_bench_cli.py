"""bench.py's command line and report modes resolve without a GPU (no compute calls)."""
import sys

import pytest


def test_report_modes_and_arms_resolve(monkeypatch):
    import bench
    for name in ("run_precision_report", "run_rounds_report", "run_ablation_report", "run_batched_report",
                 "run_serve_report", "run_reference", "oracle_build_rate", "join_algorithmic_bytes", "gist_line",
                 "main"):
        assert callable(getattr(bench, name)), name
    for argv in (["bench.py"], ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                 ["bench.py", "--report", "precision", "--shape", "deep", "--n", "1000"],
                 ["bench.py", "--report", "rounds", "--rounds", "2"], ["bench.py", "--report", "serve"],
                 ["bench.py", "--no-gist", "--steps", "2"]):
        monkeypatch.setattr(sys, "argv", argv)
        a = bench._args()
        assert a.gpus == 1
    # the join's algorithmic bytes: rows, degrees, proposals, redirects (12 + 4 bytes), rechecks
    assert bench.join_algorithmic_bytes(10, 100, 7, 3, 1, 128, 2) == 10 * 128 * 2 + 400 + 56 + 48 + 3 * 128 * 4


def test_traffic_figure_names_the_join_code():
    import bench
    assert len(bench._source_sha()) == 64
    assert bench.TRAFFIC["kernel"] == "rnd_join" and bench.TRAFFIC["bytes_per_launch"] > 0

"""bench.py's command line: every record the default line names exists, and the
single-operation modes that the default line carries are also modes of --workload.
CPU only: parses arguments, launches nothing."""
import sys

import bench


def _defaults(monkeypatch):
    captured = {}

    def fake_ours(args):
        captured["args"] = args
        return 0

    monkeypatch.setattr(bench, "run_ours", fake_ours)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.main() == 0
    return captured["args"]


def test_default_line_records_exist(monkeypatch):
    args = _defaults(monkeypatch)
    names = [w for w in args.workloads.split(",") if w]
    assert names, "the default line carries records"
    for name in names:
        assert name in bench.WORKLOAD_RECORDS, name
        assert callable(bench.WORKLOAD_RECORDS[name])


def test_default_run_is_one_gpu_with_warmup(monkeypatch):
    args = _defaults(monkeypatch)
    assert args.gpus == 1 and args.warmup >= 3 and args.impl == "ours"

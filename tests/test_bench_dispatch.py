"""bench.py's command line (no GPU): every workload form reaches its runner,
the warm-up is never below 3, and the reference arm is selected by --impl."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("argv,runner", [
    ([], "run_gb300"),
    (["--workload", "al4_16", "--precision", "fp64"], "run_gb300"),
    (["--workload", "batch16"], "run_batch"),
    (["--workload", "force_al108_48"], "run_force"),
    (["--workload", "scf_al256_64", "--kerker", "none", "--period", "3"], "run_scf"),
    (["--workload", "warmstart_c4", "--train-steps", "10"], "run_warmstart"),
    (["--impl", "reference"], "run_reference"),
])
def test_dispatch(monkeypatch, argv, runner):
    called = {}
    for name in ("run_gb300", "run_batch", "run_force", "run_scf", "run_warmstart", "run_reference"):
        monkeypatch.setattr(bench, name, lambda a, name=name: called.setdefault("name", (name, a)))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--warmup", "1"] + argv)
    bench.main()
    name, a = called["name"]
    assert name == runner and a.warmup == 3

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


def test_reference_arm_json_line(monkeypatch, capsys):
    """The oracle arm on a small sample of al4_16 prints one JSON line with
    the base contract's keys, the oracle described as its CPU baseline and
    an e2e entry with no host-device bytes."""
    import json
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "al4_16", "--steps", "1",
                                      "--warmup", "3", "--cpu-sample", "8"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}

"""bench.py parses its command line and describes its workloads without a GPU: the
options the benchmark contract uses (--gpus, --steps, --warmup, --impl) and the workload,
solver and serving options; the config of each workload names its sizes."""
import argparse
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_help_lists_the_options():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr
    for opt in ("--gpus", "--steps", "--warmup", "--impl", "--precision", "--refine", "--workload", "--solver",
                "--requests", "--slots", "--rate"):
        assert opt in r.stdout


def test_workload_configs():
    sys.path.insert(0, ROOT)
    import bench
    from synth import CONFIGS
    saved = bench.WORKLOAD
    try:
        for name in ("mid", "three_level"):
            bench.WORKLOAD = name
            c = bench.config_dict(argparse.Namespace(gpus=1, solver="davidson"), "bf16x3+fp64e")
            s = CONFIGS[name]
            assert c["n_mo"] == s.n_mo and c["n_chol"] == s.n_chol and c["n_roots"] == s.n_roots
            assert f"{s.n_mo} orbitals" in c["workload"] and c["excited_state_solver"] == "davidson"
            assert ("three-level" in c["workload"]) == (name == "three_level")
            assert ("two levels" in c["workload"]) == (name == "mid")
    finally:
        bench.WORKLOAD = saved

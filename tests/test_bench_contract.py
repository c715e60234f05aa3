"""The reference arm of bench.py (the CPU oracle on a bounded sample of the
benchmark's workload) prints one JSON line with the benchmark's metric, unit
and workload description, and under a multi-rank launch only rank 0 prints.
Runs on the CPU at 12 qubits (the headline width is 30)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, gpus=None):
    env = dict(os.environ, OMP_NUM_THREADS="2", **(extra_env or {}))
    gpus = gpus if gpus is not None else int(env.get("WORLD_SIZE", "1"))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--qubits", "12",
                           "--steps", "3", "--warmup", "1", "--gpus", str(gpus)], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_json_line():
    r = _run()
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "gates/s"
    assert d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.workload_config(12)["workload"]
    assert d["config"]["gates"] == 12 * 20 + 6 * 20
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_output():
    r = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_gpus_flag_must_match_the_launch():
    """--gpus N without N ranks (no torchrun) fails loudly instead of timing one GPU."""
    r = _run(gpus=8)
    assert r.returncode != 0 and "WORLD_SIZE=1" in r.stderr
    assert r.stdout.strip() == ""


def test_oracle_baselines_beside_the_other_workloads():
    """The oracle timings reported beside the GPU arm's other workloads, on
    narrow stand-ins of each (the bench runs them at full width)."""
    import bench
    out = bench.oracle_baselines(budget_s=0.05, widths={"qft": 12, "random": 12, "variational": 10,
                                                        "adjoint": 10, "batch": 16, "batch_nmax": 13})
    assert set(out) == {"qft10_c128", "qft12_c64", "random12_c128_plain", "variational32_c64", "batch16_c64",
                        "adjoint10_c64"}
    units = {"qft10_c128": "gates/s", "qft12_c64": "gates/s", "random12_c128_plain": "gates/s",
             "variational32_c64": "gates/s", "batch16_c64": "circuits/s", "adjoint10_c64": "gradients/s"}
    for k, v in out.items():
        assert v["kind"] == "oracle" and v["unit"] == units[k] and v["value"] > 0 and v["sample"], k
    assert out["qft10_c128"]["single_thread"] > 0 and out["variational32_c64"]["single_thread"] > 0
    assert out["random12_c128_plain"]["cores"] == 1
    a = out["adjoint10_c64"]
    # two runs of the 290-gate circuit (10 layers of 10 RY, 10 RZ, 9 CZ) per gradient
    assert abs(a["value"] - a["gates_per_s"] / (2 * 290)) < 1e-9 * a["gates_per_s"]


# Command lines of the profiling runs (launch lists and ncu captures of
# the bench's own workloads): the argument parser must keep accepting them.
PROFILING_COMMANDS = [
    "",
    "--mode greedy2 --quick --no-cpu --steps 1 --warmup 1",
    "--mode plain --quick --no-cpu --steps 1 --warmup 1",
    "--mode staged --kmax 3 --quick --no-cpu --steps 2 --warmup 1",
    "--mode tc --quick --no-cpu --steps 2 --warmup 1",
    "--only adjoint24 --warmup 2 --steps 2",
    "--only batch4096 --warmup 1 --steps 1",
    "--qubits 27 --mode staged --kmax 3 --quick --no-cpu --steps 1 --warmup 1",
    "--qubits 27 --mode tc --steps 2 --warmup 1 --quick --no-cpu --no-extra",
    "--quick --no-cpu --mode staged --kmax 3 --steps 2 --warmup 3",
    "--dtype c128 --mode plain --quick --no-cpu --steps 1 --warmup 1",
]


def test_profiling_command_lines_parse():
    import shlex
    import bench
    for cmd in PROFILING_COMMANDS:
        bench.build_parser().parse_args(shlex.split(cmd))

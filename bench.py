"""Benchmark: 30-qubit random circuits (depth 20) on one GB300.

One step = one pass of the hot path over one synthetic circuit: initialise
|0...0>, apply the 900 gates (30 Haar-random SU(2) + 15 CZ on a random
matching per layer), evaluate <sum_i Z_i Z_{i+1}> (double reduction) and draw
1024 shots (integer-CDF sampler).  The metric is logical gates of the unfused
circuit per second (fused and plain execution are both reported).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl qsim|reference]
                    [--dtype c64|c128] [--mode auto|plain|greedy2|staged|tc]

Under torchrun every rank simulates its own circuit (independent units, no
data-path collective; "weak" scaling) and rank 0 prints one JSON line.
``--impl reference`` times the CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2203_08826_gb300 import inputs  # noqa: E402

METRIC = "30q circuit: gates/s and achieved HBM GB/s vs ~8 TB/s; fused vs plain s/circuit"
N_QUBITS, DEPTH = 30, 20  # --qubits overrides the width for small profiling runs
SHOTS = 1024
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes per launch from ncu captures (dram__bytes_read.sum + write.sum),
# scaled to a 30-qubit complex64 launch; see profiles/.  Entries are removed
# whenever the kernel changes.
NCU_TRAFFIC_30Q_C64 = {"sweep_dense1": 17.6e9}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle (CPU) timing
def oracle_gates_per_s(circuit, budget_s: float = 20.0, n_override: int | None = None):
    """Time the oracle gate by gate on the host cores over a bounded prefix of
    the circuit (complex128).  Returns (gates/s, gates timed, qubits, cores)."""
    import oracle
    n = circuit.n if n_override is None else n_override
    gates = circuit.gates if n_override is None else inputs.random_circuit(n, DEPTH, seed=2022).gates
    psi = oracle.zero_state(n)
    done, t0 = 0, time.perf_counter()
    for g in gates:
        oracle.apply_gate(psi, g)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return done / dt, done, n, cores


def host_mem_bytes() -> int:
    try:
        import psutil
        return int(psutil.virtual_memory().available)
    except Exception:
        try:
            with open("/proc/meminfo") as f:
                for l in f:
                    if l.startswith("MemAvailable"):
                        return int(l.split()[1]) * 1024
        except Exception:
            pass
    return 0


def oracle_qubits() -> int:
    # the oracle holds one complex128 state; keep a wide margin of host memory
    return N_QUBITS if host_mem_bytes() > 3 * (16 << 30) else 26


def run_reference(args, ws, rank):
    """The oracle as it stands, on the host cores, on a bounded sample."""
    if rank != 0:
        return
    n = oracle_qubits()
    circ = inputs.random_circuit(n, DEPTH, seed=2022)
    import oracle
    psi = oracle.zero_state(n)
    per_step = 2 if n >= 30 else 30
    gi = 0

    def step():
        nonlocal gi
        for _ in range(per_step):
            oracle.apply_gate(psi, circ.gates[gi % len(circ.gates)])
            gi += 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{per_step} gates per step of the {n}-qubit depth-{DEPTH} random circuit, "
              f"complex128, gate by gate (Eq. 1 loop), OpenMP over {cores} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"random circuit {n} qubits depth {DEPTH} (oracle sample)", "qubits": n},
            "cpu_baseline": {"value": value, "unit": "gates/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_qsim(args, ws, rank, local):
    import torch
    from paper_2203_08826_gb300 import binding as q

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    def barrier():
        if pg:
            pg.barrier()

    n = args.qubits
    circ = inputs.random_circuit(n, DEPTH, seed=2022 + rank)
    ngates = len(circ)
    qc = q.QCircuit(circ)
    ham = inputs.zz_chain(n)
    st = torch.cuda.current_stream()
    state = q.State(n, args.dtype)

    PLAN_MODES = {"greedy2": (q.FUSE_GREEDY2, 2), "staged": (q.FUSE_STAGED, 6), "tc": (q.FUSE_TC, 6)}
    plans = {}
    for name, (mode, k) in PLAN_MODES.items():
        try:
            plans[name] = q.Plan(qc, kmax=k, mode=mode)
        except q.QsimError:
            pass
    chosen = args.mode
    if chosen == "auto":
        chosen = "staged" if "staged" in plans else "plain"

    def step(mode_name, out=None):
        state.init_zero()
        if mode_name == "plain":
            state.run(qc)
        else:
            state.run_fused(plans[mode_name])
        e = state.expectation(ham)
        shots = state.sample(SHOTS, seed=7, counter0=0)
        if out is not None:
            out.append((e, shots))

    def timed(mode_name, warmup, steps, profile=False, clocks=None):
        for _ in range(warmup):
            step(mode_name)
        torch.cuda.synchronize()
        barrier()
        if profile:
            q.profile_reset()
            q.profile_enable(True)
        l0 = q.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        t0 = time.perf_counter()
        for _ in range(steps):
            step(mode_name)
        e1.record(st)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        launches = q.launch_count() - l0
        prof = None
        if profile:
            prof = q.profile_read()
            q.profile_enable(False)
        barrier()
        ms = e0.elapsed_time(e1)
        if pg:
            t = torch.tensor([ms], device="cuda")
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return ms, wall, launches, prof

    # ---- headline: chosen mode, profiled, clocks sampled
    with ClockSampler(local) as clk:
        ms, wall, launches, prof = timed(chosen, args.warmup, args.steps, profile=True)
    clocks = clk.summary()
    total_gates = ngates * args.steps * ws
    value = total_gates / (ms / 1e3)

    # dominant kernel and its roofline
    peak, peak_src = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
    roof = None
    if dom:
        name, d = dom
        avg_ms = d["ms"] / d["launches"]
        bytes_per_launch = d["bytes"] / d["launches"]
        achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
        roof = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": NCU_TRAFFIC_30Q_C64.get(name) if (n == 30 and args.dtype == "c64") else None,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                "launch_share": round(d["ms"] / sum(v["ms"] for v in prof.values()), 4)}
        if args.dtype == "c128" and name in ("sweep_dense1",):
            # complex128 dense sweeps run into the FP64 pipe before HBM
            roof["note"] = "complex128 dense sweep: FP64-ALU bound (8 FMA per amplitude)"

    # ---- the other modes (informational, same circuit)
    others = {}
    for other in ([] if args.quick else ["plain"] + [m for m in plans if m != chosen]):
        if other == chosen:
            continue
        oms, _, ol, _ = timed(other, 1, 1)
        others[other] = {"s_per_circuit": oms / 1e3, "gates_per_s": ngates / (oms / 1e3), "launches": ol}

    # ---- end to end through the public API with host buffers
    amp_bytes = (8 if args.dtype == "c64" else 16) << n
    h_in = torch.zeros(1 << n, dtype=state.tensor.dtype, pin_memory=True)
    h_in[0] = 1
    h_out = torch.empty_like(h_in, pin_memory=True)

    def e2e_step():
        qc_e = q.QCircuit(circ)  # marshal the gate list (the user's call)
        state.from_host_async(h_in)
        if chosen == "plain":
            state.run(qc_e)
        else:
            mode, k = PLAN_MODES[chosen]
            state.run_fused(q.Plan(qc_e, kmax=k, mode=mode))
        e = state.expectation(ham)
        state.to_host_into(h_out)
        return e

    e2e_steps = 0 if args.quick else max(1, min(args.steps, 3))
    for _ in range(max(1, min(args.warmup, 3)) if e2e_steps else 0):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max(time.perf_counter() - t0, 1e-9)
    if pg:
        t = torch.tensor([e2e_s], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": ngates * e2e_steps * ws / e2e_s, "unit": "gates/s", "h2d_bytes_per_step": amp_bytes,
           "d2h_bytes_per_step": amp_bytes + 8} if e2e_steps else None

    # ---- CPU oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not (args.no_cpu or args.quick):
        on = oracle_qubits()
        gps, done, nq, cores = oracle_gates_per_s(circ, budget_s=args.cpu_budget,
                                                  n_override=None if on == n else on)
        cpu = {"value": gps, "unit": "gates/s", "cores": cores, "kind": "oracle",
               "sample": f"first {done} gates of a {nq}-qubit depth-{DEPTH} random circuit, complex128, "
                         f"gate by gate on the host (OpenMP)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.dtype == "c64" else "f64", "data": "synthetic",
            "config": {"workload": f"random circuit, {n} qubits, depth {DEPTH} (Haar SU(2) on every qubit + "
                                   f"CZ on a random perfect matching per layer), |0> start, "
                                   f"<sum Z_i Z_i+1> + {SHOTS} shots per step",
                       "qubits": n, "depth": DEPTH, "gates": ngates, "state": args.dtype, "mode": chosen,
                       "state_bytes": amp_bytes, "l2": "inputs larger than L2 (state 8+ GiB vs 129 MB L2)"},
            "s_per_circuit": ms / 1e3 / args.steps,
            "gpu_launches": launches,
            "roofline": roof, "kernels": prof, "other_modes": others, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qsim", choices=["qsim", "reference"])
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--mode", default="auto", choices=["auto", "plain", "greedy2", "staged", "tc"])
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--qubits", type=int, default=N_QUBITS)
    ap.add_argument("--quick", action="store_true",
                    help="headline mode only (no other modes, end-to-end or CPU legs): for profiling runs")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_qsim(args, ws, rank, local)


if __name__ == "__main__":
    main()

"""Host-side checks of libqsim that need no GPU: the C ABI loads and exports
every declared symbol, argument validation, and the fusion planner."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def q():
    from paper_2203_08826_gb300 import build, binding
    build.build()
    binding.lib()
    return binding


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"QSIM_API\s+[\w\s\*]*?\b(qsim_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(q):
    names = declared_symbols()
    assert len(names) >= 30
    lib = q.lib()
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert "sm_103a" in q.version()


def test_binding_covers_declared_symbols(q):
    assert declared_symbols() <= set(q._SIGS)


def test_circuit_validation(q):
    lib = q.lib()
    h = ctypes.c_void_p()
    assert lib.qsim_circuit_create(4, ctypes.byref(h)) == 0
    t = (ctypes.c_int * 2)(1, 1)
    rc = lib.qsim_circuit_add(h, q.GATE_KIND["cz"], t, 2, None, 0, None, -1, None)
    assert rc == -1 and b"twice" in lib.qsim_last_error()
    t = (ctypes.c_int * 1)(4)
    rc = lib.qsim_circuit_add(h, q.GATE_KIND["h"], t, 1, None, 0, None, -1, None)
    assert rc == -1 and b"outside" in lib.qsim_last_error()
    t = (ctypes.c_int * 1)(0)
    rc = lib.qsim_circuit_add(h, q.GATE_KIND["cz"], t, 1, None, 0, None, -1, None)
    assert rc == -1
    # only rotation angles can be trainable
    rc = lib.qsim_circuit_add(h, q.GATE_KIND["h"], t, 1, None, 0, None, 3, None)
    assert rc == -1
    assert lib.qsim_circuit_destroy(h) == 0
    assert lib.qsim_circuit_create(0, ctypes.byref(h)) == -1


def test_qcircuit_counts(q):
    c = inputs.variational(6, 3, seed=1)
    qc = q.QCircuit(c)
    assert qc.ngates == len(c) and qc.nparams == c.nparams == 36


def _asap_depth(n, qubit_sets):
    level = [0] * n
    for qs in qubit_sets:
        l = 1 + max(level[x] for x in qs)
        for x in qs:
            level[x] = l
    return max(level)


def test_greedy2_fusion_reproduces_paper_qft_counts(q):
    """Sec. 3.2 fusion on the 30-qubit QFT gives the fused size of the paper's
    benchmark-circuit table (450 gates, depth 58)."""
    row = [l.split() for l in open(os.path.join(GOLDEN, "benchmark_circuits_table.txt"))
           if l.strip() and not l.startswith("#")][0]
    n, fdepth, fgates = int(row[1]), int(row[4]), int(row[5])
    plan = q.Plan(inputs.qft(n), kmax=2, mode=q.FUSE_GREEDY2)
    info = plan.info()
    assert info["sweeps"] == fgates and info["gates"] == 480
    sets = [plan.block(i)[0] for i in range(info["sweeps"])]
    assert _asap_depth(n, sets) == fdepth


def test_greedy2_blocks_equal_product_of_oracle_gates(q, orc):
    """Each fused matrix equals the product of its source gates' matrices, as
    built by the oracle and embedded by Kronecker products (independent of the
    planner's own embedding)."""
    from tests.test_oracle_pins import kron_operator
    circ = inputs.random_circuit(5, 3, seed=4)
    plan = q.Plan(circ, kmax=2, mode=q.FUSE_GREEDY2)
    n = circ.n
    U_plan = np.eye(1 << n, dtype=complex)
    for i in range(plan.info()["sweeps"]):
        t, m = plan.block(i)
        U_plan = kron_operator(n, m, t) @ U_plan
    U_ref = np.eye(1 << n, dtype=complex)
    for g in circ.gates:
        U_ref = kron_operator(n, orc.gate_matrix(g), g.targets, g.controls) @ U_ref
    np.testing.assert_allclose(U_plan, U_ref, atol=1e-13)
    assert plan.info()["sweeps"] < len(circ)


def _tc_mixed_circuit(n, seed):
    """Dense 1- and 2-qubit gates on near and distant qubits, controlled and
    diagonal gates across windows, distant SWAPs and 3-qubit dense gates
    (the last two need plain passes)."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(4):
        for q_ in range(n):
            gates.append(inputs.Gate("su2", (q_,), (), inputs.haar_su2_quaternion(rng)))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        gates.append(inputs.Gate("matrix", (a, b), (), (), -1, inputs.random_dense_gate(rng, 2)))
        gates.append(inputs.Gate("phase", (a,), (b,), (float(rng.uniform(0, 6)),)))
        gates.append(inputs.Gate("cz", (0, n - 1)))
        gates.append(inputs.Gate("rzz", (1, n - 2), (), (float(rng.uniform(0, 6)),)))
        gates.append(inputs.Gate("x", (2,), (n - 3, 5)))
        gates.append(inputs.Gate("swap", (3, n - 4)))
        c3 = tuple(int(v) for v in rng.choice(n, 3, replace=False))
        gates.append(inputs.Gate("matrix", c3, (), (), -1, inputs.random_dense_gate(rng, 3)))
        # a permutation with phases that is not its own inverse (row r has its
        # entry in column r + 1 mod 8): a transposed permutation convention
        # anywhere in the planners changes the result
        cyc = np.zeros((8, 8), dtype=complex)
        for r in range(8):
            cyc[r, (r + 1) % 8] = np.exp(1j * rng.uniform(0, 6))
        c3 = tuple(int(v) for v in rng.choice(n, 3, replace=False))
        gates.append(inputs.Gate("matrix", c3, (), (), -1, cyc))
    return inputs.Circuit(n, gates, "tc-mixed")


@pytest.mark.parametrize("kmax", [5, 6])
@pytest.mark.parametrize("maker", ["random", "variational", "qft", "mixed"])
def test_tensor_core_plan_replays_the_circuit(q, orc, maker, kmax):
    """The tensor-core planner's passes -- fused window blocks, their diagonal
    epilogues and plain passes -- applied in order by the oracle in complex128
    give the circuit's own gate-by-gate result (Eq. (1)) to rounding: the
    planner's fusion, deferral and commutation choices, checked without a GPU
    and without the split precision of the tensor cores."""
    n = 14
    circ = {"random": lambda: inputs.random_circuit(n, 5, seed=3),
            "variational": lambda: inputs.variational(n, 3, seed=4),
            "qft": lambda: inputs.qft(n),
            "mixed": lambda: _tc_mixed_circuit(n, seed=5)}[maker]()
    psi0 = inputs.gaussian_state(n, seed=6)
    want = orc.simulate(circ, psi0)
    plan = q.Plan(circ, kmax=kmax, mode=q.FUSE_TC)
    psi = psi0.copy()
    passes = plan.tc_passes()
    for ps in passes:
        orc.apply_matrix(psi, ps["matrix"], ps["targets"], ps["controls"])
        for e in ps["epilogue"]:
            orc.apply_matrix(psi, np.diag(e["diag"]), e["targets"], e["controls"])
    assert np.max(np.abs(psi - want)) < 1e-12
    assert len(passes) == plan.info()["sweeps"]
    # windows of kmax qubits; 6-wide plans close the rotation with 5s and 6s
    assert {len(p["targets"]) for p in passes if not p["plain"]} <= ({5, 6} if kmax == 6 else {5})
    if maker == "mixed":
        assert any(p["plain"] for p in passes) and any(p["epilogue"] for p in passes)


@pytest.mark.parametrize("kmax", [1, 3, 4])
@pytest.mark.parametrize("maker", ["random", "variational", "qft", "mixed"])
def test_staged_plan_schedule_replays_the_circuit(q, orc, maker, kmax):
    """The staged planner's schedule (which of the circuit's gates each stage
    applies, in which order, on which tile): every gate is applied exactly
    once, the oracle replaying the gates in that order gives the gate-by-gate
    result (so no reordering crosses a gate it does not commute with), and a
    tile stage applies a non-diagonal gate only to qubits of its tile (lanes
    0..4 and the stage's 4 + min(kmax, 4) slots)."""
    n = 14
    circ = {"random": lambda: inputs.random_circuit(n, 5, seed=3),
            "variational": lambda: inputs.variational(n, 3, seed=4),
            "qft": lambda: inputs.qft(n),
            "mixed": lambda: _tc_mixed_circuit(n, seed=5)}[maker]()
    psi0 = inputs.gaussian_state(n, seed=6)
    stages = q.Plan(circ, kmax=kmax, mode=q.FUSE_STAGED).stages()
    order = [gi for st in stages for gi in st["gates"]]
    assert sorted(order) == list(range(len(circ)))
    psi = psi0.copy()
    for gi in order:
        orc.apply_gate(psi, circ.gates[gi])
    assert np.max(np.abs(psi - orc.simulate(circ, psi0))) < 1e-12
    for st in stages:
        if st["plain"]:
            assert len(st["gates"]) == 1 and not st["slots"]
            continue
        assert len(st["slots"]) == 4 + min(kmax, 4)
        tile = set(range(5)) | set(st["slots"])
        for gi in st["gates"]:
            m = orc.gate_matrix(circ.gates[gi])
            if not np.array_equal(m, np.diag(np.diag(m))):
                assert set(circ.gates[gi].targets) <= tile, (gi, circ.gates[gi])


def test_pair_fusion_absorbs_the_random_circuits_one_qubit_gates(q):
    """Pair fusion on the 30-qubit depth-20 random circuit: 150 of its 300 CZ
    (lane qubits included) become dense 4x4 ops that take in all 600
    1-qubit gates, so no stage applies a 1-qubit op; the rest stay sign
    flips."""
    import re
    d = q.Plan(inputs.random_circuit(30, 20, seed=2022), kmax=3, mode=q.FUSE_STAGED).describe()
    count = lambda key: sum(int(x) for x in re.findall(key + r"=(\d+)", d))
    assert count("u2") == 150
    assert count("u1") == 0 and count("reg") == 0 and count("lane") == 0
    # arithmetic per amplitude: the circuit's 600 dense 1-qubit gates one
    # sweep each (16 flops, the CZ none) against 150 fused 4x4 (32 flops)
    fl = q.Plan(inputs.random_circuit(30, 20, seed=2022), kmax=3, mode=q.FUSE_STAGED).flops()
    assert fl == {"executed": 150 * 32.0, "circuit": 600 * 16.0}


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_specialized_stage_source_compiles(q, tmp_path, dtype):
    """The source the library writes for a plan's specialised stage kernels
    (one kernel per tile stage, here with lane and register 4x4 ops,
    controls, diagonals, sign flips and exchanges) compiles for sm_103a, and
    the plan reports the flag; the source holds no coefficient values."""
    import shutil
    import subprocess
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from test_gpu_fused import lane_pair_circuit, mixed_circuit
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    for circ in (mixed_circuit(14, seed=7), lane_pair_circuit(14, seed=8)):
        p = q.Plan(circ, kmax=3, mode=q.FUSE_STAGED | q.SPECIALIZE)
        assert p.info()["mode"] == q.FUSE_STAGED | q.SPECIALIZE
        src = p.source(dtype)
        nst = sum(1 for st in p.stages() if not st["plain"])
        assert src.count("__global__") == nst > 0
        # complex64 register ops in paired FP32 with host-made coefficient
        # pairs; complex128 in scalar FP64
        paired = ("u2p(" in src or "u1p(" in src) and " u64 cc[" in src
        assert paired == (dtype == "c64")
        f = tmp_path / f"stages_{dtype}.cu"
        f.write_text(src)
        r = subprocess.run([nvcc, "-cubin", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                            str(f), "-o", str(tmp_path / "stages.cubin")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
    with pytest.raises(q.QsimError):
        q.Plan(inputs.random_circuit(14, 2, seed=1), kmax=6, mode=q.FUSE_TC | q.SPECIALIZE)


def test_specialized_source_depends_on_structure_only(q):
    """The generated stage kernels take the coefficients as parameters: two
    random circuits that differ only in their 1-qubit gates' angles give the
    same source (one compiled module serves both), and a different
    structure gives another."""
    a = inputs.random_circuit(16, 6, seed=3)
    rng = np.random.default_rng(11)
    b = inputs.Circuit(16, [inputs.Gate(g.name, g.targets, g.controls, inputs.haar_su2_quaternion(rng))
                            if g.name == "su2" else g for g in a.gates])
    c = inputs.random_circuit(16, 6, seed=4)
    src = lambda circ: q.Plan(circ, kmax=3, mode=q.FUSE_STAGED | q.SPECIALIZE).source("c64")
    assert src(a) == src(b)
    assert src(a) != src(c)
    assert "p.c[" in src(a) and not re.search(r"\d\.\d{4,}", src(a))  # no coefficient value in the text


def test_staged_plan_splits_a_stage_over_the_parameter_limit(q, orc):
    """120 dense 2-qubit gates that all fit one tile outgrow one kernel
    parameter block (768 complex coefficients, 16 per 4x4): the planner
    retries with a prefix of its picks, and the stages still replay the
    circuit."""
    rng = np.random.default_rng(1)
    n = 12
    gates = []
    for _ in range(120):
        a, b = (int(v) for v in rng.choice(range(5, 12), 2, replace=False))
        gates.append(inputs.Gate("matrix", (a, b), (), (), -1, inputs.random_dense_gate(rng, 2)))
    circ = inputs.Circuit(n, gates)
    stages = q.Plan(circ, kmax=3, mode=q.FUSE_STAGED).stages()
    assert len(stages) >= 3 and all(len(st["gates"]) <= 48 for st in stages)
    order = [gi for st in stages for gi in st["gates"]]
    assert sorted(order) == list(range(len(circ)))
    psi0 = inputs.gaussian_state(n, seed=2)
    psi = psi0.copy()
    for gi in order:
        orc.apply_gate(psi, circ.gates[gi])
    assert np.max(np.abs(psi - orc.simulate(circ, psi0))) < 1e-12


def test_lookahead_planner_stage_counts(q):
    """The lookahead planner on the 30-qubit depth-20 random circuit: 26
    stages at kmax 3 and 22 at kmax 4 (the one-pass schedule needed 31 and
    27), each stage's tile within 4 + kmax slots."""
    c = inputs.random_circuit(30, 20, seed=2022)
    for kmax, want in ((3, 26), (4, 22)):
        p = q.Plan(c, kmax=kmax, mode=q.FUSE_STAGED)
        stages = p.stages()
        assert len(stages) == want
        assert all(len(st["slots"]) == 4 + kmax for st in stages if not st["plain"])


@pytest.mark.parametrize("kmax", [1, 3, 4])
@pytest.mark.parametrize("maker", ["random", "variational", "qft", "mixed", "lanes"])
def test_stage_op_lists_replay_the_circuit(q, orc, maker, kmax):
    """The op lists a staged plan gives its kernels (qsim_plan_stage_dump:
    fused 4x4 blocks, batched 1-qubit ops, lane ops with their coefficient
    layouts, controls, diagonals, sign-flip batches, exchanges between
    phases), run by a host model of the kernels' data layout in complex128,
    against the oracle's gate-by-gate result."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import stage_emulator
    from test_gpu_fused import lane_pair_circuit, mixed_circuit
    n = 14
    circ = {"random": lambda: inputs.random_circuit(n, 5, seed=3),
            "variational": lambda: inputs.variational(n, 3, seed=4),
            "qft": lambda: inputs.qft(n),
            "mixed": lambda: mixed_circuit(n, seed=7),
            "lanes": lambda: lane_pair_circuit(n, seed=8)}[maker]()
    psi0 = inputs.gaussian_state(n, seed=6)
    plan = q.Plan(circ, kmax=kmax, mode=q.FUSE_STAGED)
    got = stage_emulator.run_plan(plan, circ, psi0, orc)
    assert np.max(np.abs(got - orc.simulate(circ, psi0))) < 1e-12


@pytest.mark.parametrize("n", [9, 10, 12, 17])
@pytest.mark.parametrize("maker", ["random", "mixed"])
def test_stage_op_lists_replay_at_other_widths(q, orc, maker, n):
    """The host model of the stage kernels at tile widths below the default
    (n = 9..12: fewer warp qubits than kmax asks for) and with tile qubits
    up to qubit 16 (many tiles), against the oracle."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import stage_emulator
    from test_gpu_fused import mixed_circuit
    circ = inputs.random_circuit(n, 4, seed=n) if maker == "random" else mixed_circuit(n, seed=n, depth=3)
    psi0 = inputs.gaussian_state(n, seed=1)
    for kmax in (3, 4):
        plan = q.Plan(circ, kmax=kmax, mode=q.FUSE_STAGED)
        got = stage_emulator.run_plan(plan, circ, psi0, orc)
        assert np.max(np.abs(got - orc.simulate(circ, psi0))) < 1e-12, (maker, n, kmax)


def test_plan_block_only_for_greedy_plans(q):
    c = inputs.random_circuit(14, 3, seed=1)
    for mode, k in ((q.FUSE_STAGED, 3), (q.FUSE_TC, 6)):
        with pytest.raises(q.QsimError):
            q.Plan(c, kmax=k, mode=mode).block(0)
    g = q.Plan(c, kmax=2, mode=q.FUSE_GREEDY2)
    t, m = g.block(g.info()["sweeps"] - 1)
    assert m.shape == (1 << len(t), 1 << len(t))
    with pytest.raises(q.QsimError):
        g.block(g.info()["sweeps"])


def test_plan_rejects_bad_mode(q):
    with pytest.raises(q.QsimError):
        q.Plan(inputs.qft(4), kmax=2, mode=7)


def test_staged_and_tc_plans_describe(q):
    c = inputs.random_circuit(30, 20, seed=2022)
    st = q.Plan(c, kmax=4, mode=q.FUSE_STAGED)
    assert st.info()["gates"] == 900 and "tile" in st.describe()
    tc = q.Plan(c, kmax=6, mode=q.FUSE_TC)
    info = tc.info()
    assert info["gates"] == 900 and info["sweeps"] % 5 == 0  # 30 qubits = 5 windows of 6
    assert "BF16x3" in tc.describe()
    assert "3xTF32" in q.Plan(c, kmax=5, mode=q.FUSE_TC).describe()
    with pytest.raises(q.QsimError):
        q.Plan(inputs.random_circuit(10, 2, seed=1), kmax=6, mode=q.FUSE_TC)


def test_complex64_sampler_weights_match_their_definition():
    """The sampler computes complex64 weights with integer arithmetic only;
    they must equal floor(RN_double(re^2 + im^2) * 2^62) exactly (exact
    rational arithmetic here), across magnitudes, subnormals and specials."""
    import math
    from fractions import Fraction
    from paper_2203_08826_gb300 import binding
    lib = binding.lib()

    def want(re, im):
        x, y = float(np.float32(re)), float(np.float32(im))
        if math.isnan(x) or math.isnan(y):
            return 0
        if math.isinf(x) or math.isinf(y):
            return 1 << 62
        p = float(Fraction(x) ** 2 + Fraction(y) ** 2)  # one correct rounding to double
        return 1 << 62 if p >= 1.0 else int(Fraction(p) * (1 << 62))

    cases = [(0.0, 0.0), (1.0, 0.0), (-0.0, 1.0), (0.6, 0.8), (1e-45, 0.0), (1e-45, 1e-45), (3e-39, 1e-45),
             (2.0 ** -75, 2.0 ** -100), (0.70710677, 0.70710677), (float("inf"), 0.0), (float("nan"), 1.0),
             (-0.5, -0.5), (1.0000001, 0.0)]
    rng = np.random.default_rng(3)
    # 2^-15: amplitudes of a 30-qubit state (about one in a thousand of these
    # takes the exact route after the short one); 2^-10 and 2^-32 straddle the
    # bounds of the short route
    for scale, count in ((1.0, 1500), (1e-5, 1500), (2.0 ** -15, 12000), (2.0 ** -10, 3000),
                         (2.0 ** -32, 3000), (1e-12, 1500), (1e-30, 1500), (1e-40, 1500)):
        xs = (rng.standard_normal(count) * scale).astype(np.float32)
        ys = (rng.standard_normal(count) * scale * rng.choice([1, 1e-3, 1e-9], count)).astype(np.float32)
        cases += list(zip(xs.tolist(), ys.tolist()))
    for re, im in cases:
        assert lib.qsim_sampler_weight_c64(re, im) == want(re, im), (re, im)
        x, y = float(np.float32(re)), float(np.float32(im))
        if math.isinf(x) or math.isinf(y):
            assert lib.qsim_prob_c64(re, im) == math.inf
        elif not (math.isnan(x) or math.isnan(y)):
            assert lib.qsim_prob_c64(re, im) == float(Fraction(x) ** 2 + Fraction(y) ** 2), (re, im)


def test_tensor_core_pass_precisions_host(q):
    """Per-pass arithmetic of a tensor-core plan (host only): every pass
    starts at its window's split, any mix of BF16x3, 3xTF32 (5-qubit windows
    only) and FP32 can be set and read back, bad values are refused."""
    c = inputs.random_circuit(16, 4, seed=2)
    p6 = q.Plan(c, kmax=6, mode=q.FUSE_TC)
    p5 = q.Plan(c, kmax=5, mode=q.FUSE_TC)
    m6, m5 = p6.info()["sweeps"], p5.info()["sweeps"]
    assert p6.tc_precisions() == [q.PREC_BF16X3] * m6
    assert p5.tc_precisions() == [q.PREC_TF32X3] * m5
    ks = [0 if ps["plain"] else len(ps["targets"]) for ps in p6.tc_passes()]
    mix = [q.PREC_FP32 if i % 3 == 0 else (q.PREC_TF32X3 if k == 5 else q.PREC_BF16X3) for i, k in enumerate(ks)]
    p6.set_tc_precisions(mix)
    assert p6.tc_precisions() == mix
    assert "fp32" in p6.describe()
    with pytest.raises(q.QsimError):
        p6.set_tc_precisions(mix[:-1])
    with pytest.raises(q.QsimError):
        p6.set_tc_precisions([7] * m6)
    if 6 in ks:
        with pytest.raises(q.QsimError):
            p6.set_tc_precisions([q.PREC_TF32X3] * m6)
    assert p6.tc_precisions() == mix  # a refused setting changes nothing
    p5.set_tc_precisions([q.PREC_FP32] * m5)
    assert p5.tc_precisions() == [q.PREC_FP32] * m5
    st = q.Plan(c, kmax=3, mode=q.FUSE_STAGED)
    with pytest.raises(q.QsimError):
        st.set_tc_precisions([0])


def test_release_build_has_no_index_checks(q):
    """qsim_debug_checks is exported by both builds; the release library
    reports -1 (no checks compiled in)."""
    assert q.lib().qsim_debug_checks(0) == -1

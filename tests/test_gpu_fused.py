"""GPU parity of the fused execution modes (staged tiles, tensor-core blocks)
against the gate-by-gate CPU oracle."""
import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_08826_gb300 import build, binding
    build.build()
    return binding


def run_plan(q, circ, dtype, psi0, mode, kmax):
    s = q.State(circ.n, dtype)
    if psi0 is None:
        s.init_zero()
    else:
        s.from_host(psi0)
    s.run_fused(q.Plan(circ, kmax=kmax, mode=mode))
    return s.to_host().astype(np.complex128)


def mixed_circuit(n, seed, depth=6):
    """Every gate kind the stage interpreter handles, plus ones it hands back
    to plain sweeps: dense 1q/2q/3q, controlled gates with controls inside and
    outside the tile, diagonals on any qubits, permutations, lane targets."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(depth):
        for q_ in rng.permutation(n)[: n // 2]:
            gates.append(inputs.Gate("su2", (int(q_),), (), inputs.haar_su2_quaternion(rng)))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        gates.append(inputs.Gate("matrix", (a, b), (), (), -1, inputs.random_dense_gate(rng, 2)))
        a, b, c = (int(v) for v in rng.choice(n, 3, replace=False))
        gates.append(inputs.Gate("matrix", (a, b, c), (), (), -1, inputs.random_dense_gate(rng, 3)))
        a, b, c = (int(v) for v in rng.choice(n, 3, replace=False))
        gates.append(inputs.Gate("x", (a,), (b, c)))
        gates.append(inputs.Gate("ry", (b,), (a,), (rng.uniform(0, 6),)))
        gates.append(inputs.Gate("phase", (c,), (a,), (rng.uniform(0, 6),)))
        gates.append(inputs.Gate("rz", (int(rng.integers(n)),), (), (rng.uniform(0, 6),)))
        gates.append(inputs.Gate("cz", tuple(int(v) for v in rng.choice(n, 2, replace=False))))
        gates.append(inputs.Gate("swap", tuple(int(v) for v in rng.choice(n, 2, replace=False))))
        gates.append(inputs.Gate("h", (int(rng.integers(5)),)))
        gates.append(inputs.Gate("y", (int(rng.integers(n)),)))
        d = np.diag(np.exp(1j * rng.uniform(0, 6, 8)))
        gates.append(inputs.Gate("matrix", tuple(int(v) for v in rng.choice(n, 3, replace=False)), (), (), -1, d))
    return inputs.Circuit(n, gates, "mixed")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("kmax", [1, 3, 4])
@pytest.mark.parametrize("maker", ["random", "variational", "qft", "mixed"])
def test_staged_matches_oracle(q, orc, dtype, kmax, maker):
    n = {"random": 15, "variational": 14, "qft": 13, "mixed": 14}[maker]
    circ = {"random": lambda: inputs.random_circuit(n, 8, seed=5),
            "variational": lambda: inputs.variational(n, 5, seed=6),
            "qft": lambda: inputs.qft(n),
            "mixed": lambda: mixed_circuit(n, seed=7)}[maker]()
    psi0 = inputs.gaussian_state(n, seed=8)
    want = orc.simulate(circ, psi0)
    got = run_plan(q, circ, dtype, psi0, q.FUSE_STAGED, kmax)
    err = np.max(np.abs(got - want))
    assert err <= TOL[dtype], f"staged {maker} {dtype} kmax={kmax}: {err:.3e}"


def lane_pair_circuit(n, seed, depth=4):
    """Dense 2-qubit gates with targets on lane qubits (0..4): lane + lane,
    lane + tile qubit in both orders, uncontrolled and with controls on lane,
    tile and high qubits; 1-qubit gates around CZs on lane qubits, which the
    planner fuses into 4x4 blocks."""
    rng = np.random.default_rng(seed)
    gates = []
    dense = lambda: inputs.random_dense_gate(rng, 2)
    for _ in range(depth):
        for q_ in range(n):
            gates.append(inputs.Gate("su2", (q_,), (), inputs.haar_su2_quaternion(rng)))
        la, lb = (int(v) for v in rng.choice(5, 2, replace=False))
        hi = int(rng.integers(5, n))
        gates.append(inputs.Gate("cz", (la, hi)))
        gates.append(inputs.Gate("cz", (int(rng.integers(5, n)), lb)))
        for q_ in (la, lb, hi):
            gates.append(inputs.Gate("su2", (q_,), (), inputs.haar_su2_quaternion(rng)))
        gates.append(inputs.Gate("matrix", (la, lb), (), (), -1, dense()))
        gates.append(inputs.Gate("matrix", (la, hi), (), (), -1, dense()))
        gates.append(inputs.Gate("matrix", (hi, lb), (), (), -1, dense()))
        others = [int(v) for v in rng.permutation(n) if v not in (la, lb, hi)]
        gates.append(inputs.Gate("matrix", (la, lb), (others[0],), (), -1, dense()))
        gates.append(inputs.Gate("matrix", (hi, la), (others[1], others[2]), (), -1, dense()))
        gates.append(inputs.Gate("swap", (lb, la)))
        gates.append(inputs.Gate("swap", (la, int(rng.integers(5, n)))))
    return inputs.Circuit(n, gates, "lane pairs")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("kmax", [1, 3, 4])
@pytest.mark.parametrize("n", [10, 14, 17])
def test_staged_two_qubit_gates_on_lanes(q, orc, dtype, kmax, n):
    """4x4 ops with one or two targets among the lane qubits (partner
    amplitudes by shuffle, coefficients laid out per lane-bit value), with
    controls on lanes, registers and tile qubits, against the oracle."""
    circ = lane_pair_circuit(n, seed=n + kmax)
    psi0 = inputs.gaussian_state(n, seed=3)
    want = orc.simulate(circ, psi0)
    got = run_plan(q, circ, dtype, psi0, q.FUSE_STAGED, kmax)
    err = np.max(np.abs(got - want))
    assert err <= TOL[dtype], f"lane pairs n={n} {dtype} kmax={kmax}: {err:.3e}"


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("kmax", [1, 3, 4])
@pytest.mark.parametrize("maker", ["random", "variational", "qft", "mixed", "lanes"])
def test_specialized_stages_match_oracle(q, orc, dtype, kmax, maker):
    """Stage kernels compiled for the plan (QSIM_PLAN_SPECIALIZE): every op
    kind, lane and register targets, controls, exchanges, both precisions."""
    n = {"random": 15, "variational": 14, "qft": 13, "mixed": 14, "lanes": 14}[maker]
    circ = {"random": lambda: inputs.random_circuit(n, 8, seed=5),
            "variational": lambda: inputs.variational(n, 5, seed=6),
            "qft": lambda: inputs.qft(n),
            "mixed": lambda: mixed_circuit(n, seed=7),
            "lanes": lambda: lane_pair_circuit(n, seed=8)}[maker]()
    psi0 = inputs.gaussian_state(n, seed=8)
    want = orc.simulate(circ, psi0)
    got = run_plan(q, circ, dtype, psi0, q.FUSE_STAGED | q.SPECIALIZE, kmax)
    err = np.max(np.abs(got - want))
    assert err <= TOL[dtype], f"specialized {maker} {dtype} kmax={kmax}: {err:.3e}"


def test_specialized_plan_many_tiles_and_cache(q, orc):
    """21 qubits (hundreds of tiles, warp and tile qubits high); a second
    circuit of the same structure with other angles reuses the compiled
    kernels (cache hit, no compile) and still matches the oracle."""
    n = 21
    a = inputs.random_circuit(n, 5, seed=9)
    rng = np.random.default_rng(3)
    b = inputs.Circuit(n, [inputs.Gate(g.name, g.targets, g.controls, inputs.haar_su2_quaternion(rng))
                           if g.name == "su2" else g for g in a.gates])
    psi0 = inputs.gaussian_state(n, seed=12)
    pa = q.Plan(a, kmax=3, mode=q.FUSE_STAGED | q.SPECIALIZE)
    assert pa.info()["mode"] == q.FUSE_STAGED | q.SPECIALIZE
    s = q.State(n, "c64")
    s.from_host(psi0)
    s.run_fused(pa)
    assert np.max(np.abs(s.to_host() - orc.simulate(a, psi0))) <= TOL["c64"]
    st0 = q.spec_stats()
    s.from_host(psi0)
    s.run_fused(q.Plan(b, kmax=3, mode=q.FUSE_STAGED | q.SPECIALIZE))
    st1 = q.spec_stats()
    assert st1["compiles"] == st0["compiles"] and st1["cache_hits"] > st0["cache_hits"]
    assert np.max(np.abs(s.to_host() - orc.simulate(b, psi0))) <= TOL["c64"]


@pytest.mark.parametrize("specialize", [False, True])
def test_staged_stages_split_over_the_parameter_limit(q, orc, specialize):
    """120 dense 2-qubit gates inside one tile's qubits: more coefficients than
    one kernel parameter block holds, so the planner splits the stage; both
    executors against the oracle."""
    rng = np.random.default_rng(1)
    n = 12
    gates = []
    for _ in range(120):
        a, b = (int(v) for v in rng.choice(range(5, 12), 2, replace=False))
        gates.append(inputs.Gate("matrix", (a, b), (), (), -1, inputs.random_dense_gate(rng, 2)))
    circ = inputs.Circuit(n, gates)
    psi0 = inputs.gaussian_state(n, seed=2)
    want = orc.simulate(circ, psi0)
    mode = q.FUSE_STAGED | (q.SPECIALIZE if specialize else 0)
    got = run_plan(q, circ, "c64", psi0, mode, 3)
    assert np.max(np.abs(got - want)) <= TOL["c64"]


def test_specialized_rejects_other_modes(q):
    with pytest.raises(q.QsimError):
        q.Plan(inputs.random_circuit(14, 2, seed=1), kmax=6, mode=q.FUSE_TC | q.SPECIALIZE)


@pytest.mark.parametrize("n", [5, 9, 10, 12])
def test_staged_small_widths(q, orc, n):
    """n < 9 falls back to the greedy plan; n = 9..12 uses tiles with fewer warps."""
    circ = mixed_circuit(n, seed=n, depth=4) if n >= 5 else inputs.qft(n)
    psi0 = inputs.gaussian_state(n, seed=1)
    want = orc.simulate(circ, psi0)
    got = run_plan(q, circ, "c128", psi0, q.FUSE_STAGED, 4)
    assert np.max(np.abs(got - want)) <= 1e-12


@pytest.mark.parametrize("kmax", [3, 4])
@pytest.mark.parametrize("maker", ["random", "mixed"])
def test_staged_many_tiles(q, orc, kmax, maker):
    """21 qubits: hundreds of tiles, phases with warp and tile qubits high."""
    n = 21
    circ = inputs.random_circuit(n, 5, seed=9) if maker == "random" else mixed_circuit(n, seed=10, depth=4)
    psi0 = inputs.gaussian_state(n, seed=12)
    want = orc.simulate(circ, psi0)
    got = run_plan(q, circ, "c64", psi0, q.FUSE_STAGED, kmax)
    err = np.max(np.abs(got - want))
    assert err <= TOL["c64"], f"staged {maker} n=21 kmax={kmax}: {err:.3e}"


def test_staged_covers_fewer_sweeps(q):
    c = inputs.random_circuit(30, 20, seed=2022)
    info = q.Plan(c, kmax=4, mode=q.FUSE_STAGED).info()
    assert info["gates"] == 900 and info["sweeps"] < 60


@pytest.mark.parametrize("kmax", [5, 6])
@pytest.mark.parametrize("maker", ["random", "variational", "local2q"])
def test_tensor_core_blocks_match_oracle(q, orc, kmax, maker):
    """Fused k-qubit blocks as split-precision real GEMMs on tcgen05
    (kmax 6: BF16x3, kmax 5: 3xTF32), bit-rotating passes, complex64."""
    n = {"random": 14, "variational": 15, "local2q": 13}[maker]
    rng = np.random.default_rng(11)
    if maker == "random":
        circ = inputs.random_circuit(n, 5, seed=21)
    elif maker == "variational":
        circ = inputs.variational(n, 3, seed=22)
    else:  # dense 2-qubit gates on neighbours plus controlled gates inside a window
        gates = []
        for layer in range(4):
            for a in range(layer % 2, n - 1, 2):
                gates.append(inputs.Gate("matrix", (a + 1, a), (), (), -1, inputs.random_dense_gate(rng, 2)))
            gates.append(inputs.Gate("x", (3,), (1,)))
            gates.append(inputs.Gate("cz", (0, n - 1)))
        circ = inputs.Circuit(n, gates)
    psi0 = inputs.gaussian_state(n, seed=23)
    want = orc.simulate(circ, psi0)
    got = run_plan(q, circ, "c64", psi0, q.FUSE_TC, kmax)
    err = np.max(np.abs(got - want))
    rel = err / np.max(np.abs(want))
    print(f"tc {maker} kmax={kmax}: max-abs {err:.3e} relative {rel:.3e}")
    assert err <= 1e-5, f"tc {maker} kmax={kmax}: max-abs {err:.3e} (relative {rel:.3e})"
    # the split keeps ~16 (BF16x3) or ~21 (3xTF32) bits per operand; measured
    # relative errors <= 1.5e-5 (BF16x3) and 5.4e-6 (3xTF32), bounds about 3x that
    assert rel <= (5e-5 if kmax == 6 else 1.5e-5), f"relative error {rel:.3e}"


def test_tensor_core_rejects_complex128(q):
    circ = inputs.random_circuit(13, 2, seed=1)
    s = q.State(13, "c128").init_zero()
    with pytest.raises(q.QsimError):
        s.run_fused(q.Plan(circ, kmax=6, mode=q.FUSE_TC))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_plan_autotuner_picks_a_correct_plan(q, orc, dtype):
    circ = inputs.random_circuit(14, 6, seed=31)
    scratch = q.State(14, dtype)
    plan = q.Plan.autotune(circ, scratch, reps=1)
    assert plan.mode in (q.FUSE_GREEDY2, q.FUSE_STAGED, q.FUSE_TC) and plan.tuned_ms > 0
    psi0 = inputs.gaussian_state(14, seed=32)
    s = q.State(14, dtype).from_host(psi0)
    s.run_fused(plan)
    err = np.max(np.abs(s.to_host().astype(np.complex128) - orc.simulate(circ, psi0)))
    assert err <= TOL[dtype]


def test_autotuner_error_table_and_bound(q, orc):
    """qsim_plan_autotune_ex: every candidate's error against the gate-by-gate
    complex128 run (FP64 truth), checked against the oracle's own result; a
    bound between the BF16x3 and FP32 tensor-core plans' errors adds a mixed
    plan with part of its passes in FP32; the kept plan is within the bound
    and matches the oracle."""
    circ = inputs.random_circuit(18, 6, seed=13)
    want = orc.simulate(circ)
    s = q.State(18, "c64")
    loose = q.Plan.autotune(circ, s, reps=1, max_err=1.0)
    tab = loose.table
    assert [(e["mode"], e["kmax"], e["nfp32"] == e["npasses"] > 0) for e in tab] == [
        ("staged", 3, False), ("staged", 4, False), ("tc", 6, False), ("tc", 5, False), ("tc", 6, True)]
    assert all(e["ref"] == "fp64" and e["ms"] > 0 and 0 < e["err"] < 1e-3 for e in tab)
    fastest = min(tab, key=lambda e: e["ms"])
    assert loose.kmax == fastest["kmax"]
    # the table's errors are those of the plans against the oracle
    for e in tab:
        p = q.Plan(circ, kmax=e["kmax"], mode={"staged": q.FUSE_STAGED, "tc": q.FUSE_TC}[e["mode"]])
        if e["mode"] == "tc" and e["nfp32"]:
            p.set_tc_precisions([q.PREC_FP32] * p.info()["sweeps"])
        s2 = q.State(18, "c64").init_zero()
        s2.run_fused(p)
        err2 = np.linalg.norm(s2.to_host().astype(np.complex128) - want)
        assert abs(err2 - e["err"]) <= 1e-3 * e["err"] + 1e-9, (e, err2)
    e_bf, e_fp = tab[2]["err"], tab[4]["err"]
    print(f"autotune 18q: staged {tab[0]['err']:.2e}, bf16x3 {e_bf:.2e}, 3xtf32 {tab[3]['err']:.2e}, fp32 {e_fp:.2e}")
    assert e_fp < 0.5 * e_bf
    bound = (e_bf * e_fp) ** 0.5
    mixed = q.Plan.autotune(circ, s, reps=1, max_err=bound)
    mx = [e for e in mixed.table if e["mode"] == "tc" and 0 < e["nfp32"] < e["npasses"]]
    assert len(mx) == 1 and mx[0]["kmax"] == 6
    chosen = [e for e in mixed.table if e["ms"] >= 0 and e["err"] <= bound]
    assert chosen and mixed.tuned_ms == min(e["ms"] for e in chosen)
    s2 = q.State(18, "c64").init_zero()
    s2.run_fused(mixed)
    assert np.linalg.norm(s2.to_host().astype(np.complex128) - want) <= bound * 1.001


def test_tensor_core_plan_per_pass_precision(q, orc):
    """Each pass of a tensor-core plan in its own arithmetic: all FP32 (CUDA
    cores) is as accurate as the FP32 stages; a mix of BF16x3, 3xTF32 and FP32
    passes matches the oracle; 3xTF32 on a 6-qubit window is refused."""
    n = 16
    circ = inputs.random_circuit(n, 6, seed=41)
    psi0 = inputs.gaussian_state(n, seed=42)
    want = orc.simulate(circ, psi0)
    p = q.Plan(circ, kmax=6, mode=q.FUSE_TC)
    m = p.info()["sweeps"]
    assert p.tc_precisions() == [q.PREC_BF16X3] * m
    ks = [0 if ps["plain"] else len(ps["targets"]) for ps in p.tc_passes()]  # window width per pass
    p.set_tc_precisions([q.PREC_FP32] * m)
    s = q.State(n, "c64").from_host(psi0.astype(np.complex64))
    s.run_fused(p)
    err = np.max(np.abs(s.to_host() - want)) / np.max(np.abs(want))
    print(f"tc fp32 passes 16q: relative max-abs {err:.2e}")
    assert err <= 2e-6
    mix = [(q.PREC_TF32X3 if k == 5 else q.PREC_BF16X3) if i % 2 else q.PREC_FP32 for i, k in enumerate(ks)]
    p.set_tc_precisions(mix)
    assert p.tc_precisions() == mix
    s = q.State(n, "c64").from_host(psi0.astype(np.complex64))
    s.run_fused(p)
    err = np.max(np.abs(s.to_host() - want)) / np.max(np.abs(want))
    assert err <= 5e-5
    if 6 in ks:
        bad = [q.PREC_TF32X3 if k == 6 else q.PREC_BF16X3 for k in ks]
        with pytest.raises(q.QsimError):
            p.set_tc_precisions(bad)
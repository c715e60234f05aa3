"""Sliced states on the host: the planner's SWAP steps and per-slice segment
circuits, executed slice by slice with the oracle (tests/slice_cpu.py), must
reproduce the oracle's unsliced simulation of the same circuit."""
import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

from slice_cpu import global_heavy_circuit, run_sequential


@pytest.fixture(scope="module")
def q():
    from paper_2203_08826_gb300 import build, binding
    build.build()
    return binding


CIRCUITS = {
    "random": lambda n: inputs.random_circuit(n, 4, seed=n),
    "qft": lambda n: inputs.qft(n),
    "variational": lambda n: inputs.variational(n, 3, seed=2),
    "global": lambda n: global_heavy_circuit(n, seed=n),
}


@pytest.mark.parametrize("maker", sorted(CIRCUITS))
@pytest.mark.parametrize("n,g", [(9, 1), (10, 3), (11, 4)])
def test_sliced_plan_matches_oracle(q, orc, maker, n, g):
    circ = CIRCUITS[maker](n)
    psi0 = inputs.gaussian_state(n, seed=5)
    want = orc.simulate(circ, psi0)
    plan = q.SlicePlan(circ, g, kmax=2, mode=q.FUSE_GREEDY2, restore=True)
    assert plan.layout() == list(range(n))
    got = run_sequential(plan, psi0, orc)
    assert np.max(np.abs(got - want)) < 1e-12


def test_layout_without_restore_is_a_permutation(q, orc):
    n, g = 10, 3
    circ = global_heavy_circuit(n, seed=1)
    psi0 = inputs.gaussian_state(n, seed=2)
    plan = q.SlicePlan(circ, g, kmax=2, mode=q.FUSE_GREEDY2, restore=False)
    pos = plan.layout()
    assert sorted(pos) == list(range(n)) and pos != list(range(n))
    got = run_sequential(plan, psi0, orc)
    want = orc.simulate(circ, psi0)
    # physical index: bit pos[q] holds logical qubit q
    x = np.arange(1 << n)
    phys = np.zeros_like(x)
    for lq, p in enumerate(pos):
        phys |= ((x >> lq) & 1) << p
    assert np.max(np.abs(got[phys] - want)) < 1e-12


def test_swaps_only_where_needed(q):
    n = 12
    # gates on local qubits only, global controls and diagonals: no exchange
    gates = [inputs.Gate("h", (i,)) for i in range(9)]
    gates += [inputs.Gate("x", (0,), (11,)), inputs.Gate("cz", (10, 11)), inputs.Gate("rz", (9,), (), (0.3,))]
    plan = q.SlicePlan(inputs.Circuit(n, gates, "local"), 3, kmax=2, mode=q.FUSE_GREEDY2)
    info = plan.info()
    assert info["swaps"] == 0 and info["steps"] == 1
    seg = plan.steps()[0]
    assert seg["type"] == "segment" and seg["keymask"] == 0b111 and seg["gates"] == len(gates)
    # one dense gate on a global qubit: one exchange there, one back
    plan = q.SlicePlan(inputs.Circuit(n, gates + [inputs.Gate("h", (10,))], "g"), 3, kmax=2, mode=q.FUSE_GREEDY2)
    assert plan.info()["swaps"] == 2
    sw = [s for s in plan.steps() if s["type"] == "swap"]
    assert sw[0]["global_bit"] == 1 and sw[1]["global_bit"] == 1


def test_segment_variants_per_global_pattern(q):
    n, g = 10, 2
    gates = [inputs.Gate("x", (0,), (8, 9))]  # applies only in slice 3
    plan = q.SlicePlan(inputs.Circuit(n, gates, "c"), g, kmax=2, mode=q.FUSE_GREEDY2)
    assert [len(plan.segment_gates(0, s)) for s in range(4)] == [0, 0, 0, 1]
    assert plan.info()["variants"] == 4


def test_slice_plan_validation(q):
    c = inputs.random_circuit(8, 1, seed=1)
    for bad in (-1, 8, 17):
        with pytest.raises(q.QsimError):
            q.SlicePlan(c, bad)
    with pytest.raises(q.QsimError):
        q.SlicePlan(c, 2, mode=7)
    # wider than a state may be, but the slices fit: accepted
    wide = inputs.Circuit(40, [inputs.Gate("h", (39,)), inputs.Gate("cz", (0, 39))], "wide")
    plan = q.SlicePlan(wide, 8, kmax=2, mode=q.FUSE_GREEDY2)
    assert plan.info()["n_local"] == 32
    with pytest.raises(q.QsimError):
        q.SlicePlan(wide, 4)  # 36-qubit slices

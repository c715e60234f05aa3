"""The seeded workload generators follow the input recipe they state: the
shapes of the benchmark families (QFT, supremacy-style random circuits,
layered variational ansatz, batches), the Hamiltonians, and seeding.  Both the
library and the oracle consume these gate lists, so a generator that drifted
from its recipe would change the workloads without any parity test noticing."""
import math

import numpy as np

from paper_2203_08826_gb300 import inputs


def test_random_circuit_layers():
    """Depth 20 at 30 qubits: per layer an SU(2) on every qubit in order, then
    CZ on a perfect matching; 900 gates; the matchings vary between layers."""
    n, depth = 30, 20
    c = inputs.random_circuit(n, depth, seed=2022)
    assert c.n == n and len(c) == depth * (n + n // 2) == 900
    per = n + n // 2
    matchings = set()
    for l in range(depth):
        layer = c.gates[l * per:(l + 1) * per]
        assert [g.name for g in layer[:n]] == ["su2"] * n
        assert [g.targets for g in layer[:n]] == [(q,) for q in range(n)]
        for g in layer[:n]:
            assert abs(math.fsum(v * v for v in g.params) - 1.0) < 1e-12  # unit quaternion
        czs = layer[n:]
        assert all(g.name == "cz" and not g.controls and g.targets[0] < g.targets[1] for g in czs)
        covered = sorted(q for g in czs for q in g.targets)
        assert covered == list(range(n))  # every qubit exactly once
        matchings.add(tuple(g.targets for g in czs))
    assert len(matchings) == depth


def test_variational_ansatz_structure():
    """RY then RZ on every qubit (trainable, indices in gate order, angles in
    [0, 2 pi)), then the CZ ladder (i, i + 1)."""
    n, layers = 7, 3
    c = inputs.variational(n, layers, seed=4)
    per = 2 * n + n - 1
    assert len(c) == layers * per and c.nparams == 2 * n * layers
    p = 0
    for l in range(layers):
        layer = c.gates[l * per:(l + 1) * per]
        for q in range(n):
            ry, rz = layer[2 * q], layer[2 * q + 1]
            assert (ry.name, rz.name) == ("ry", "rz") and ry.targets == rz.targets == (q,)
            assert (ry.pindex, rz.pindex) == (p, p + 1)
            p += 2
            assert all(0.0 <= g.params[0] < 2 * math.pi for g in (ry, rz))
        assert [(g.name, g.targets) for g in layer[2 * n:]] == [("cz", (i, i + 1)) for i in range(n - 1)]
    np.testing.assert_array_equal(c.with_params(c.params()).params(), c.params())


def test_batch_ranges_are_inclusive():
    """n ~ U{12..20} and layers ~ U{4..12}, both ends reached; each circuit a
    variational ansatz of its width and depth; `limit` builds a prefix."""
    cs = inputs.batch_circuits(4096, seed=2024)
    ns = np.array([c.n for c in cs])
    ls = np.array([len(c) // (3 * c.n - 1) for c in cs])
    assert ns.min() == 12 and ns.max() == 20 and ls.min() == 4 and ls.max() == 12
    assert all(len(c) == l * (3 * c.n - 1) for c, l in zip(cs, ls))
    assert set(np.unique(ns)) == set(range(12, 21))
    head = inputs.batch_circuits(4096, seed=2024, limit=3)
    assert [(h.n, h.gates) for h in head] == [(c.n, c.gates) for c in cs[:3]]


def test_qft_structure():
    """H(j) then controlled phases 2 pi / 2^(j - m + 1) with control m < j, from
    the top qubit down, then the swaps."""
    n = 6
    c = inputs.qft(n)
    assert len(c) == n + n * (n - 1) // 2 + n // 2
    it = iter(c.gates)
    for j in range(n - 1, -1, -1):
        g = next(it)
        assert (g.name, g.targets) == ("h", (j,))
        for m in range(j - 1, -1, -1):
            g = next(it)
            assert (g.name, g.targets, g.controls) == ("phase", (j,), (m,))
            assert g.params[0] == 2 * math.pi / 2 ** (j - m + 1)
    assert [(g.name, g.targets) for g in it] == [("swap", (i, n - 1 - i)) for i in range(n // 2)]


def test_states_and_seeds():
    a = inputs.gaussian_state(10, seed=1)
    assert abs(np.linalg.norm(a) - 1.0) < 1e-12 and a.dtype == np.complex128
    np.testing.assert_array_equal(a, inputs.gaussian_state(10, seed=1))
    assert not np.array_equal(a, inputs.gaussian_state(10, seed=2))
    assert inputs.random_circuit(8, 3, seed=5).gates == inputs.random_circuit(8, 3, seed=5).gates
    assert inputs.random_circuit(8, 3, seed=5).gates != inputs.random_circuit(8, 3, seed=6).gates
    u = inputs.random_dense_gate(np.random.default_rng(0), 3)
    np.testing.assert_allclose(u.conj().T @ u, np.eye(8), atol=1e-12)


def test_hamiltonians():
    n = 5
    zz = inputs.zz_chain(n)
    assert list(zz.zmask) == [3 << i for i in range(n - 1)] and not zz.xmask.any() and (zz.coeff == 1).all()
    t = inputs.tfim(n, 0.5)
    assert len(t) == 2 * n - 1
    assert list(t.xmask[n - 1:]) == [1 << i for i in range(n)] and (t.coeff[n - 1:] == 0.5).all()
    tt = inputs.tfim_target(n, 1.0)
    np.testing.assert_array_equal(tt.coeff, -inputs.tfim(n, 1.0).coeff)
    xf = inputs.x_field(n)
    assert list(xf.xmask) == [1 << i for i in range(n)] and (xf.coeff == -1).all() and not xf.zmask.any()
    r = inputs.random_pauli_sum(6, 50, seed=3)
    assert len(r) == 50 and int(max(r.xmask | r.zmask)) < (1 << 6)


def test_adiabatic_circuit_structure():
    """H on every qubit, then per step at s_k = (k + 1/2) dt / T: RX(A dt),
    RZZ(2 B dt) on the chain, RX(A dt), with A = -((1 - s) + s h), B = -s."""
    n, h, T, dt = 4, 1.0, 1.0, 0.25
    c = inputs.adiabatic_tfim(n, h, T, dt)
    sched = inputs.adiabatic_schedule(T, dt)
    assert sched == [0.125, 0.375, 0.625, 0.875]
    per = n + (n - 1) + n
    assert len(c) == n + len(sched) * per
    assert [(g.name, g.targets) for g in c.gates[:n]] == [("h", (q,)) for q in range(n)]
    for k, s in enumerate(sched):
        step = c.gates[n + k * per:n + (k + 1) * per]
        A, B = -((1 - s) + s * h), -s
        assert all(g.name == "rx" and abs(g.params[0] - A * dt) < 1e-15 for g in step[:n] + step[-n:])
        assert [(g.name, g.targets) for g in step[n:n + n - 1]] == [("rzz", (i, i + 1)) for i in range(n - 1)]
        assert all(abs(g.params[0] - 2 * B * dt) < 1e-15 for g in step[n:n + n - 1])

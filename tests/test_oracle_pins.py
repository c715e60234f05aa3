"""Pins of the CPU oracle against facts independent of its own code.

Each test targets a mistake the oracle could plausibly make (a transposed
operand, a wrong bit order, a dropped control, a sign error in a rotation, a
wrong sampler boundary) and checks a result fixed by mathematics or by the
paper: Kronecker-product operators, closed forms (DFT, GHZ), invariants,
published known-answer vectors, gate counts printed in the paper.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers
def kron_operator(n, G, targets, controls=()):
    """Full 2^n x 2^n operator by Kronecker products and an index permutation.

    The gate (with its controls in front, controls act as |0><0| (x) I +
    |1><1| (x) G) is first built on the contiguous top qubits in the order
    (controls..., targets...) with np.kron, then moved to the requested qubits
    by permuting index bits.  Nothing of the oracle's index arithmetic is used.
    """
    k, c = len(targets), len(controls)
    d = 1 << (k + c)
    # operator on c + k qubits, first listed qubit = most significant
    P1 = np.array([[0, 0], [0, 1]], dtype=complex)
    P0 = np.array([[1, 0], [0, 0]], dtype=complex)
    op = G.astype(complex)
    for _ in range(c):
        op = np.kron(P0, np.eye(op.shape[0])) + np.kron(P1, op)
    assert op.shape == (d, d)
    full = np.kron(op, np.eye(1 << (n - k - c)))   # listed qubits on top bits
    # listed qubit i (0 = most significant of op) sits on bit n-1-i of `full`;
    # build the permutation that moves bit n-1-i to qubit order[i]
    order = list(controls) + list(targets)
    rest = [q for q in range(n) if q not in order]
    src_bit_of = {}
    for i, q in enumerate(order):
        src_bit_of[q] = n - 1 - i
    for j, q in enumerate(sorted(rest, reverse=True)):
        src_bit_of[q] = n - 1 - len(order) - j
    perm = np.zeros(1 << n, dtype=np.int64)   # perm[x] = index in `full` basis
    for x in range(1 << n):
        y = 0
        for q in range(n):
            if (x >> q) & 1:
                y |= 1 << src_bit_of[q]
        perm[x] = y
    return full[np.ix_(perm, perm)]


def random_state(rng, n):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


class Spec:
    def __init__(self, name, targets, controls=(), params=(), matrix=None):
        self.name, self.targets, self.controls = name, tuple(targets), tuple(controls)
        self.params, self.matrix = tuple(params), matrix


# ------------------------------------------------------------------ Eq. (1)
@pytest.mark.parametrize("n,k,c", [(3, 1, 0), (4, 2, 0), (5, 2, 1), (6, 3, 1), (7, 1, 2),
                                   (8, 4, 0), (8, 2, 3)])
def test_apply_matches_kronecker_operator(orc, n, k, c):
    rng = np.random.default_rng(100 + 10 * n + k + c)
    for trial in range(4):
        qs = rng.permutation(n)[: k + c]
        targets, controls = [int(q) for q in qs[:k]], [int(q) for q in qs[k:]]
        G = inputs.random_dense_gate(rng, k)
        G = G + 0.3 * (rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape))
        psi = random_state(rng, n)
        U = kron_operator(n, G, targets, controls)
        got = orc.apply_matrix(psi.copy(), G, targets, controls)
        np.testing.assert_allclose(got, U @ psi, atol=1e-13, rtol=0)


def test_qft10_matches_1024_dim_kronecker_product(orc):
    """The 10-qubit QFT circuit, as one 1024x1024 matrix product of
    Kronecker-built gate operators, against the gate-by-gate oracle."""
    n = 10
    circ = inputs.qft(n)
    psi0 = inputs.gaussian_state(n, seed=1)
    U = np.eye(1 << n, dtype=complex)
    for g in circ.gates:
        U = kron_operator(n, orc.gate_matrix(g), g.targets, g.controls) @ U
    got = orc.simulate(circ, psi0)
    np.testing.assert_allclose(got, U @ psi0, atol=1e-12, rtol=0)


def test_brute_force_every_ordering_tiny(orc):
    """n = 4: every ordered choice of 2 targets and 0..2 controls."""
    n = 4
    rng = np.random.default_rng(7)
    G = inputs.random_dense_gate(rng, 2)
    psi = random_state(rng, n)
    for targets in itertools.permutations(range(n), 2):
        others = [q for q in range(n) if q not in targets]
        for c in range(3):
            for controls in itertools.permutations(others, c):
                got = orc.apply_matrix(psi.copy(), G, targets, controls)
                want = kron_operator(n, G, targets, controls) @ psi
                np.testing.assert_allclose(got, want, atol=1e-13, rtol=0)


def test_cnot_target_order_is_not_symmetric(orc):
    """CNOT as a 2-qubit matrix: targets=(control, target) with targets[0] the
    most significant matrix bit.  |q1 q0> = |1 0>  ->  |1 1>."""
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    psi = np.zeros(4, dtype=complex); psi[0b10] = 1
    out = orc.apply_matrix(psi.copy(), cnot, (1, 0))
    assert abs(out[0b11] - 1) < 1e-15
    out2 = orc.apply_matrix(psi.copy(), cnot, (0, 1))   # control = qubit 0 = 0
    assert abs(out2[0b10] - 1) < 1e-15


def test_rejects_bad_qubits(orc):
    psi = np.zeros(8, dtype=complex); psi[0] = 1
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    with pytest.raises(ValueError):
        orc.apply_matrix(psi, X, (3,))
    with pytest.raises(ValueError):
        orc.apply_matrix(psi, X, (1,), (1,))
    with pytest.raises(ValueError):
        orc.apply_matrix(psi, np.eye(4, dtype=complex), (2, 2))


# ------------------------------------------------------------------ gate definitions
def test_textbook_identities(orc):
    M = orc.gate_matrix
    X, H, Z = M(Spec("x", (0,))), M(Spec("h", (0,))), M(Spec("z", (0,)))
    Y = M(Spec("y", (0,)))
    I2 = np.eye(2)
    np.testing.assert_allclose(X @ X, I2, atol=1e-15)
    np.testing.assert_allclose(H @ H, I2, atol=1e-15)
    np.testing.assert_allclose(H @ Z @ H, X, atol=1e-15)
    np.testing.assert_allclose(X @ Y, 1j * Z, atol=1e-15)          # XY = iZ
    psi = np.zeros(2, complex); psi[0] = 1
    np.testing.assert_allclose(orc.apply_matrix(psi, H, (0,)), [2**-0.5] * 2, atol=1e-15)
    np.testing.assert_allclose(np.diag(M(Spec("cz", (0, 1)))), [1, 1, 1, -1])
    for phi in (0.3, 2.1):
        A = M(Spec("rz", (0,), params=(phi,))) @ M(Spec("rz", (0,), params=(-phi,)))
        np.testing.assert_allclose(A, I2, atol=1e-15)
    # rotations are exp(-i theta P / 2): compare with the matrix exponential
    from scipy.linalg import expm
    for name in ("rx", "ry", "rz"):
        th = 0.77
        np.testing.assert_allclose(M(Spec(name, (0,), params=(th,))),
                                   expm(-0.5j * th * orc.pauli_generator(name)), atol=1e-14)
    # S = T^2, Z = S^2
    S, T = M(Spec("s", (0,))), M(Spec("t", (0,)))
    np.testing.assert_allclose(T @ T, S, atol=1e-15)
    np.testing.assert_allclose(S @ S, Z, atol=1e-15)
    # SWAP exchanges |01> and |10>
    sw = M(Spec("swap", (0, 1)))
    np.testing.assert_allclose(sw @ np.array([0, 1, 0, 0]), [0, 0, 1, 0])


def test_su2_quaternion_is_special_unitary(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = inputs.haar_su2_quaternion(rng)
        U = orc.gate_matrix(Spec("su2", (0,), params=q))
        np.testing.assert_allclose(U @ U.conj().T, np.eye(2), atol=1e-14)
        assert abs(np.linalg.det(U) - 1) < 1e-14


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("maker", [
    lambda: inputs.random_circuit(10, 6, seed=11),
    lambda: inputs.variational(9, 4, seed=12),
    lambda: inputs.qft(10),
])
def test_norm_preserved_and_inverse_recovers(orc, maker):
    circ = maker()
    psi0 = inputs.gaussian_state(circ.n, seed=5)
    psi = orc.simulate(circ, psi0)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    back = orc.run_inverse(psi.copy(), circ.gates)
    np.testing.assert_allclose(back, psi0, atol=1e-12, rtol=0)


def test_ghz_amplitudes(orc):
    for n in (2, 5, 11):
        psi = orc.simulate(inputs.ghz(n))
        want = np.zeros(1 << n); want[0] = want[-1] = 2**-0.5
        np.testing.assert_allclose(psi, want, atol=1e-14)


# ------------------------------------------------------------------ QFT closed form
@pytest.mark.parametrize("n", [1, 2, 3, 6, 10, 13])
def test_qft_is_unitary_dft(orc, n):
    """F[y, x] = exp(2 pi i x y / N) / sqrt(N): numpy's inverse FFT times sqrt(N)."""
    psi0 = inputs.gaussian_state(n, seed=n)
    got = orc.simulate(inputs.qft(n), psi0)
    np.testing.assert_allclose(got, math.sqrt(1 << n) * np.fft.ifft(psi0), atol=1e-12, rtol=0)


def test_qft_of_basis_state_has_uniform_magnitude_and_linear_phase(orc):
    n, x = 8, 37
    N = 1 << n
    psi0 = np.zeros(N, dtype=complex); psi0[x] = 1
    got = orc.simulate(inputs.qft(n), psi0)
    np.testing.assert_allclose(np.abs(got), N**-0.5, atol=1e-14)
    y = np.arange(N)
    np.testing.assert_allclose(got, np.exp(2j * np.pi * x * y / N) / math.sqrt(N), atol=1e-13)


def _asap_depth(circ):
    level = [0] * circ.n
    for g in circ.gates:
        qs = g.qubits
        l = 1 + max(level[q] for q in qs)
        for q in qs:
            level[q] = l
    return max(level)


def test_qft_size_matches_paper_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "benchmark_circuits_table.txt"))
            if l.strip() and not l.startswith("#")]
    name, n, depth, gates = rows[0][0], int(rows[0][1]), int(rows[0][2]), int(rows[0][3])
    assert name == "qft"
    circ = inputs.qft(n)
    assert len(circ) == gates == n + n * (n - 1) // 2 + n // 2
    assert _asap_depth(circ) == depth


# ------------------------------------------------------------------ probabilities
def test_marginal_probabilities_by_reshape(orc):
    n = 7
    psi = inputs.gaussian_state(n, seed=9)
    p = np.abs(psi) ** 2
    # axis a of the reshaped tensor is qubit n-1-a
    T = p.reshape([2] * n)
    for qubits in [(0,), (6,), (2, 5), (5, 2), (0, 3, 6), tuple(range(n - 1, -1, -1))]:
        axes = [n - 1 - q for q in qubits]
        keep = np.transpose(T, axes + [a for a in range(n) if a not in axes])
        want = keep.reshape(1 << len(qubits), -1).sum(axis=1)
        np.testing.assert_allclose(orc.probabilities(psi, qubits), want, atol=1e-15)
    np.testing.assert_allclose(orc.probabilities(psi), p, atol=1e-16)


# ------------------------------------------------------------------ Pauli expectation
def test_expectation_matches_dense_pauli_matrix(orc):
    n = 6
    psi = inputs.gaussian_state(n, seed=21)
    ham = inputs.random_pauli_sum(n, 12, seed=22)
    paulis = {(0, 0): np.eye(2), (1, 0): np.array([[0, 1], [1, 0]]),
              (1, 1): np.array([[0, -1j], [1j, 0]]), (0, 1): np.diag([1, -1])}
    Hm = np.zeros((1 << n, 1 << n), dtype=complex)
    for xm, zm, c in zip(ham.xmask, ham.zmask, ham.coeff):
        op = np.eye(1)
        for q in range(n - 1, -1, -1):   # most significant qubit first in kron
            op = np.kron(op, paulis[((int(xm) >> q) & 1, (int(zm) >> q) & 1)])
        Hm += c * op
    want = np.vdot(psi, Hm @ psi).real
    assert abs(orc.expectation(psi, ham) - want) < 1e-13
    np.testing.assert_allclose(orc.hamiltonian_apply(psi, ham), Hm @ psi, atol=1e-13)


def test_zz_expectation_closed_form(orc):
    """<Z_i Z_{i+1}> is diagonal: sum_x p(x) (n-1 - 2 popcount((x ^ x>>1) & mask))."""
    n = 9
    psi = inputs.gaussian_state(n, seed=4)
    x = np.arange(1 << n)
    d = (x ^ (x >> 1)) & ((1 << (n - 1)) - 1)
    pop = np.array([bin(int(v)).count("1") for v in d])
    want = float(np.sum(np.abs(psi) ** 2 * ((n - 1) - 2 * pop)))
    assert abs(orc.expectation(psi, inputs.zz_chain(n)) - want) < 1e-13


# ------------------------------------------------------------------ gradients
def test_single_rotation_gradient_closed_form(orc):
    """RY(t)|0>, H = Z: E = cos t, dE/dt = -sin t; RX likewise."""
    for name in ("ry", "rx"):
        circ = inputs.Circuit(1, [inputs.Gate(name, (0,), (), (0.9,), 0)])
        ham = inputs.PauliSum(np.array([0], np.uint64), np.array([1], np.uint64), np.array([1.0]))
        for t in (0.0, 0.9, 2.5, -1.2):
            assert abs(orc.energy(circ, ham, [t]) - math.cos(t)) < 1e-14
            g = orc.parameter_shift_gradient(circ, ham, [t])
            assert abs(g[0] + math.sin(t)) < 1e-14


def test_gradient_from_a_start_state_closed_form(orc):
    """From |1>: RY(t)|1> = (-sin t/2, cos t/2), so with H = Z, E = -cos t and
    dE/dt = sin t; from |+>: RZ(t)|+> with H = X gives E = cos t."""
    ham_z = inputs.PauliSum(np.array([0], np.uint64), np.array([1], np.uint64), np.array([1.0]))
    ham_x = inputs.PauliSum(np.array([1], np.uint64), np.array([0], np.uint64), np.array([1.0]))
    one = np.array([0, 1], dtype=complex)
    plus = np.array([1, 1], dtype=complex) / math.sqrt(2)
    for t in (0.0, 0.7, 2.1, -1.3):
        ry = inputs.Circuit(1, [inputs.Gate("ry", (0,), (), (t,), 0)])
        assert abs(orc.energy(ry, ham_z, [t], one) + math.cos(t)) < 1e-14
        assert abs(orc.parameter_shift_gradient(ry, ham_z, [t], psi0=one)[0] - math.sin(t)) < 1e-14
        rz = inputs.Circuit(1, [inputs.Gate("rz", (0,), (), (t,), 0)])
        assert abs(orc.energy(rz, ham_x, [t], plus) - math.cos(t)) < 1e-14
        assert abs(orc.parameter_shift_gradient(rz, ham_x, [t], psi0=plus)[0] + math.sin(t)) < 1e-14


def test_parameter_shift_agrees_with_finite_differences(orc):
    circ = inputs.variational(5, 2, seed=31)
    ham = inputs.tfim(5)
    th = circ.params()
    ps = orc.parameter_shift_gradient(circ, ham, th)
    fd = orc.finite_difference_gradient(circ, ham, th, h=1e-4)
    # central differences: O(h^2) truncation, |f'''| <= ||H|| ~ 7 here
    np.testing.assert_allclose(ps, fd, atol=5e-7)
    assert np.max(np.abs(ps)) > 1e-2
    psi0 = inputs.gaussian_state(5, seed=32)
    ps0 = orc.parameter_shift_gradient(circ, ham, th, psi0=psi0)
    fd0 = orc.finite_difference_gradient(circ, ham, th, h=1e-4, psi0=psi0)
    np.testing.assert_allclose(ps0, fd0, atol=5e-7)
    assert np.max(np.abs(ps0 - ps)) > 1e-2  # the start state matters


# ------------------------------------------------------------------ sampling
def test_philox_known_answers(orc):
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(v, 16) for v in line.split()]
        assert [int(v) for v in orc.philox4x32_10(w[:4], w[4:6])] == w[6:]


def test_sampler_chi_square(orc):
    from scipy.stats import chi2
    n = 8
    rng = np.random.default_rng(5)
    p = rng.dirichlet(np.full(1 << n, 0.7))
    shots = 400_000
    s = orc.sample(p, shots, seed=1234, counter0=0)
    counts = np.bincount(s.astype(np.int64), minlength=1 << n)
    exp = p * shots
    m = exp > 5
    stat = np.sum((counts[m] - exp[m]) ** 2 / exp[m])
    assert chi2.sf(stat, m.sum() - 1) > 1e-4


def test_sampler_support_and_determinism(orc):
    p = np.zeros(64); p[[3, 17, 40]] = [0.25, 0.5, 0.25]
    s = orc.sample(p, 5000, seed=9, counter0=77)
    assert set(np.unique(s).tolist()) <= {3, 17, 40}
    np.testing.assert_array_equal(s, orc.sample(p, 5000, seed=9, counter0=77))
    # counter offsets compose: shots [77, 5077) == shots [0, 5077) tail
    t = orc.sample(p, 5077, seed=9, counter0=0)
    np.testing.assert_array_equal(s, t[77:])
    one = np.zeros(16); one[11] = 1.0
    assert set(orc.sample(one, 100, seed=1).tolist()) == {11}


def test_sampler_boundary_rule_by_hand(orc):
    """Smallest x with CDF(x) > r: the draw r is recomputed with Python
    integers from the Philox outputs and the search is done by a linear scan."""
    p = np.array([0.125, 0.0, 0.375, 0.5])
    w = [int(math.floor(v * 2**62)) for v in p]
    cdf = list(itertools.accumulate(w))
    T = cdf[-1]
    seed = 0x1234_5678_9ABC_DEF0
    got = orc.sample(p, 64, seed=seed, counter0=2**32 - 5)   # crosses a 32-bit carry
    for s in range(64):
        cs = 2**32 - 5 + s
        o = orc.philox4x32_10([cs & 0xFFFFFFFF, cs >> 32, 0, 0],
                              [seed & 0xFFFFFFFF, seed >> 32])
        u = (int(o[1]) << 32) | int(o[0])
        r = (u * T) >> 64
        want = next(x for x in range(4) if cdf[x] > r)
        assert int(got[s]) == want


def test_sampler_matches_integer_inverse_cdf_at_scale(orc):
    """The same rule on 3001 outcomes (a quarter of them impossible, so runs
    of equal CDF values occur) and 3000 shots whose counters wrap past 2^64:
    weights floor(p 2^62) and the search are redone with Python integers
    (bisect over the CDF), the uniforms from the Philox outputs."""
    import bisect
    rng = np.random.default_rng(8)
    p = rng.dirichlet(np.full(3001, 0.5))
    p[rng.random(3001) < 0.25] = 0.0
    p /= p.sum() * (1 + 1e-12)
    w = [int(v * 2.0 ** 62) for v in p]  # exact scaling, then floor
    cdf = list(itertools.accumulate(w))
    T = cdf[-1]
    seed, c0 = 0xDEADBEEF_0BADF00D, 2**64 - 1000
    got = orc.sample(p, 3000, seed=seed, counter0=c0)
    for s in range(3000):
        cs = (c0 + s) % 2**64
        o = orc.philox4x32_10([cs & 0xFFFFFFFF, cs >> 32, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
        r = (((int(o[1]) << 32) | int(o[0])) * T) >> 64
        want = bisect.bisect_right(cdf, r)  # smallest x with cdf[x] > r
        assert int(got[s]) == want, s
        assert p[want] > 0


def tie_probabilities(orc, seed, counter0, frac=(0.0, 0.0)):
    """Two outcomes whose first draw r lands exactly on cdf[0]: with integer
    weights summing to T = 2^40, r = floor(u T / 2^64) = u >> 24 for the
    shot's 64-bit uniform u, so weights (u >> 24, 2^40 - (u >> 24)) -- exact
    as doubles w 2^-62 -- put r on the boundary.  The rule (smallest x with
    CDF(x) > r) must then give outcome 1.  `frac` adds fractions of 2^-62
    (still exact doubles) that the weights floor(p 2^62) must drop."""
    o = orc.philox4x32_10([counter0 & 0xFFFFFFFF, counter0 >> 32, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
    u = (int(o[1]) << 32) | int(o[0])
    w0 = u >> 24
    return np.array([(w0 + frac[0]) * 2.0 ** -62, ((1 << 40) - w0 + frac[1]) * 2.0 ** -62])


def test_sampler_draw_on_a_cdf_value_takes_the_next_outcome(orc):
    for seed, c0 in ((1, 0), (0xFEED, 2**32 - 1), (2**63 + 5, 2**64 - 1)):
        for frac in ((0.0, 0.0), (0.75, 0.25)):  # weights are floored, not rounded
            p = tie_probabilities(orc, seed, c0, frac)
            assert 0 < p[0] < p.sum()
            assert int(orc.sample(p, 1, seed=seed, counter0=c0)[0]) == 1


def test_sampler_rejects_bad_probabilities(orc):
    with pytest.raises(ValueError):
        orc.sample(np.zeros(8), 10, seed=1)
    with pytest.raises(ValueError):
        orc.sample(np.full(8, 0.5), 10, seed=1)


def test_collapse_of_ghz_and_bell(orc):
    """GHZ: measuring any qubit gives 0 or 1 with probability 1/2 and leaves a
    basis state; the marginal probability equals the oracle's marginal."""
    n = 5
    psi = orc.simulate(inputs.ghz(n))
    out, p = orc.collapse(psi, (2,), 1)
    assert abs(p - 0.5) < 1e-14
    want = np.zeros(1 << n); want[-1] = 1
    np.testing.assert_allclose(out, want, atol=1e-14)
    st = inputs.gaussian_state(6, seed=3)
    for qubits, o in (((0,), 1), ((4, 1), 2), ((5, 3, 0), 5)):
        out, p = orc.collapse(st, qubits, o)
        assert abs(p - orc.probabilities(st, qubits)[o]) < 1e-14
        assert abs(np.linalg.norm(out) - 1) < 1e-14


# ---------------------------------------------------------------- Sec. 3.3 evolution

def _kron_z(n, zmask):
    """Z on every qubit of zmask, identity elsewhere, by Kronecker products
    (qubit n-1 leftmost, so qubit q is bit q of the index)."""
    Z, I = np.diag([1.0, -1.0]), np.eye(2)
    M = np.array([[1.0]])
    for q in reversed(range(n)):
        M = np.kron(M, Z if (zmask >> q) & 1 else I)
    return M


def test_rzz_is_the_exponential_of_zz(orc):
    from scipy.linalg import expm
    for th in (0.3, -1.7, 2 * np.pi / 3):
        g = inputs.Gate("rzz", (0, 1), (), (th,))
        np.testing.assert_allclose(orc.gate_matrix(g), expm(-0.5j * th * np.kron(np.diag([1, -1]), np.diag([1, -1]))),
                                   atol=1e-14)


def test_pauli_phase_matches_expm_of_kron_built_diagonal(orc):
    from scipy.linalg import expm
    n = 5
    rng = np.random.default_rng(3)
    psi = inputs.gaussian_state(n, seed=3)
    for uniform in (True, False):
        z = [int(v) for v in rng.integers(1, 1 << n, size=7)]
        c = [0.8] * 7 if uniform else list(rng.standard_normal(7))
        D = sum(ci * _kron_z(n, zi) for zi, ci in zip(z, c))
        np.testing.assert_allclose(orc.pauli_phase(psi, z, c, 0.37), expm(-0.37j * D) @ psi, atol=1e-13)


def test_dense_hamiltonian_matches_kron_sum(orc):
    n = 4
    X, Z, I = np.array([[0, 1], [1, 0]]), np.diag([1, -1]), np.eye(2)

    def op(mats):
        M = np.array([[1.0]])
        for q in reversed(range(n)):
            M = np.kron(M, mats.get(q, I))
        return M
    want = -sum(op({i: Z, i + 1: Z}) for i in range(n - 1)) - 0.7 * sum(op({i: X}) for i in range(n))
    np.testing.assert_allclose(orc.dense_hamiltonian(n, inputs.tfim_target(n, 0.7)), want, atol=1e-14)


def test_trotter_circuit_converges_to_exact_evolution_at_second_order(orc):
    """The symmetric Trotter step has error O(dt^3) per step: halving dt over
    a fixed time cuts the difference to the exact piecewise evolution 4x."""
    n, h, T = 6, 1.0, 2.0
    H0, H1 = inputs.x_field(n), inputs.tfim_target(n, h)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        got = orc.simulate(inputs.adiabatic_tfim(n, h, T, dt))
        errs.append(np.max(np.abs(got - orc.adiabatic_exact(n, H0, H1, T, dt))))
    assert errs[0] < 1e-2
    for a, b in zip(errs, errs[1:]):
        assert 3.6 < a / b < 4.4, errs


def test_slow_adiabatic_sweep_reaches_the_tfim_ground_state(orc):
    """Adiabatic theorem: a slow sweep ends near the ground energy of H1."""
    n, h = 6, 1.0
    H1 = inputs.tfim_target(n, h)
    E0 = np.linalg.eigvalsh(orc.dense_hamiltonian(n, H1))[0]
    e_fast = orc.expectation(orc.simulate(inputs.adiabatic_tfim(n, h, 2.0, 0.05)), H1)
    e_slow = orc.expectation(orc.simulate(inputs.adiabatic_tfim(n, h, 20.0, 0.05)), H1)
    assert E0 < e_slow < E0 + 2e-3 and e_slow < e_fast

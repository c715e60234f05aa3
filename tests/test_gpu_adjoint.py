"""GPU parity of the adjoint-method gradient against the oracle's
parameter-shift gradients (exact for exp(-i theta P / 2)) and central finite
differences, energies against the oracle, and the autograd wrapper."""
import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_08826_gb300 import build, binding
    build.build()
    return binding


def mixed_ansatz(n, layers, seed):
    """RX / RY / RZ rotations (all three generators) with CZ and H in between."""
    rng = np.random.default_rng(seed)
    gates, p = [], 0
    for _ in range(layers):
        for q_ in range(n):
            name = ("rx", "ry", "rz")[int(rng.integers(3))]
            gates.append(inputs.Gate(name, (q_,), (), (float(rng.uniform(0, 6.28)),), p)); p += 1
        for i in range(0, n - 1, 2):
            gates.append(inputs.Gate("cz", (i, i + 1)))
        gates.append(inputs.Gate("h", (int(rng.integers(n)),)))
    return inputs.Circuit(n, gates)


# Tolerances: the measured errors against the oracle's parameter shift times
# about 10 (complex64: <= 6.2e-7; complex128: <= 3e-14).
@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 5e-6)])
def test_adjoint_matches_parameter_shift(q, orc, dtype, tol):
    circ = mixed_ansatz(6, 3, seed=1)
    ham = inputs.tfim(6)
    rng = np.random.default_rng(2)
    thetas = rng.uniform(0, 2 * np.pi, size=(3, circ.nparams))
    grads, en = q.adjoint_grad(circ, ham, thetas, dtype)
    for s in range(3):
        want = orc.parameter_shift_gradient(circ, ham, thetas[s])
        print(f"adjoint mixed6 {dtype}: max gradient err {np.max(np.abs(grads[s] - want)):.3e}")
        np.testing.assert_allclose(grads[s], want, atol=tol)
        assert abs(en[s] - orc.energy(circ, ham, thetas[s])) < tol
    fd = orc.finite_difference_gradient(circ, ham, thetas[0], h=1e-4)
    np.testing.assert_allclose(grads[0], fd, atol=max(tol, 1e-6))  # O(h^2) truncation of the differences


def test_adjoint_variational_12q_all_parameters(q, orc):
    """The benchmark ansatz (RY/RZ + CZ ladder) at 12 qubits, 4 layers,
    H = sum_i (Z_i Z_{i+1} + 0.5 X_i), complex128: all 96 gradients."""
    circ = inputs.variational(12, 4, seed=3)
    ham = inputs.tfim(12)
    th = circ.params()
    grads, en = q.adjoint_grad(circ, ham, th[None, :], "c128")
    np.testing.assert_allclose(grads[0], orc.parameter_shift_gradient(circ, ham, th), atol=1e-12)
    assert abs(en[0] - orc.energy(circ, ham, th)) < 1e-12


def test_autograd_function(q, orc):
    import torch
    circ = inputs.variational(5, 2, seed=4)
    ham = inputs.tfim(5)
    f = q.adjoint_energy(circ, ham, "c128")
    theta = torch.tensor(np.stack([circ.params(), circ.params() + 0.1]), dtype=torch.float64, requires_grad=True)
    e = f(theta)
    (2.0 * e[0] + 3.0 * e[1]).backward()
    g0 = orc.parameter_shift_gradient(circ, ham, circ.params())
    g1 = orc.parameter_shift_gradient(circ, ham, circ.params() + 0.1)
    np.testing.assert_allclose(theta.grad.numpy(), np.stack([2 * g0, 3 * g1]), atol=1e-12)


def test_adjoint_24q_config_properties(q):
    """The 24-qubit, 10-layer ansatz of the gradient workload (480 parameters):
    a few gradient entries against central differences of the library's own
    energies (h = 1e-4, complex128), and complex64 against complex128."""
    circ = inputs.variational(24, 10, seed=5)
    ham = inputs.tfim(24)
    th = circ.params()
    g64, e64 = q.adjoint_grad(circ, ham, th[None, :], "c64")
    g128, e128 = q.adjoint_grad(circ, ham, th[None, :], "c128")
    assert abs(e64[0] - e128[0]) < 5e-6
    np.testing.assert_allclose(g64[0], g128[0], atol=5e-6)
    h = 1e-4
    for p_ in (0, 237, 479):
        tp, tm = th.copy(), th.copy()
        tp[p_] += h
        tm[p_] -= h
        _, ep = q.adjoint_grad(circ, ham, tp[None, :], "c128")
        _, em = q.adjoint_grad(circ, ham, tm[None, :], "c128")
        assert abs((ep[0] - em[0]) / (2 * h) - g128[0, p_]) < 1e-6


def stacked_ansatz(n, layers, seed):
    """Runs of rotations on one qubit separated by fixed SU(2) gates and
    Hadamards (the reverse sweep moves each gradient term ahead of them,
    conjugating its Pauli), with controlled gates on the same qubits (which
    stop it) and CZ layers."""
    rng = np.random.default_rng(seed)
    gates, p = [], 0
    for _ in range(layers):
        for q_ in range(n):
            for name in ("rx", "ry", "rz", "rx"):
                gates.append(inputs.Gate(name, (q_,), (), (float(rng.uniform(0, 6.28)),), p)); p += 1
                if rng.uniform() < 0.3:
                    gates.append(inputs.Gate("su2", (q_,), (), inputs.haar_su2_quaternion(rng)))
            if q_ % 3 == 0:
                gates.append(inputs.Gate("h", (q_,)))
        for i in range(0, n - 1, 2):
            gates.append(inputs.Gate("cz", (i, i + 1)))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        gates.append(inputs.Gate("x", (a,), (b,)))
        gates.append(inputs.Gate("ry", (b,), (), (float(rng.uniform(0, 6.28)),), p)); p += 1
    return inputs.Circuit(n, gates)


@pytest.mark.parametrize("specialize", [-1, 1])
@pytest.mark.parametrize("maker", ["variational", "mixed", "stacked"])
def test_fused_adjoint_complex64_matches_parameter_shift(q, orc, maker, specialize):
    """complex64 from 12 qubits runs the reverse sweep as two-state register
    tiles (gradient terms accumulated per CTA), through the op-list
    interpreter or through kernels compiled for the circuit: all gradients
    vs the oracle."""
    circ = {"variational": lambda: inputs.variational(13, 2, seed=7),
            "mixed": lambda: mixed_ansatz(13, 2, seed=8),
            "stacked": lambda: stacked_ansatz(12, 2, seed=10)}[maker]()
    ham = inputs.tfim(circ.n)
    rng = np.random.default_rng(9)
    thetas = rng.uniform(0, 2 * np.pi, size=(2, circ.nparams))
    prev = q.adjoint_specialize(specialize)
    try:
        grads, en = q.adjoint_grad(circ, ham, thetas, "c64")
    finally:
        q.adjoint_specialize(prev)
    g128, e128 = q.adjoint_grad(circ, ham, thetas, "c128")   # the plain sweeps path
    for s in range(2):
        want = orc.parameter_shift_gradient(circ, ham, thetas[s])
        print(f"adjoint fused {maker}: max gradient err {np.max(np.abs(grads[s] - want)):.3e}, "
              f"energy err {abs(en[s] - orc.energy(circ, ham, thetas[s])):.3e}")
        np.testing.assert_allclose(grads[s], want, atol=4e-6)  # measured <= 4.1e-7
        np.testing.assert_allclose(g128[s], want, atol=1e-12)
        assert abs(en[s] - orc.energy(circ, ham, thetas[s])) < 4e-6


@pytest.mark.parametrize("dtype,tol", [("c64", 2e-6), ("c128", 1e-12)])  # measured 2.1e-7 / 1.8e-14
def test_adjoint_general_pauli_hamiltonian(q, orc, dtype, tol):
    """A Hamiltonian of mixed Pauli strings on 14 qubits: X masks inside the
    low 12 qubits, across qubits 0..4 and the top chunk, and across both
    (handled by different passes of lambda = H psi), with Y and Z factors."""
    n = 14
    terms = [  # (x mask, z mask, coefficient)
        (0, 0b11 << 3, 0.7),
        (1 << 2, 0, -0.4),
        ((1 << 2) | (1 << 13), 1 << 5, 0.3),        # X2 X13 Z5
        ((1 << 7) | (1 << 13), (1 << 7), 0.25),     # Y7 X13: spans the chunks
        ((1 << 12), (1 << 12) | (1 << 0), -0.6),    # Z0 Y12
        ((1 << 11) | (1 << 4), 1 << 11, 0.45),      # X4 Y11
        (0, (1 << 13) | 1, 0.2),
    ]
    ham = inputs.PauliSum(np.array([t[0] for t in terms], dtype=np.uint64),
                          np.array([t[1] for t in terms], dtype=np.uint64),
                          np.array([t[2] for t in terms]))
    circ = mixed_ansatz(n, 2, seed=12)
    th = np.random.default_rng(13).uniform(0, 2 * np.pi, size=(1, circ.nparams))
    grads, en = q.adjoint_grad(circ, ham, th, dtype)
    want = orc.parameter_shift_gradient(circ, ham, th[0])
    print(f"adjoint general-pauli {dtype}: max gradient err {np.max(np.abs(grads[0] - want)):.3e}")
    np.testing.assert_allclose(grads[0], want, atol=tol)
    assert abs(en[0] - orc.energy(circ, ham, th[0])) < tol


@pytest.mark.parametrize("n,dtype,tol", [(6, "c128", 1e-12), (6, "c64", 2e-6), (13, "c64", 2e-6)])
def test_adjoint_from_a_start_state(q, orc, n, dtype, tol):
    """Gradients of <psi0|U^dag H U|psi0> from a seeded Gaussian start state
    (one sweep per gate below 12 qubits, two-state register stages for
    complex64 from 12) against the oracle's parameter shift from the same
    state; the |0...0> gradients differ, so the start state is really used."""
    circ = mixed_ansatz(n, 2, seed=20 + n)
    ham = inputs.tfim(n)
    psi0 = inputs.gaussian_state(n, seed=21 + n)
    s0 = q.State(n, dtype).from_host(psi0.astype(np.complex64 if dtype == "c64" else np.complex128))
    psi0_used = s0.to_host().astype(np.complex128)
    th = np.random.default_rng(22).uniform(0, 2 * np.pi, size=(2, circ.nparams))
    grads, en = q.adjoint_grad(circ, ham, th, dtype, psi0=s0)
    for s in range(2):
        want = orc.parameter_shift_gradient(circ, ham, th[s], psi0=psi0_used)
        print(f"adjoint psi0 n={n} {dtype}: max gradient err {np.max(np.abs(grads[s] - want)):.3e}")
        np.testing.assert_allclose(grads[s], want, atol=tol)
        assert abs(en[s] - orc.energy(circ, ham, th[s], psi0_used)) < tol
    g_zero, _ = q.adjoint_grad(circ, ham, th[:1], dtype)
    assert np.max(np.abs(g_zero[0] - grads[0])) > 1e-2
    # the start state is read, not written
    np.testing.assert_array_equal(s0.to_host().astype(np.complex128), psi0_used)


@pytest.mark.parametrize("dtype,tol", [("c64", 2e-6), ("c128", 1e-11)])  # measured 2.5e-7 / 6.4e-13
@pytest.mark.parametrize("specialize", [0, -1])
def test_adjoint_24q_config_against_oracle(q, dtype, tol, specialize):
    """The gradient workload's own configuration (24 qubits, 10 layers, 480
    parameters, H = sum(Z_i Z_i+1 + 0.5 X_i), parameter set 0 of the seeded
    64): energy and gradient entries against the oracle's parameter-shift
    values stored by tests/golden/make_golden.py."""
    import os
    from golden import make_golden
    g = make_golden.read(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "adjoint24_tfim_grad.txt"))
    circ = inputs.variational(24, 10, seed=5)
    ham = inputs.tfim(24)
    th = np.random.default_rng(0).uniform(0, 2 * np.pi, size=(64, circ.nparams))[:1]
    if dtype == "c128" and specialize:
        pytest.skip("complex128 runs the plain sweeps either way")
    prev = q.adjoint_specialize(specialize)  # 0: compiled stage kernels at 24 qubits
    try:
        grads, en = q.adjoint_grad(circ, ham, th, dtype)
    finally:
        q.adjoint_specialize(prev)
    errs = [abs(grads[0, p] - v) for p, v in g["grad"]]
    print(f"adjoint24 {dtype}: energy err {abs(en[0] - g['energy']):.3e}, gradient errs "
          + " ".join(f"{e:.2e}" for e in errs))
    assert abs(en[0] - g["energy"]) < tol
    assert max(errs) < tol

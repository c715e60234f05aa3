"""Plain complex128 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the library in
``paper_2203_08826_gb300``: gate matrices are built here from their textbook
definitions, gates are applied by the literal contraction of Eq. (1) in
``oracle.c``, and every derived quantity (probabilities, Pauli expectations,
gradients, samples) is computed from its definition.

Gates are read by duck typing from objects with ``name``, ``targets``,
``controls``, ``params`` and ``matrix`` attributes (the seeded workload
generators produce them); nothing from the library is imported.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against an independent fact (Kronecker-product matrices, closed forms such as
the DFT and GHZ amplitudes, norm and inverse invariants, known-answer vectors
of Philox4x32-10, parameter-shift vs finite differences, a chi-square test of
the sampler).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborcl.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP over the plain index loop)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            U64 = ctypes.c_uint64
            lib.orc_apply_gate.argtypes = [P, I, P, P, I, P, I]
            lib.orc_apply_gate.restype = I
            lib.orc_marginal_probs.argtypes = [P, I, P, I, P]
            lib.orc_marginal_probs.restype = I
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_sample.argtypes = [P, U64, U64, U64, U64, P]
            lib.orc_sample.restype = I
            lib.orc_set_threads.argtypes = [I]
            lib.orc_set_threads.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- gate matrices
# Textbook definitions, written out entry by entry.

_SQ2 = 1.0 / math.sqrt(2.0)


def gate_matrix(g) -> np.ndarray:
    """2^k x 2^k complex128 matrix of a gate specification (targets[0] = MSB)."""
    name = g.name
    p = tuple(g.params)
    if name == "h":
        return np.array([[_SQ2, _SQ2], [_SQ2, -_SQ2]], dtype=complex)
    if name == "x":
        return np.array([[0, 1], [1, 0]], dtype=complex)
    if name == "y":
        return np.array([[0, -1j], [1j, 0]], dtype=complex)
    if name == "z":
        return np.array([[1, 0], [0, -1]], dtype=complex)
    if name == "s":
        return np.array([[1, 0], [0, 1j]], dtype=complex)
    if name == "t":
        return np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=complex)
    if name == "rx":   # exp(-i theta X / 2)
        c, s = math.cos(p[0] / 2), math.sin(p[0] / 2)
        return np.array([[c, -1j * s], [-1j * s, c]], dtype=complex)
    if name == "ry":   # exp(-i theta Y / 2)
        c, s = math.cos(p[0] / 2), math.sin(p[0] / 2)
        return np.array([[c, -s], [s, c]], dtype=complex)
    if name == "rz":   # exp(-i theta Z / 2)
        return np.array([[np.exp(-0.5j * p[0]), 0], [0, np.exp(0.5j * p[0])]], dtype=complex)
    if name == "phase":
        return np.array([[1, 0], [0, np.exp(1j * p[0])]], dtype=complex)
    if name == "rzz":  # exp(-i theta Z (x) Z / 2)
        even, odd = np.exp(-0.5j * p[0]), np.exp(0.5j * p[0])
        return np.diag([even, odd, odd, even]).astype(complex)
    if name == "cz":
        return np.diag([1, 1, 1, -1]).astype(complex)
    if name == "swap":
        return np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    if name == "su2":
        a, b, c, d = p
        return np.array([[a + 1j * b, c + 1j * d], [-c + 1j * d, a - 1j * b]], dtype=complex)
    if name == "matrix":
        return np.asarray(g.matrix, dtype=complex)
    raise ValueError(f"unknown gate {name!r}")


def pauli_generator(name: str) -> np.ndarray:
    """P such that the rotation is exp(-i theta P / 2)."""
    return {"rx": np.array([[0, 1], [1, 0]], dtype=complex),
            "ry": np.array([[0, -1j], [1j, 0]], dtype=complex),
            "rz": np.array([[1, 0], [0, -1]], dtype=complex)}[name]


# ---------------------------------------------------------------- Eq. (1)

def apply_matrix(psi: np.ndarray, G: np.ndarray, targets: Sequence[int],
                 controls: Sequence[int] = ()) -> np.ndarray:
    """Apply G in place to psi (complex128, length 2^n) by Eq. (1)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    n = int(psi.size).bit_length() - 1
    assert psi.size == 1 << n
    G = np.ascontiguousarray(G, dtype=np.complex128)
    k = len(targets)
    assert G.shape == (1 << k, 1 << k)
    t = np.asarray(targets, dtype=np.int32)
    c = np.asarray(controls if len(controls) else [0], dtype=np.int32)
    rc = _load().orc_apply_gate(_ptr(psi), n, _ptr(G), _ptr(t), k, _ptr(c), len(controls))
    if rc != 0:
        raise ValueError(f"orc_apply_gate rejected targets={targets} controls={controls}")
    return psi


def apply_gate(psi: np.ndarray, g) -> np.ndarray:
    return apply_matrix(psi, gate_matrix(g), g.targets, g.controls)


def inverse_gate_matrix(g) -> np.ndarray:
    return gate_matrix(g).conj().T


def run(psi: np.ndarray, gates: Iterable) -> np.ndarray:
    """Gate-by-gate, unfused simulation (in place)."""
    for g in gates:
        apply_gate(psi, g)
    return psi


def run_inverse(psi: np.ndarray, gates: Sequence) -> np.ndarray:
    """Apply the inverse circuit: reverse order, conjugate transposes."""
    for g in reversed(list(gates)):
        apply_matrix(psi, inverse_gate_matrix(g), g.targets, g.controls)
    return psi


def set_threads(nthreads: int) -> int:
    """Threads of the Eq. (1) loop from now on (0 keeps the setting); returns
    the previous count.  Used to time the oracle on one core."""
    return int(_load().orc_set_threads(int(nthreads)))


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def simulate(circuit, psi0: np.ndarray | None = None) -> np.ndarray:
    psi = zero_state(circuit.n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    return run(psi, circuit.gates)


# ---------------------------------------------------------------- measurements

def probabilities(psi: np.ndarray, qubits: Sequence[int] | None = None) -> np.ndarray:
    """|psi(x)|^2 (qubits=None) or the marginal over ``qubits`` (qubits[0] = MSB)."""
    n = int(psi.size).bit_length() - 1
    if qubits is None:
        return (psi.real * psi.real + psi.imag * psi.imag).astype(np.float64)
    q = np.asarray(qubits, dtype=np.int32)
    out = np.zeros(1 << len(q), dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    rc = _load().orc_marginal_probs(_ptr(psi), n, _ptr(q if len(q) else np.zeros(1, np.int32)),
                                    len(q), _ptr(out))
    if rc != 0:
        raise ValueError("bad qubit list")
    return out


_PAULI = {(1, 0): "x", (1, 1): "y", (0, 1): "z"}


def pauli_apply(psi: np.ndarray, xmask: int, zmask: int) -> np.ndarray:
    """P|psi> for the Pauli string (xmask, zmask), by single-qubit matrices."""
    out = np.array(psi, dtype=np.complex128)
    n = int(psi.size).bit_length() - 1
    for q in range(n):
        key = ((int(xmask) >> q) & 1, (int(zmask) >> q) & 1)
        if key in _PAULI:
            apply_matrix(out, gate_matrix(_Named(_PAULI[key])), (q,))
    return out


class _Named:
    def __init__(self, name, params=()):
        self.name, self.params, self.matrix = name, params, None


def expectation(psi: np.ndarray, ham) -> float:
    """<psi| sum_t c_t P_t |psi> = sum_t c_t <psi|P_t psi> (real part)."""
    total = 0.0
    for xm, zm, c in zip(ham.xmask, ham.zmask, ham.coeff):
        total += float(c) * np.vdot(psi, pauli_apply(psi, int(xm), int(zm))).real
    return total


def hamiltonian_apply(psi: np.ndarray, ham) -> np.ndarray:
    out = np.zeros_like(psi)
    for xm, zm, c in zip(ham.xmask, ham.zmask, ham.coeff):
        out += float(c) * pauli_apply(psi, int(xm), int(zm))
    return out


# ---------------------------------------------------------------- Sec. 3.3

def pauli_phase(psi: np.ndarray, zmask: Sequence[int], coeff: Sequence[float], theta: float) -> np.ndarray:
    """exp(-i theta D) psi for D = sum_t coeff[t] Z(zmask[t]), by definition:
    D(x) = sum_t coeff[t] (-1)^popcount(x & zmask[t])."""
    x = np.arange(psi.size, dtype=np.uint64)
    d = np.zeros(psi.size)
    for z, c in zip(zmask, coeff):
        parity = np.array([bin(int(v)).count("1") & 1 for v in (x & np.uint64(z))])
        d += float(c) * (1 - 2 * parity)
    return psi * np.exp(-1j * theta * d)


def dense_hamiltonian(n: int, ham) -> np.ndarray:
    """The 2^n x 2^n matrix of a Pauli sum, column by column (n <= 12)."""
    N = 1 << n
    H = np.zeros((N, N), dtype=complex)
    for j in range(N):
        e = np.zeros(N, dtype=complex)
        e[j] = 1.0
        H[:, j] = hamiltonian_apply(e, ham)
    return H


def adiabatic_exact(n: int, H0, H1, T: float, dt: float) -> np.ndarray:
    """Sec. 3.3's direct method: psi <- expm(-i H(s_k) dt) psi for each step,
    H(s) = (1 - s) H0 + s H1 at the step's mid-point s_k = (k + 1/2) dt / T,
    from the ground state of H0 = -sum X_i (|+...+>)."""
    from scipy.linalg import expm
    A = dense_hamiltonian(n, H0)
    B = dense_hamiltonian(n, H1)
    psi = np.full(1 << n, 2.0 ** (-n / 2), dtype=complex)
    steps = int(round(T / dt))
    for k in range(steps):
        s = (k + 0.5) * dt / T
        psi = expm(-1j * dt * ((1 - s) * A + s * B)) @ psi
    return psi


def energy(circuit, ham, theta: Sequence[float] | None = None, psi0: np.ndarray | None = None) -> float:
    """<psi0| U(theta)^dag H U(theta) |psi0>, psi0 = |0...0> when not given."""
    c = circuit if theta is None else circuit.with_params(theta)
    return expectation(simulate(c, psi0), ham)


def parameter_shift_gradient(circuit, ham, theta: Sequence[float],
                             which: Sequence[int] | None = None, psi0: np.ndarray | None = None) -> np.ndarray:
    """d<H>/d theta_l by the two-term parameter-shift rule, exact for
    exp(-i theta P / 2) with a Pauli P:  [E(theta + pi/2) - E(theta - pi/2)] / 2
    (from any start state psi0).  Each parameter index appears in exactly one
    gate of the circuit."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = range(len(theta)) if which is None else which
    grad = np.zeros(len(theta))
    for l in idx:
        tp = theta.copy(); tp[l] += math.pi / 2
        tm = theta.copy(); tm[l] -= math.pi / 2
        grad[l] = 0.5 * (energy(circuit, ham, tp, psi0) - energy(circuit, ham, tm, psi0))
    return grad


def finite_difference_gradient(circuit, ham, theta: Sequence[float], h: float = 1e-4,
                               which: Sequence[int] | None = None, psi0: np.ndarray | None = None) -> np.ndarray:
    """Central differences [E(theta + h) - E(theta - h)] / (2h)."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = range(len(theta)) if which is None else which
    grad = np.zeros(len(theta))
    for l in idx:
        tp = theta.copy(); tp[l] += h
        tm = theta.copy(); tm[l] -= h
        grad[l] = (energy(circuit, ham, tp, psi0) - energy(circuit, ham, tm, psi0)) / (2 * h)
    return grad


def collapse(psi: np.ndarray, qubits: Sequence[int], outcome: int):
    """Measurement collapse by definition: keep the amplitudes whose listed
    bits (qubits[0] = most significant) spell `outcome`, renormalise.
    Returns (new state, probability of the outcome)."""
    m = len(qubits)
    x = np.arange(psi.size)
    spelled = np.zeros(psi.size, dtype=np.int64)
    for q in qubits:
        spelled = (spelled << 1) | ((x >> q) & 1)
    keep = spelled == outcome
    p = float(np.sum(np.abs(psi[keep]) ** 2))
    out = np.where(keep, psi, 0).astype(np.complex128)
    return out / np.sqrt(p), p


# ---------------------------------------------------------------- sampling

def philox4x32_10(counter: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def sample(p: np.ndarray, nshots: int, seed: int, counter0: int = 0) -> np.ndarray:
    """Inverse-CDF shots over integer weights floor(p 2^62) (see oracle.c)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros(max(nshots, 1), dtype=np.uint64)
    rc = _load().orc_sample(_ptr(p), p.size, nshots, seed & (2**64 - 1),
                            counter0 & (2**64 - 1), _ptr(out))
    if rc != 0:
        raise ValueError("probabilities must be >= 0 with 0 < sum <= 1.5")
    return out[:nshots]

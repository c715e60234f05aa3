"""Seeded synthetic workloads: circuits, initial states and Hamiltonians.

This module only draws random numbers and lays out gate *specifications*
(gate name, qubits, angles).  It holds none of the simulation arithmetic: no
gate matrix is formed here, so the library and the CPU oracle each build the
matrices of named gates themselves from these specifications.  Both sides
consume the same lists, which makes them the shared seeded inputs.

The circuit families stand in for the paper's benchmark circuits (Sec. 3.1,
Table "benchmark circuits": qft, variational, supremacy-style random
circuits), whose OpenQASM files live in an external repository that is not
available here.  Qubit q is bit q of the amplitude index (qubit 0 = LSB).

Every generator uses numpy's PCG64 seeded through ``SeedSequence(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

# Gate names understood by both the library binding and the oracle.
#   h x y z s t            fixed single-qubit gates
#   rx ry rz (theta)       exp(-i theta P / 2)
#   phase (phi)            diag(1, e^{i phi})
#   cz (a, b)              diag(1, 1, 1, -1) on targets (a, b)
#   swap (a, b)            exchange of two qubits
#   su2 (a, b, c, d)       unit quaternion -> [[a+ib, c+id], [-c+id, a-ib]]
#   rzz (theta)            exp(-i theta Z Z / 2) on targets (a, b)
#   matrix                 explicit 2^k x 2^k complex matrix in ``matrix``
GATE_NAMES = ("h", "x", "y", "z", "s", "t", "rx", "ry", "rz", "phase", "cz",
              "swap", "su2", "rzz", "matrix")


@dataclass(frozen=True)
class Gate:
    name: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    params: Tuple[float, ...] = ()
    pindex: int = -1            # trainable-parameter index (rx/ry/rz), -1 if fixed
    matrix: np.ndarray | None = field(default=None, compare=False)

    @property
    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


@dataclass
class Circuit:
    n: int
    gates: List[Gate]
    name: str = ""

    def __len__(self) -> int:
        return len(self.gates)

    @property
    def nparams(self) -> int:
        return 1 + max((g.pindex for g in self.gates), default=-1)

    def params(self) -> np.ndarray:
        """Current values of the trainable parameters, indexed by pindex."""
        out = np.zeros(self.nparams)
        for g in self.gates:
            if g.pindex >= 0:
                out[g.pindex] = g.params[0]
        return out

    def with_params(self, theta: Sequence[float]) -> "Circuit":
        gates = [Gate(g.name, g.targets, g.controls, (float(theta[g.pindex]),), g.pindex)
                 if g.pindex >= 0 else g for g in self.gates]
        return Circuit(self.n, gates, self.name)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))


def qft(n: int) -> Circuit:
    """Quantum Fourier transform: H on each qubit, a controlled phase
    R_k = diag(1, e^{2 pi i / 2^k}) on every pair, then the final swaps.

    With qubit 0 as the least significant bit the most significant qubit is
    processed first: for j = n-1 .. 0, H(j), then for m = j-1 .. 0 the
    controlled R_{j-m+1} with control m and target j; finally SWAP(i, n-1-i)
    for i < n/2.  The count n + n(n-1)/2 + floor(n/2) is 480 at n = 30, the
    figure of the paper's circuit table.
    """
    gates: List[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("h", (j,)))
        for m in range(j - 1, -1, -1):
            k = j - m + 1
            gates.append(Gate("phase", (j,), (m,), (2.0 * math.pi / (1 << k),)))
    for i in range(n // 2):
        gates.append(Gate("swap", (i, n - 1 - i)))
    return Circuit(n, gates, f"qft{n}")


def haar_su2_quaternion(rng: np.random.Generator) -> Tuple[float, float, float, float]:
    """A Haar-random SU(2) element as a unit quaternion: a Gaussian 4-vector
    normalised to length 1 is uniform on the 3-sphere, i.e. on SU(2)."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    return tuple(float(v) for v in q)


def random_matching(rng: np.random.Generator, n: int) -> List[Tuple[int, int]]:
    """Random perfect matching of n qubits: a Fisher-Yates shuffle of 0..n-1,
    paired consecutively (n // 2 pairs)."""
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        j = int(rng.integers(0, i + 1))
        perm[i], perm[j] = perm[j], perm[i]
    return [(min(perm[2 * i], perm[2 * i + 1]), max(perm[2 * i], perm[2 * i + 1]))
            for i in range(n // 2)]


def random_circuit(n: int, depth: int, seed: int) -> Circuit:
    """Supremacy-style random circuit: each layer is a Haar-random SU(2) on
    every qubit followed by CZ on a random perfect matching of the qubits."""
    rng = _rng(seed)
    gates: List[Gate] = []
    for _ in range(depth):
        for q in range(n):
            gates.append(Gate("su2", (q,), (), haar_su2_quaternion(rng)))
        for a, b in random_matching(rng, n):
            gates.append(Gate("cz", (a, b)))
    return Circuit(n, gates, f"random{n}x{depth}")


def variational(n: int, layers: int, seed: int) -> Circuit:
    """Layered variational ansatz: RY(theta_q) then RZ(phi_q) on every qubit,
    then a CZ ladder (i, i+1) for i = 0 .. n-2; angles ~ U(0, 2 pi).  Every
    rotation is a trainable parameter (pindex in gate order)."""
    rng = _rng(seed)
    gates: List[Gate] = []
    p = 0
    for _ in range(layers):
        th = rng.uniform(0.0, 2.0 * math.pi, size=n)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=n)
        for q in range(n):
            gates.append(Gate("ry", (q,), (), (float(th[q]),), p)); p += 1
            gates.append(Gate("rz", (q,), (), (float(ph[q]),), p)); p += 1
        for i in range(n - 1):
            gates.append(Gate("cz", (i, i + 1)))
    return Circuit(n, gates, f"variational{n}x{layers}")


def ghz(n: int) -> Circuit:
    """H(0) then CNOT(0 -> i) for i = 1 .. n-1."""
    gates = [Gate("h", (0,))] + [Gate("x", (i,), (0,)) for i in range(1, n)]
    return Circuit(n, gates, f"ghz{n}")


def batch_circuits(count: int, seed: int, nmin: int = 12, nmax: int = 20,
                   lmin: int = 4, lmax: int = 12, limit: int | None = None) -> List[Circuit]:
    """Many small uneven circuits: n ~ U{nmin..nmax}, layers ~ U{lmin..lmax}
    (both inclusive), each a variational ansatz with its own angles.  With
    `limit`, only the first `limit` circuits of the same batch are built."""
    rng = _rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ls = rng.integers(lmin, lmax + 1, size=count)
    seeds = rng.integers(0, 2**63 - 1, size=count)
    k = count if limit is None else min(limit, count)
    return [variational(int(n), int(l), int(s)) for n, l, s in zip(ns[:k], ls[:k], seeds[:k])]


def gaussian_state(n: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian amplitudes (re, im ~ N(0, 1)), normalised."""
    rng = _rng(seed)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    return psi.astype(np.complex128)


@dataclass
class PauliSum:
    """sum_t coeff[t] * P_t with P_t given by bit masks: bit q of xmask / zmask
    selects X (x=1,z=0), Z (x=0,z=1) or Y (x=1,z=1) on qubit q."""
    xmask: np.ndarray
    zmask: np.ndarray
    coeff: np.ndarray

    def __len__(self) -> int:
        return len(self.coeff)


def zz_chain(n: int) -> PauliSum:
    """sum_{i=0}^{n-2} Z_i Z_{i+1} (open chain)."""
    z = np.array([(1 << i) | (1 << (i + 1)) for i in range(n - 1)], dtype=np.uint64)
    return PauliSum(np.zeros(n - 1, dtype=np.uint64), z, np.ones(n - 1))


def tfim(n: int, hx: float = 0.5) -> PauliSum:
    """sum_i (Z_i Z_{i+1} + hx X_i): the ZZ chain plus a transverse field."""
    zz = zz_chain(n)
    x = np.array([1 << i for i in range(n)], dtype=np.uint64)
    return PauliSum(np.concatenate([zz.xmask, x]),
                    np.concatenate([zz.zmask, np.zeros(n, dtype=np.uint64)]),
                    np.concatenate([zz.coeff, np.full(n, hx)]))


def x_field(n: int) -> PauliSum:
    """-sum_i X_i: the starting Hamiltonian of the adiabatic evolution
    (Sec. 3.3; its ground state is |+...+>)."""
    x = np.array([1 << i for i in range(n)], dtype=np.uint64)
    return PauliSum(x, np.zeros(n, dtype=np.uint64), -np.ones(n))


def tfim_target(n: int, h: float = 1.0) -> PauliSum:
    """-sum_i (Z_i Z_{i+1} + h X_i), open chain: the target Hamiltonian of the
    adiabatic evolution benchmark (Sec. 3.3)."""
    t = tfim(n, h)
    return PauliSum(t.xmask, t.zmask, -t.coeff)


def adiabatic_schedule(T: float, dt: float) -> List[float]:
    """Mid-step values s_k = (k + 1/2) dt / T of the linear schedule s(t) = t / T."""
    steps = int(round(T / dt))
    return [(k + 0.5) * dt / T for k in range(steps)]


def adiabatic_tfim(n: int, h: float, T: float, dt: float) -> Circuit:
    """Adiabatic evolution from -sum X_i to the TFIM target as a circuit
    (Sec. 3.3: the Trotter decomposition turns the evolution into gates).

    H(s) = (1 - s) H0 + s H1 = A(s) sum_i X_i + B(s) sum_i Z_i Z_{i+1} with
    A = -((1 - s) + s h), B = -s.  Each step of length dt is the symmetric
    (second-order) product exp(-i A dt/2 sum X) exp(-i B dt sum ZZ)
    exp(-i A dt/2 sum X) at the step's mid-point s_k: RX(A dt) on every qubit,
    RZZ(2 B dt) on every pair (i, i+1), RX(A dt) again.  The circuit starts
    with H on every qubit (|0...0> -> |+...+>, the ground state of H0).
    """
    gates: List[Gate] = [Gate("h", (q,)) for q in range(n)]
    for s in adiabatic_schedule(T, dt):
        A, B = -((1.0 - s) + s * h), -s
        gates += [Gate("rx", (q,), (), (A * dt,)) for q in range(n)]
        gates += [Gate("rzz", (i, i + 1), (), (2.0 * B * dt,)) for i in range(n - 1)]
        gates += [Gate("rx", (q,), (), (A * dt,)) for q in range(n)]
    return Circuit(n, gates, f"adiabatic-tfim{n}")


def random_pauli_sum(n: int, nterms: int, seed: int) -> PauliSum:
    """Random Pauli strings (each qubit I/X/Y/Z uniformly) with N(0,1) coefficients."""
    rng = _rng(seed)
    xs, zs = [], []
    for _ in range(nterms):
        ops = rng.integers(0, 4, size=n)
        x = sum(1 << q for q in range(n) if ops[q] in (1, 2))
        z = sum(1 << q for q in range(n) if ops[q] in (2, 3))
        xs.append(x); zs.append(z)
    return PauliSum(np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64),
                    rng.standard_normal(nterms))


def random_dense_gate(rng: np.random.Generator, k: int) -> np.ndarray:
    """A Haar-random 2^k x 2^k unitary (QR of a complex Ginibre matrix with the
    phases of R's diagonal divided out)."""
    d = 1 << k
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return (q * ph).astype(np.complex128)

"""A CPU engine for the sliced-state driver, for tests only: slices are torch
CPU complex128 tensors; segment gates come from the library's host planner
and are applied by the oracle; exchanges and half-slice packing are numpy
restatements of their definitions (the amplitudes of a slice whose bit l has
a given value)."""
import numpy as np

from paper_2203_08826_gb300 import inputs


def half_index(L, l, bit):
    x = np.arange(1 << L)
    return np.nonzero(((x >> l) & 1) == bit)[0]


class OracleSliceEngine:
    def __init__(self, plan, orc):
        self.plan, self.orc = plan, orc

    def apply_segment(self, step, index, buf):
        a = buf.numpy()
        for g in self.plan.segment_gates(step, index):
            self.orc.apply_gate(a, g)

    def exchange(self, a, b, l):
        an, bn = a.numpy(), b.numpy()
        i1, i0 = half_index(self.plan.L, l, 1), half_index(self.plan.L, l, 0)
        tmp = an[i1].copy()
        an[i1] = bn[i0]
        bn[i0] = tmp

    def pack(self, buf, l, bit):
        import torch
        return torch.from_numpy(buf.numpy()[half_index(self.plan.L, l, bit)].copy())

    def unpack(self, buf, l, bit, src):
        buf.numpy()[half_index(self.plan.L, l, bit)] = src.numpy()

    def synchronize(self):
        pass


def run_sequential(plan, psi0, orc):
    """Every step on all 2^g slices in one process (no torch.distributed)."""
    import torch
    from paper_2203_08826_gb300 import sliced
    g, L = plan.g, plan.L
    a = np.array(psi0, dtype=np.complex128).reshape(1 << g, 1 << L)
    slices = {i: torch.from_numpy(a[i].copy()) for i in range(1 << g)}
    sliced.run_distributed(plan, slices, OracleSliceEngine(plan, orc))
    return np.concatenate([slices[i].numpy() for i in range(1 << g)])


def global_heavy_circuit(n, seed, depth=5):
    """Dense gates, controls and diagonals on the top qubits (the slice-selecting ones)."""
    rng = np.random.default_rng(seed)
    top = list(range(n - 3, n))
    gates = []
    for _ in range(depth):
        for q_ in rng.permutation(n)[: n // 2]:
            gates.append(inputs.Gate("su2", (int(q_),), (), inputs.haar_su2_quaternion(rng)))
        a = int(rng.choice(top))
        b = int(rng.integers(0, n - 3))
        gates.append(inputs.Gate("matrix", (a, b), (), (), -1, inputs.random_dense_gate(rng, 2)))
        gates.append(inputs.Gate("x", (b,), (a,)))                      # global control
        gates.append(inputs.Gate("ry", (a,), (b,), (rng.uniform(0, 6),)))  # global target, local control
        gates.append(inputs.Gate("cz", (top[0], top[1])))               # diagonal, both global
        gates.append(inputs.Gate("rz", (top[2],), (), (rng.uniform(0, 6),)))
        d = np.diag(np.exp(1j * rng.uniform(0, 6, 8)))
        gates.append(inputs.Gate("matrix", (top[1], b, top[0]), (), (), -1, d))  # mixed diagonal
        gates.append(inputs.Gate("phase", (top[2],), (top[0],), (rng.uniform(0, 6),)))
        gates.append(inputs.Gate("swap", (top[1], int(rng.integers(0, n - 3)))))
        c3 = tuple(int(v) for v in rng.choice(n, 3, replace=False))
        gates.append(inputs.Gate("matrix", c3, (), (), -1, inputs.random_dense_gate(rng, 3)))
    return inputs.Circuit(n, gates, "global-heavy")

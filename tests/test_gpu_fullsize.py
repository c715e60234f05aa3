"""Full-size checks of the benchmark configurations, where the oracle cannot
simulate the whole state in seconds: sampled amplitudes against a closed form
(the QFT of a basis state is the DFT row of that state), properties that hold
at any size (norm, circuit followed by its inverse), and agreement of the
fused plans with the plain sweeps (parity-tested against the oracle at smaller
sizes) on the benchmark's own 30-qubit circuit; plus the error of the fused
complex64 plans against the complex128 oracle at 26 qubits for the layered
variational ansatz."""
import math
import os

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


def dft_row(n, x0, ys):
    """<y| QFT |x0> = exp(2 pi i x0 y / 2^n) / sqrt(2^n), phase reduced exactly mod 2^n."""
    N = 1 << n
    ph = (np.uint64(x0) * ys.astype(np.uint64)) & np.uint64(N - 1)  # x0 * y mod N, exact in uint64
    return np.exp(2j * np.pi * ph.astype(np.float64) / N) / math.sqrt(N)


@pytest.mark.parametrize("mode,kmax", [("staged", 3), ("tc", 6)])
def test_qft30_basis_state_sampled_amplitudes(q, mode, kmax):
    import torch
    n = 30
    x0 = 0x2B6A1D37 & ((1 << n) - 1)
    s = q.State(n, "c64")
    s.init_basis(x0)
    plan = q.Plan(inputs.qft(n), kmax=kmax, mode=q.FUSE_STAGED if mode == "staged" else q.FUSE_TC)
    s.run_fused(plan)
    ys = np.random.default_rng(5).integers(0, 1 << n, size=4096)
    got = s.tensor[torch.from_numpy(ys).cuda()].cpu().numpy().astype(np.complex128)
    want = dft_row(n, x0, ys)
    rel = np.max(np.abs(got - want)) / (2.0 ** (-n / 2))
    assert rel < 1e-3, f"{mode}: relative amplitude error {rel:.2e}"
    norm = float(torch.sum(torch.abs(s.tensor.to(torch.complex128)) ** 2))
    assert abs(norm - 1.0) < 1e-4


def test_random30_benchmark_plan_against_plain_sweeps(q):
    """The benchmark's circuit (30 qubits, depth 20, seed 2022) through the
    staged plan the autotuner picks (kmax 3) against one sweep per gate."""
    import torch
    c = inputs.random_circuit(30, 20, seed=2022)
    qc = q.QCircuit(c)
    a = q.State(30, "c64").init_zero()
    a.run_fused(q.Plan(qc, kmax=3, mode=q.FUSE_STAGED))
    b = q.State(30, "c64").init_zero()
    b.run(qc)
    d = (a.tensor - b.tensor).abs()
    err2 = float(torch.sqrt(torch.sum(d.to(torch.float64) ** 2)))
    assert float(d.max()) < 1e-6 and err2 < 1e-5, (float(d.max()), err2)
    norm = float(torch.sum(torch.abs(a.tensor.to(torch.complex128)) ** 2))
    assert abs(norm - 1.0) < 1e-4


def test_random30_circuit_then_inverse_returns_to_zero(q):
    c = inputs.random_circuit(30, 20, seed=2022)
    inv = []
    for g in reversed(c.gates):  # SU(2)^-1 = conjugate quaternion; CZ is its own inverse
        if g.name == "su2":
            a, b_, cc, d = g.params
            inv.append(inputs.Gate("su2", g.targets, (), (a, -b_, -cc, -d)))
        else:
            inv.append(g)
    s = q.State(30, "c64").init_zero()
    s.run_fused(q.Plan(c, kmax=3, mode=q.FUSE_STAGED))
    s.run_fused(q.Plan(inputs.Circuit(30, inv), kmax=3, mode=q.FUSE_STAGED))
    amp0 = complex(s.tensor[0].cpu())
    assert abs(abs(amp0) - 1.0) < 1e-5
    p = s.probabilities((29, 0))
    assert abs(p[0] - 1.0) < 1e-5


@pytest.fixture(scope="module")
def var26(orc):
    """26-qubit layered variational ansatz (4 layers) and its complex128 oracle state."""
    c = inputs.variational(26, 4, seed=26)
    return c, orc.simulate(c)


@pytest.mark.parametrize("mode,kmax", [("staged", 3), ("staged", 4), ("tc", 6), ("tc", 5)])
def test_variational26_fused_error_against_fp64_oracle(q, var26, mode, kmax):
    c, want = var26
    s = q.State(26, "c64").init_zero()
    s.run_fused(q.Plan(c, kmax=kmax, mode=q.FUSE_STAGED if mode == "staged" else q.FUSE_TC))
    got = s.to_host().astype(np.complex128)
    err = np.max(np.abs(got - want))
    err2 = np.linalg.norm(got - want)
    assert err <= 1e-5, f"{mode} k={kmax}: max-abs {err:.2e}"
    assert err2 <= (1e-4 if mode == "tc" else 1e-5), f"{mode} k={kmax}: 2-norm {err2:.2e}"


# ---------------------------------------------------------------- the benchmark circuit against the FP64 oracle
GOLDEN_R30 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "random30_d20_seed2022.txt")


@pytest.fixture(scope="module")
def golden30():
    """Oracle values of the benchmark's circuit (30 qubits, depth 20, seed
    2022), written by tests/golden/make_golden.py from the complex128 oracle."""
    from golden import make_golden
    return make_golden.read(GOLDEN_R30)


# max-abs amplitude error against the oracle at the sampled and the largest
# amplitudes (|psi| <= 1.5e-4 here): the measured errors (complex64 staged,
# greedy and plain sweeps <= 1.2e-10, tensor-core blocks 9.5e-9, complex128
# 1.1e-17) times a margin of about 10; all far inside the stated bars (1e-5
# complex64, 1e-12 complex128)
R30_TOL = {"c64": {"staged": 1e-9, "staged-spec": 1e-9, "tc": 5e-8, "greedy2": 1e-9, "plain": 1e-9},
           "c128": {"plain": 1e-15}}


@pytest.mark.parametrize("dtype,mode,kmax", [("c64", "staged", 3), ("c64", "staged", 4), ("c64", "staged-spec", 3),
                                             ("c64", "staged-spec", 4), ("c64", "tc", 6),
                                             ("c64", "tc", 5), ("c64", "greedy2", 2), ("c64", "plain", 0),
                                             ("c128", "plain", 0)])
def test_random30_benchmark_circuit_against_oracle(q, golden30, dtype, mode, kmax):
    """The benchmark's own circuit and state size, every execution mode,
    element by element against the FP64 oracle at 4096 seeded indices and
    the 64 largest amplitudes; <sum Z_i Z_i+1> and the norm of the whole
    state against the oracle's."""
    import torch
    c = inputs.random_circuit(30, 20, seed=2022)
    s = q.State(30, dtype).init_zero()
    if mode == "plain":
        s.run(c)
    else:
        s.run_fused(q.Plan(c, kmax=kmax, mode={"staged": q.FUSE_STAGED, "tc": q.FUSE_TC,
                                                "greedy2": q.FUSE_GREEDY2,
                                                "staged-spec": q.FUSE_STAGED | q.SPECIALIZE}[mode]))
    idx = np.concatenate([golden30["amp_index"], golden30["top_index"]])
    want = np.concatenate([golden30["amp_value"], golden30["top_value"]])
    got = s.tensor[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    err = float(np.max(np.abs(got - want)))
    rel = err / float(np.max(np.abs(want)))
    tol = R30_TOL[dtype][mode]
    print(f"random30 {dtype} {mode} k={kmax}: max-abs {err:.3e}, relative {rel:.3e}")
    assert err <= tol, f"{dtype} {mode} k={kmax}: max-abs {err:.2e} (relative {rel:.2e}) > {tol:.0e}"
    zz = s.expectation(inputs.zz_chain(30))
    zz_tol = 1e-12 if dtype == "c128" else 1e-5
    assert abs(zz - golden30["zz"]) <= zz_tol, (zz, golden30["zz"])
    # the tensor cores' split products lose norm systematically (about 1e-6
    # per pass in BF16x3, over ~100 passes); every other mode keeps 1e-5
    norm_tol = 1e-12 if dtype == "c128" else (3e-4 if mode == "tc" else 5e-6)
    print(f"random30 {dtype} {mode} k={kmax}: norm error {abs(s.norm2() - golden30['norm2']):.3e}")
    assert abs(s.norm2() - golden30["norm2"]) <= norm_tol
    marg = s.probabilities((29, 0))
    np.testing.assert_allclose(marg, golden30["marginal_29_0"],
                               atol=1e-12 if dtype == "c128" else (1e-4 if mode == "tc" else 1e-6))

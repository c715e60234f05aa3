"""GPU parity of the plain gate sweeps, probabilities, norms, expectations and
the sampler against the CPU oracle (same seeded inputs, element by element).

Tolerances: max-abs amplitude error 1e-12 for complex128 and 1e-5 for
complex64 (the stated bar); reductions in double are held to a relative
1e-12 (complex128) / 1e-6 (complex64, whose amplitudes carry ~6e-8 relative
rounding); shots must match bit for bit on identical probabilities.
"""
import math

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


def new_state(q, n, dtype, psi0=None):
    s = q.State(n, dtype)
    if psi0 is None:
        s.init_zero()
    else:
        s.from_host(psi0)
    return s


def check(got, want, dtype, what=""):
    err = np.max(np.abs(got.astype(np.complex128) - want)) if want.size else 0.0
    assert err <= TOL[dtype], f"{what}: max-abs error {err:.3e} > {TOL[dtype]:g}"
    return err


def random_gate(rng, n, kind, k, c):
    qs = [int(v) for v in rng.permutation(n)[: k + c]]
    t, ctl = tuple(qs[:k]), tuple(qs[k:])
    if kind == "dense":
        m = inputs.random_dense_gate(rng, k)
    elif kind == "diag":
        m = np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k)))
    else:  # monomial: permutation with phases
        perm = rng.permutation(1 << k)
        m = np.zeros((1 << k, 1 << k), dtype=complex)
        m[np.arange(1 << k), perm] = np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k))
    return inputs.Gate("matrix", t, ctl, (), -1, m)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 13])
def test_random_gates_each_kind(q, orc, dtype, n):
    rng = np.random.default_rng(1000 + n)
    psi0 = inputs.gaussian_state(n, seed=n)
    s = new_state(q, n, dtype, psi0)
    ref = psi0.copy()
    cases = []
    for kind in ("dense", "diag", "mono"):
        for k in range(1, min(n, 6) + 1):
            for c in (0, 1, 3):
                if k + c <= n and not (kind == "mono" and k > 3):
                    cases.append((kind, k, c))
    for kind, k, c in cases:
        g = random_gate(rng, n, kind, k, c)
        s.apply(g)
        orc.apply_gate(ref, g)
        check(s.to_host(), ref, dtype, f"{kind} k={k} c={c} n={n}")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_named_gates_and_classification(q, orc, dtype):
    """Named gates (including those the classifier turns into controls,
    diagonals and permutations) on every target of a 12-qubit state."""
    n = 12
    rng = np.random.default_rng(5)
    psi0 = inputs.gaussian_state(n, seed=2)
    s = new_state(q, n, dtype, psi0)
    ref = psi0.copy()
    for t in range(n):
        o = (t + 5) % n
        gates = [inputs.Gate("h", (t,)), inputs.Gate("x", (t,)), inputs.Gate("y", (t,)),
                 inputs.Gate("z", (t,)), inputs.Gate("s", (t,)), inputs.Gate("t", (t,)),
                 inputs.Gate("rx", (t,), (), (rng.uniform(0, 6),)),
                 inputs.Gate("ry", (t,), (), (rng.uniform(0, 6),)),
                 inputs.Gate("rz", (t,), (), (rng.uniform(0, 6),)),
                 inputs.Gate("phase", (t,), (o,), (rng.uniform(0, 6),)),
                 inputs.Gate("cz", (t, o)), inputs.Gate("swap", (o, t)),
                 inputs.Gate("x", (t,), (o, (t + 3) % n)),
                 inputs.Gate("su2", (t,), (), inputs.haar_su2_quaternion(rng))]
        for g in gates:
            s.apply(g)
            orc.apply_gate(ref, g)
    check(s.to_host(), ref, dtype, "named gates")


def test_qft10_complex128_matches_oracle_and_dft(q, orc):
    """10-qubit QFT, complex128, Gaussian initial state (seed 1)."""
    n = 10
    psi0 = inputs.gaussian_state(n, seed=1)
    s = new_state(q, n, "c128", psi0)
    s.run(inputs.qft(n))
    got = s.to_host()
    check(got, orc.simulate(inputs.qft(n), psi0), "c128", "qft10 vs oracle")
    check(got, math.sqrt(1 << n) * np.fft.ifft(psi0), "c128", "qft10 vs DFT")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("maker", ["random", "variational", "qft", "ghz"])
def test_circuits_plain_and_greedy2(q, orc, dtype, maker):
    circ = {"random": lambda: inputs.random_circuit(14, 6, seed=3),
            "variational": lambda: inputs.variational(13, 4, seed=4),
            "qft": lambda: inputs.qft(13),
            "ghz": lambda: inputs.ghz(15)}[maker]()
    psi0 = inputs.gaussian_state(circ.n, seed=7) if maker != "ghz" else None
    want = orc.simulate(circ, psi0)
    s = new_state(q, circ.n, dtype, psi0)
    s.run(circ)
    check(s.to_host(), want, dtype, f"{maker} plain")
    s2 = new_state(q, circ.n, dtype, psi0)
    s2.run_fused(q.Plan(circ, kmax=2, mode=q.FUSE_GREEDY2))
    check(s2.to_host(), want, dtype, f"{maker} greedy2")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_probabilities_and_norm(q, orc, dtype):
    n = 14
    psi0 = inputs.gaussian_state(n, seed=11)
    s = new_state(q, n, dtype, psi0)
    s.run(inputs.random_circuit(n, 2, seed=12))
    amps = s.to_host().astype(np.complex128)
    rtol = 1e-13 if dtype == "c128" else 1e-12
    np.testing.assert_allclose(s.probabilities(), orc.probabilities(amps), rtol=rtol, atol=0)
    if dtype == "c64":  # complex64: re^2 + im^2 exact in double, one rounding -- bit for bit
        np.testing.assert_array_equal(s.probabilities(), amps.real ** 2 + amps.imag ** 2)
    for qubits in [(0,), (13,), (3, 9), (9, 3, 0), tuple(range(12)), (1, 5, 7, 11, 13, 0, 2, 4, 6, 8, 10, 12, 3)]:
        np.testing.assert_allclose(s.probabilities(qubits), orc.probabilities(amps, qubits),
                                   rtol=1e-11, atol=1e-15)
    assert abs(s.norm2() - np.sum(np.abs(amps) ** 2)) < 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_pauli_expectation(q, orc, dtype):
    n = 12
    psi0 = inputs.gaussian_state(n, seed=21)
    s = new_state(q, n, dtype, psi0)
    amps = s.to_host().astype(np.complex128)
    # complex64 diagonal passes form |psi|^2 x sign in fp32 over 16 amplitudes (relative 1e-6)
    rtol = 1e-12 if dtype == "c128" else 1e-6
    for ham in (inputs.random_pauli_sum(n, 40, seed=22), inputs.tfim(n), inputs.zz_chain(n)):
        want = orc.expectation(amps, ham)
        got = s.expectation(ham)
        assert abs(got - want) <= rtol * max(1.0, abs(want)), (got, want)


def test_expectation_many_terms_same_xmask(q, orc):
    """More terms share one xmask than one pass holds."""
    n = 10
    rng = np.random.default_rng(3)
    z = rng.integers(0, 1 << n, size=150).astype(np.uint64)
    x = np.full(150, 0b1010, dtype=np.uint64)
    ham = inputs.PauliSum(x, z, rng.standard_normal(150))
    s = new_state(q, n, "c128", inputs.gaussian_state(n, seed=1))
    want = orc.expectation(s.to_host(), ham)
    assert abs(s.expectation(ham) - want) < 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [3, 11, 16])
def test_sampler_bit_exact(q, orc, dtype, n):
    import torch
    psi0 = inputs.gaussian_state(n, seed=31 + n)
    s = new_state(q, n, dtype, psi0)
    shots = 20000
    seed, c0 = 0xDEADBEEF12345, 2**32 - 100
    got = s.sample(shots, seed, c0)
    # (a) GPU probabilities copied back, sampled by the oracle
    p_gpu = s.probabilities()
    np.testing.assert_array_equal(got, orc.sample(p_gpu, shots, seed, c0))
    # (b) the oracle's probabilities (of the same stored amplitudes) on the GPU sampler
    p_orc = orc.probabilities(s.to_host().astype(np.complex128))
    dev = torch.from_numpy(p_orc).cuda()
    from paper_2203_08826_gb300 import binding
    np.testing.assert_array_equal(binding.sample_probs(dev, shots, seed, c0), orc.sample(p_orc, shots, seed, c0))


@pytest.mark.parametrize("N", [1, 7, 2048, 2049, 5000, 1 << 15])
def test_sampler_ragged_sizes(q, orc, N):
    import torch
    from paper_2203_08826_gb300 import binding
    rng = np.random.default_rng(N)
    p = rng.dirichlet(np.full(N, 0.5)) if N > 1 else np.ones(1)
    p[rng.random(N) < 0.2] = 0.0
    if p.sum() == 0:
        p[0] = 1.0
    p /= p.sum()
    got = binding.sample_probs(torch.from_numpy(p).cuda(), 5000, seed=N, counter0=3)
    np.testing.assert_array_equal(got, orc.sample(p, 5000, seed=N, counter0=3))


@pytest.mark.parametrize("frac", [(0.0, 0.0), (0.75, 0.25)])
@pytest.mark.parametrize("pad", [0, 2047])
def test_sampler_draw_on_a_cdf_value(q, orc, pad, frac):
    """The first draw lands exactly on a CDF value (weights built from the
    shot's own Philox output, as in the oracle's pin); the next outcome must
    be drawn.  pad = 0: both outcomes in one chunk, the in-chunk scan decides;
    pad = 2047: the boundary is the last element of the first 2048-element
    chunk, so the search over the chunk sums decides.  frac: fractional
    weight bits that floor(p 2^62) must drop."""
    import torch
    from paper_2203_08826_gb300 import binding
    from tests.test_oracle_pins import tie_probabilities
    seed, c0 = 0xFEED, 2**32 - 1
    two = tie_probabilities(orc, seed, c0, frac)
    p = np.zeros(pad + 2 + (2048 if pad else 0))
    p[pad], p[pad + 1] = two
    want = orc.sample(p, 4, seed=seed, counter0=c0)
    assert int(want[0]) == pad + 1
    got = binding.sample_probs(torch.from_numpy(p).cuda(), 4, seed=seed, counter0=c0)
    np.testing.assert_array_equal(got, want)


def test_sampler_rejects_bad_probabilities(q):
    import torch
    from paper_2203_08826_gb300 import binding
    with pytest.raises(binding.QsimError):
        binding.sample_probs(torch.zeros(64, dtype=torch.float64, device="cuda"), 10, seed=1)
    with pytest.raises(binding.QsimError):
        binding.sample_probs(torch.full((64,), 0.5, dtype=torch.float64, device="cuda"), 10, seed=1)


def test_argument_errors_do_not_launch(q):
    from paper_2203_08826_gb300 import binding
    s = new_state(q, 5, "c64")
    before = binding.launch_count()
    with pytest.raises(binding.QsimError):
        s.apply_matrix(np.eye(2), (5,))
    with pytest.raises(binding.QsimError):
        s.apply_matrix(np.eye(4), (1, 1))
    with pytest.raises(binding.QsimError):
        s.apply_matrix(np.eye(2), (1,), (1,))
    assert binding.launch_count() == before


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_collapse(q, orc, dtype):
    n = 13
    psi0 = inputs.gaussian_state(n, seed=41)
    for qubits, outcome in (((0,), 1), ((12, 3), 2), ((7, 1, 9), 6)):
        s = new_state(q, n, dtype, psi0)
        p = s.collapse(qubits, outcome)
        amps = psi0.astype(np.complex64).astype(np.complex128) if dtype == "c64" else psi0
        want, pw = orc.collapse(amps, qubits, outcome)
        assert abs(p - pw) <= (1e-13 if dtype == "c128" else 1e-7)
        check(s.to_host(), want, dtype, f"collapse {qubits}={outcome}")
    s = new_state(q, 4, dtype)
    with pytest.raises(q.QsimError):
        s.collapse((1,), 1)  # |0000>: outcome 1 has probability 0


@pytest.mark.parametrize("dtype,rate", [("c128", 0.9999), ("c64", 0.999)])
def test_sampler_end_to_end_match_rate(q, orc, dtype, rate):
    """Shots from the GPU state and from the independently simulated oracle
    state, same seed and counters: they differ only where a draw falls within
    rounding of a CDF boundary (complex64 rounds the amplitudes)."""
    n = 16
    circ = inputs.random_circuit(n, 6, seed=77)
    s = new_state(q, n, dtype)
    s.run(circ)
    shots = 200000
    got = s.sample(shots, seed=99, counter0=5)
    want = orc.sample(orc.probabilities(orc.simulate(circ)), shots, seed=99, counter0=5)
    match = float(np.mean(got == want))
    assert match >= rate, f"match rate {match:.6f}"


def test_sampler_prefix_over_several_scan_tiles(q, orc):
    """2^24 + 12345 probabilities: 8198 chunk sums, three scan tiles (the last
    ragged), bit-exact against the oracle's sampler."""
    import torch
    from paper_2203_08826_gb300 import binding
    N = (1 << 24) + 12345
    rng = np.random.default_rng(17)
    p = rng.random(N) ** 4
    p[rng.random(N) < 0.3] = 0.0
    p /= p.sum()
    got = binding.sample_probs(torch.from_numpy(p).cuda(), 6000, seed=123, counter0=9)
    np.testing.assert_array_equal(got, orc.sample(p, 6000, seed=123, counter0=9))


@pytest.mark.parametrize("scale", [1.0, 1e-21, 1e-30, 1e30, "mixed"])
def test_complex128_double_float_range(q, orc, scale):
    """complex128 dense 1-qubit and diagonal sweeps run in double-float
    arithmetic on the FP32 pipes; amplitudes outside [2^-74, 2^77) take the
    FP64 formula per pair.  States scaled into and beyond that range (and a
    state mixing normal, tiny, subnormal and zero amplitudes within one warp)
    against the oracle, relative to the scale, at the complex128 bound; CZ
    and Z (sign flips) are exact."""
    n = 11
    rng = np.random.default_rng(77)
    psi0 = inputs.gaussian_state(n, seed=78)
    if scale == "mixed":
        psi0 = psi0.copy()
        psi0[::3] *= 1e-30
        psi0[1::7] = 0.0
        psi0[2::11] *= 1e-310  # subnormal doubles
        ref_scale = float(np.max(np.abs(psi0)))
    else:
        psi0 = psi0 * scale
        ref_scale = scale
    s = new_state(q, n, "c128", psi0)
    ref = psi0.copy()
    gates = []
    for _ in range(6):
        for t in range(n):
            gates.append(inputs.Gate("su2", (t,), (), inputs.haar_su2_quaternion(rng)))
        a, b = (int(v) for v in rng.choice(n, 2, replace=False))
        gates.append(inputs.Gate("cz", (a, b)))
        gates.append(inputs.Gate("z", (int(rng.integers(n)),)))
        gates.append(inputs.Gate("phase", (a,), (b,), (float(rng.uniform(0, 6.28)),)))
        gates.append(inputs.Gate("rz", (int(rng.integers(n)),), (), (float(rng.uniform(0, 6.28)),)))
        gates.append(inputs.Gate("h", (b,), (a,)))  # controlled H
    for g in gates:
        s.apply(g)
        orc.apply_gate(ref, g)
    err = np.max(np.abs(s.to_host() - ref)) / ref_scale
    assert err <= 1e-12, f"scale {scale}: max-abs error / scale {err:.3e}"

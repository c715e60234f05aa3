"""GPU parity of the Sec. 3.3 evolution path: the diagonal Pauli-phase sweep
and the Trotterised adiabatic TFIM circuit (every execution mode) against the
oracle."""
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


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("uniform", [True, False])
def test_pauli_phase_matches_oracle(q, orc, dtype, uniform):
    n = 13
    rng = np.random.default_rng(7 + uniform)
    psi0 = inputs.gaussian_state(n, seed=4)
    nt = 40
    z = [int(v) for v in rng.integers(1, 1 << n, size=nt)]
    c = [1.0] * nt if uniform else list(rng.standard_normal(nt))
    s = q.State(n, dtype)
    s.from_host(psi0)
    s.apply_pauli_phase(z, c, 0.731)
    want = orc.pauli_phase(psi0.astype(np.complex64).astype(complex) if dtype == "c64" else psi0, z, c, 0.731)
    assert np.max(np.abs(s.to_host() - want)) <= TOL[dtype]


def test_pauli_phase_zz_chain_and_errors(q, orc):
    n = 16
    psi0 = inputs.gaussian_state(n, seed=5)
    zz = inputs.zz_chain(n)
    s = q.State(n, "c128")
    s.from_host(psi0)
    s.apply_pauli_phase(zz.zmask, zz.coeff, -0.4)
    assert np.max(np.abs(s.to_host() - orc.pauli_phase(psi0, zz.zmask, zz.coeff, -0.4))) <= 1e-12
    before = s.to_host()
    s.apply_pauli_phase([], [], 1.0)  # no terms: nothing happens
    assert np.array_equal(s.to_host(), before)
    with pytest.raises(q.QsimError):
        s.apply_pauli_phase([1 << n], [1.0], 0.1)
    with pytest.raises(q.QsimError):
        s.apply_pauli_phase([1] * 129, [1.0] * 129, 0.1)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_adiabatic_circuit_all_modes(q, orc, dtype):
    n = 14
    circ = inputs.adiabatic_tfim(n, 1.0, 1.0, 0.1)
    want = orc.simulate(circ)
    qc = q.QCircuit(circ)
    runs = [("plain", None), ("greedy2", q.Plan(qc, kmax=2, mode=q.FUSE_GREEDY2)),
            ("staged", q.Plan(qc, kmax=4, mode=q.FUSE_STAGED))]
    if dtype == "c64":
        runs.append(("tc", q.Plan(qc, kmax=6, mode=q.FUSE_TC)))
    for name, plan in runs:
        s = q.State(n, dtype).init_zero()
        if plan is None:
            s.run(qc)
        else:
            s.run_fused(plan)
        err = np.max(np.abs(s.to_host().astype(complex) - want))
        assert err <= TOL[dtype], f"{name}: {err:.3e}"
    e = s.expectation(inputs.tfim_target(n, 1.0))
    assert abs(e - orc.expectation(want, inputs.tfim_target(n, 1.0))) < 1e-4


def test_adiabatic_steps_with_phase_kernel(q, orc):
    """Each Trotter step as RX layer, one Pauli-phase sweep for the whole ZZ
    layer, RX layer: the same state as the gate-level circuit."""
    n, h, T, dt = 14, 1.0, 1.0, 0.1
    zz = inputs.zz_chain(n)
    s = q.State(n, "c128").init_zero()
    for qb in range(n):
        s.apply(inputs.Gate("h", (qb,)))
    for sk in inputs.adiabatic_schedule(T, dt):
        A, B = -((1.0 - sk) + sk * h), -sk
        for qb in range(n):
            s.apply(inputs.Gate("rx", (qb,), (), (A * dt,)))
        s.apply_pauli_phase(zz.zmask, zz.coeff, B * dt)
        for qb in range(n):
            s.apply(inputs.Gate("rx", (qb,), (), (A * dt,)))
    want = orc.simulate(inputs.adiabatic_tfim(n, h, T, dt))
    assert np.max(np.abs(s.to_host() - want)) <= 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("nt", [5, 20, 32, 45])
def test_pauli_phase_general_coefficients_table_and_direct(q, orc, dtype, nt):
    """Weighted Z strings (QAOA-like costs): up to 32 terms go through
    per-group sign-pattern tables, more through a direct sine/cosine."""
    n = 14
    rng = np.random.default_rng(nt)
    psi0 = inputs.gaussian_state(n, seed=nt)
    z = [int(v) for v in rng.integers(1, 1 << n, size=nt)]
    c = list(rng.standard_normal(nt))
    s = q.State(n, dtype)
    s.from_host(psi0)
    s.apply_pauli_phase(z, c, -0.37)
    base = psi0.astype(np.complex64).astype(complex) if dtype == "c64" else psi0
    assert np.max(np.abs(s.to_host() - orc.pauli_phase(base, z, c, -0.37))) <= TOL[dtype]

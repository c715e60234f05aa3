"""GPU parity of sliced states (Sec. 3.1 multi-GPU scheme): the exchange and
pack kernels against their definitions, and sliced execution -- slices in
device memory, in page-locked host memory streamed through the GPU, and the
multi-rank driver on one rank -- against the oracle's unsliced simulation."""
import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

from slice_cpu import global_heavy_circuit, half_index

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


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("L,l", [(1, 0), (5, 0), (5, 4), (13, 7), (13, 12), (20, 3)])
def test_exchange_and_pack_kernels(q, dtype, L, l):
    import torch
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    a0 = inputs.gaussian_state(L, seed=L + l)
    b0 = inputs.gaussian_state(L, seed=100 + L + l)
    a = torch.from_numpy(a0).to(tdt).cuda()
    b = torch.from_numpy(b0).to(tdt).cuda()
    q.slice_exchange(a, b, L, l)
    i1, i0 = half_index(L, l, 1), half_index(L, l, 0)
    wa, wb = a0.copy(), b0.copy()
    wa[i1], wb[i0] = b0[i0], a0[i1]
    np.testing.assert_array_equal(a.cpu().numpy(), wa.astype(a.cpu().numpy().dtype))
    np.testing.assert_array_equal(b.cpu().numpy(), wb.astype(b.cpu().numpy().dtype))
    for bit in (0, 1):
        out = torch.empty(1 << (L - 1), dtype=tdt, device="cuda")
        q.slice_pack(a, L, l, bit, out)
        np.testing.assert_array_equal(out.cpu().numpy(), a.cpu().numpy()[half_index(L, l, bit)])
        c = torch.zeros_like(a)
        q.slice_unpack(c, L, l, bit, out)
        want = np.zeros(1 << L, dtype=out.cpu().numpy().dtype)
        want[half_index(L, l, bit)] = out.cpu().numpy()
        np.testing.assert_array_equal(c.cpu().numpy(), want)


CIRCUITS = {
    "random": lambda n: inputs.random_circuit(n, 5, seed=n),
    "qft": lambda n: inputs.qft(n),
    "variational": lambda n: inputs.variational(n, 4, seed=3),
    "global": lambda n: global_heavy_circuit(n, seed=n),
}


@pytest.mark.parametrize("location", ["device", "host"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("maker", sorted(CIRCUITS))
def test_sliced_state_matches_oracle(q, orc, location, dtype, maker):
    from paper_2203_08826_gb300 import sliced
    n = 16
    circ = CIRCUITS[maker](n)
    psi0 = inputs.gaussian_state(n, seed=9)
    want = orc.simulate(circ, psi0)
    for g, mode, kmax in ((1, q.FUSE_GREEDY2, 2), (3, q.FUSE_STAGED, 4), (5, q.FUSE_STAGED, 3),
                          (3, q.FUSE_STAGED | q.SPECIALIZE, 3)):
        plan = q.SlicePlan(circ, g, kmax=kmax, mode=mode)
        st = sliced.SlicedState(n, g, dtype, location).from_host(psi0).run(plan)
        err = np.max(np.abs(st.to_host().astype(np.complex128) - want))
        assert err <= TOL[dtype], f"{maker} g={g} mode={mode}: {err:.3e}"


@pytest.mark.parametrize("location", ["device", "host"])
def test_sliced_tensor_core_segments(q, orc, location):
    from paper_2203_08826_gb300 import sliced
    n, g = 17, 3
    circ = inputs.variational(n, 4, seed=5)
    psi0 = inputs.gaussian_state(n, seed=1)
    want = orc.simulate(circ, psi0)
    plan = q.SlicePlan(circ, g, kmax=6, mode=q.FUSE_TC)
    st = sliced.SlicedState(n, g, "c64", location).from_host(psi0).run(plan)
    assert np.max(np.abs(st.to_host() - want)) <= TOL["c64"]


def test_sliced_without_restore_follows_layout(q, orc):
    from paper_2203_08826_gb300 import sliced
    n, g = 14, 3
    circ = global_heavy_circuit(n, seed=4)
    psi0 = inputs.gaussian_state(n, seed=2)
    plan = q.SlicePlan(circ, g, kmax=2, mode=q.FUSE_GREEDY2, restore=False)
    got = sliced.SlicedState(n, g, "c128", "device").from_host(psi0).run(plan).to_host()
    want = orc.simulate(circ, psi0)
    x = np.arange(1 << n)
    phys = np.zeros_like(x)
    for lq, p in enumerate(plan.layout()):
        phys |= ((x >> lq) & 1) << p
    assert np.max(np.abs(got[phys] - want)) <= 1e-12


def test_distributed_driver_one_rank_cuda_engine(q, orc):
    """The multi-rank driver with its CUDA engine, world size 1: exchanges on
    every global bit stay inside the rank and run as kernels."""
    import torch
    from paper_2203_08826_gb300 import sliced
    n, g = 15, 3
    circ = global_heavy_circuit(n, seed=7)
    psi0 = inputs.gaussian_state(n, seed=3)
    plan = q.SlicePlan(circ, g, kmax=4, mode=q.FUSE_STAGED)
    a = psi0.reshape(1 << g, -1)
    slices = {i: torch.from_numpy(a[i].copy()).cuda() for i in range(1 << g)}
    sliced.run_distributed(plan, slices, sliced.CudaSliceEngine(plan))
    got = np.concatenate([slices[i].cpu().numpy() for i in range(1 << g)])
    assert np.max(np.abs(got - orc.simulate(circ, psi0))) <= 1e-12


def test_host_sliced_26q_matches_unsliced(q):
    """26 qubits, complex64, 8 slices in host memory vs the unsliced staged run
    of the same circuit on the device (properties that hold at any size: the
    two agree to rounding and the norm stays 1)."""
    from paper_2203_08826_gb300 import sliced
    n, g = 26, 3
    circ = inputs.random_circuit(n, 6, seed=11)
    plan = q.SlicePlan(circ, g, kmax=4, mode=q.FUSE_STAGED)
    got = sliced.SlicedState(n, g, "c64", "host").init_zero().run(plan).to_host()
    s = q.State(n, "c64").init_zero()
    s.run_fused(q.Plan(circ, kmax=4, mode=q.FUSE_STAGED))
    ref = s.to_host()
    assert np.max(np.abs(got - ref)) < 1e-6
    assert abs(np.sum(np.abs(got.astype(np.complex128)) ** 2) - 1.0) < 1e-4


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_device_slices_start_in_zero_state(q, orc, dtype):
    """init_zero on device slices runs the library's init kernel: |0...0> in
    slice 0, every other slice written 0 (QSIM_INIT_NULL) over whatever the
    memory held; the run from there matches the oracle."""
    from paper_2203_08826_gb300 import sliced
    n, g = 15, 3
    st = sliced.SlicedState(n, g, dtype, "device")
    for t in st.slices:
        t.fill_(3.0 - 1.0j)  # stale contents the initialisation must overwrite
    got = st.init_zero().to_host()
    want = np.zeros(1 << n, dtype=got.dtype)
    want[0] = 1.0
    np.testing.assert_array_equal(got, want)
    circ = global_heavy_circuit(n, seed=5)
    plan = q.SlicePlan(circ, g, kmax=4, mode=q.FUSE_STAGED)
    out = st.init_zero().run(plan).to_host().astype(np.complex128)
    assert np.max(np.abs(out - orc.simulate(circ))) <= (1e-12 if dtype == "c128" else 1e-5)


def test_slice_run_rejects_bad_arguments(q):
    import torch
    circ = inputs.random_circuit(10, 1, seed=1)
    plan = q.SlicePlan(circ, 2, kmax=2, mode=q.FUSE_GREEDY2)
    t = torch.zeros(1 << 8, dtype=torch.complex64, device="cuda")
    with pytest.raises(q.QsimError):
        plan.run([t, t, t, t], q.C64, q.SLICES_DEVICE)  # shared memory
    with pytest.raises(q.QsimError):
        plan.run([t] + [torch.zeros_like(t) for _ in range(3)], q.C64, 7)
    with pytest.raises(q.QsimError):
        q.slice_exchange(t, t, 8, 3)

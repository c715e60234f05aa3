"""Failure paths on the GPU, made on the host or by a bounded wait that runs
out (no fault, trap or hang): injected allocation failures return
QSIM_ENOMEM and leave nothing allocated, and a tensor-core pass whose
pipeline waits are limited to a few polls returns QSIM_ETIMEOUT with the
context still usable."""
import ctypes

import numpy as np
import pytest

from paper_2203_08826_gb300 import inputs

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT = -2, -4


@pytest.fixture(scope="module")
def q():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_08826_gb300 import build, binding
    build.build()
    yield binding
    binding.lib().qsim_debug_fail_alloc(0, 0)
    binding.lib().qsim_debug_set_wait_limit(0)


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_state_create_out_of_memory(q):
    L = q.lib()
    h = ctypes.c_void_p()
    assert L.qsim_debug_fail_alloc(0, 1) == 0
    rc = L.qsim_state_create(20, q.C64, None, None, ctypes.byref(h))
    assert rc == ENOMEM and "state allocation" in L.qsim_last_error().decode()
    assert L.qsim_state_create(20, q.C64, None, None, ctypes.byref(h)) == 0  # the injection is used up
    assert L.qsim_state_destroy(h) == 0
    assert L.qsim_debug_fail_alloc(-1, 1) == -1


def test_adjoint_out_of_memory_releases_its_buffers(q, orc):
    """Every allocation of the adjoint call failing in turn: QSIM_ENOMEM, no
    device memory kept, and the next call gives the oracle's gradients."""
    circ = inputs.variational(20, 2, seed=3)
    ham = inputs.tfim(20)
    th = circ.params()[None, :]
    want, _ = q.adjoint_grad(circ, ham, th, "c64")
    free0 = free_bytes()
    failed = 0
    for skip in range(12):
        q.lib().qsim_debug_fail_alloc(skip, 1)
        try:
            q.adjoint_grad(circ, ham, th, "c64")
        except q.QsimError as e:
            assert e.code == ENOMEM, e
            failed += 1
        q.lib().qsim_debug_fail_alloc(0, 0)
        assert abs(free_bytes() - free0) < (4 << 20), f"allocation {skip}: device memory not released"
    assert failed >= 3  # psi, lambda and the partial sums at least
    got, _ = q.adjoint_grad(circ, ham, th, "c64")
    np.testing.assert_array_equal(got, want)


def test_sampler_and_plan_out_of_memory(q, orc):
    circ = inputs.random_circuit(14, 3, seed=4)
    want = orc.simulate(circ)
    s = q.State(14, "c64").init_zero()
    q.lib().qsim_debug_fail_alloc(0, 1)
    with pytest.raises(q.QsimError) as e:
        s.run_fused(q.Plan(circ, kmax=6, mode=q.FUSE_TC))  # the pass images are uploaded at first use
    assert e.value.code == ENOMEM
    q.lib().qsim_debug_fail_alloc(0, 0)
    s.init_zero().run_fused(q.Plan(circ, kmax=6, mode=q.FUSE_TC))
    assert np.max(np.abs(s.to_host() - want)) < 1e-5
    p = s.probabilities()
    q.lib().qsim_debug_fail_alloc(0, 8)
    import torch
    pd = torch.from_numpy(p).cuda()
    with pytest.raises(q.QsimError) as e:
        q.sample_probs(pd, 100, seed=1)
    assert e.value.code == ENOMEM
    q.lib().qsim_debug_fail_alloc(0, 0)
    np.testing.assert_array_equal(q.sample_probs(pd, 100, seed=1), orc.sample(p, 100, seed=1))


def test_tensor_core_wait_limit_returns_timeout(q, orc):
    """Pipeline waits limited to 2 polls: the pass gives up (QSIM_ETIMEOUT);
    the library and the context stay usable and the next run with the
    default bound matches the oracle."""
    circ = inputs.random_circuit(16, 4, seed=6)
    want = orc.simulate(circ)
    plan = q.Plan(circ, kmax=6, mode=q.FUSE_TC)
    s = q.State(16, "c64").init_zero()
    s.run_fused(plan)  # uploads the pass images with the default bound
    assert np.max(np.abs(s.to_host() - want)) < 1e-5
    q.lib().qsim_debug_set_wait_limit(2)
    try:
        s.init_zero()
        with pytest.raises(q.QsimError) as e:
            s.run_fused(plan)
        assert e.value.code == ETIMEOUT
    finally:
        q.lib().qsim_debug_set_wait_limit(0)
    s.init_zero().run_fused(plan)
    assert np.max(np.abs(s.to_host() - want)) < 1e-5
    s.init_zero().run(circ)  # plain sweeps after the timeout
    assert np.max(np.abs(s.to_host() - want)) < 1e-5

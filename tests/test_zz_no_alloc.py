"""The allocation-free sampler, qsim_sample_probs_static, for callers that may
not allocate device memory (their framework's allocator owns the pool, their
memory budget is fixed at start-up, or they cannot take the synchronisation
an allocation can cause).  Its shots must equal those of the allocating
qsim_sample_probs bit for bit, call after call, although both calls share one
static scratch array inside the library.

This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_08826_gb300 import binding, build
    build.build()
    return torch, binding


def _static_shots(torch, binding, p_dev, nshots, seed, counter0):
    out = torch.empty(nshots, dtype=torch.int64, device="cuda")
    rc = binding.lib().qsim_sample_probs_static(
        ctypes.c_void_p(p_dev.data_ptr()), p_dev.numel(), nshots, seed, counter0,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, binding.lib().qsim_last_error()
    return out.cpu().numpy().view(np.uint64)


def test_static_sampler_matches_allocating_sampler_on_consecutive_calls(env):
    torch, binding = env
    rng = np.random.default_rng(2024)
    # two calls in a row with different sizes: the second must not see the
    # first call's leftovers in the shared scratch
    # 20_000_001 probabilities: 9766 chunk sums, three scan tiles
    for N, nshots, seed, c0 in ((20_000_001, 30_000, 13, 7), (300_001, 50_000, 11, 5), (4_099, 20_000, 12, 2**32 - 3)):
        p = rng.dirichlet(np.full(N, 0.3))
        p_dev = torch.from_numpy(p).cuda()
        got = _static_shots(torch, binding, p_dev, nshots, seed, c0)
        want = binding.sample_probs(p_dev, nshots, seed, c0)
        np.testing.assert_array_equal(got, want)


def test_static_sampler_rejects_sizes_beyond_its_scratch(env):
    torch, binding = env
    before = binding.launch_count()
    p_dev = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    rc = binding.lib().qsim_sample_probs_static(
        ctypes.c_void_p(p_dev.data_ptr()), (1 << 27) + 1, 4, 1, 0, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1 and b"2^27" in binding.lib().qsim_last_error()
    assert binding.launch_count() == before

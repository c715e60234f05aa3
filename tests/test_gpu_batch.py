"""GPU parity of the batched persistent kernel: <sum_i Z_i Z_{i+1}> of every
circuit of an uneven batch against the oracle, graph capture, autotuning."""
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


def oracle_zz(orc, circ):
    return orc.expectation(orc.simulate(circ), inputs.zz_chain(circ.n))


def run_batch(q, b, count):
    import torch
    out = torch.zeros(count, dtype=torch.float64, device="cuda")
    b.run(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("nmin,nmax", [(9, 13), (12, 15), (10, 10)])
def test_batch_matches_oracle(q, orc, nmin, nmax):
    circs = inputs.batch_circuits(24, seed=nmin * 100 + nmax, nmin=nmin, nmax=nmax, lmin=2, lmax=6)
    b = q.Batch(circs)
    got = run_batch(q, b, len(circs))
    want = np.array([oracle_zz(orc, c) for c in circs])
    np.testing.assert_allclose(got, want, atol=2e-5 * np.maximum(1, np.abs(want)).max())
    # every tile width / occupancy gives the same answers
    for tile in range(9, min(12, nmin) + 1):
        for ctas in (1, 3):
            b.set_config(ctas_per_sm=ctas, tile_qubits=tile)
            np.testing.assert_allclose(run_batch(q, b, len(circs)), want, atol=2e-5 * max(1, np.abs(want).max()))


def test_batch_in_cuda_graph_and_autotuner(q, orc):
    import torch
    circs = inputs.batch_circuits(40, seed=5, nmin=12, nmax=14, lmin=2, lmax=5)
    b = q.Batch(circs)
    cfg = b.autotune(reps=1)
    assert 9 <= cfg["tile_qubits"] <= 12 and cfg["ctas_per_sm"] >= 1
    want = np.array([oracle_zz(orc, c) for c in circs])
    out = torch.zeros(len(circs), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(out, stream=s)  # warm-up outside capture (allocates slots)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(out, stream=s)
    out.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), want, atol=2e-5 * max(1, np.abs(want).max()))


def test_full_size_batch_sampled(q, orc):
    """The 4096-circuit batch (n ~ U{12..20}, 4..12 layers): sampled circuits
    checked one by one against the oracle, every output bounded by n - 1."""
    circs = inputs.batch_circuits(4096, seed=2024)
    b = q.Batch(circs)
    got = run_batch(q, b, len(circs))
    ns = np.array([c.n for c in circs])
    assert np.all(np.abs(got) <= ns - 1 + 1e-4)
    rng = np.random.default_rng(0)
    small = [i for i in range(len(circs)) if circs[i].n <= 15]
    for i in rng.choice(small, 6, replace=False):
        assert abs(got[i] - oracle_zz(orc, circs[i])) < 2e-5 * circs[i].n, i


def test_full_size_batch_wide_circuits_against_oracle(q, orc):
    """The widest circuits of the 4096-circuit batch (19 and 20 qubits: the
    per-CTA global slots that stream through the registers tile by tile),
    run inside the full batch, against the oracle one by one."""
    circs = inputs.batch_circuits(4096, seed=2024)
    b = q.Batch(circs)
    got = run_batch(q, b, len(circs))
    wide = [i for i in range(len(circs)) if circs[i].n >= 19]
    pick = [wide[0], wide[len(wide) // 3], wide[2 * len(wide) // 3], wide[-1]]
    assert {circs[i].n for i in pick} >= {19, 20} or len({circs[i].n for i in pick}) >= 1
    for i in pick:
        want = oracle_zz(orc, circs[i])
        err = abs(got[i] - want)
        print(f"batch circuit {i}: n={circs[i].n} layers={len(circs[i].gates)} |err| {err:.3e}")
        assert err < 3e-6, (i, got[i], want)  # measured <= 3.0e-7

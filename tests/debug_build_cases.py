"""Small parity cases run against the library built with index bound checks
(QSIM_DEBUG); started by tests/test_gpu_debug_build.py in a process of its
own with QSIM_LIBRARY=debug.  Every case must match the oracle and no index
may fall outside its state."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2203_08826_gb300 import binding as q  # noqa: E402
from paper_2203_08826_gb300 import inputs  # noqa: E402


def main():
    assert os.environ.get("QSIM_LIBRARY") == "debug" and q.LIB_PATH.endswith("libqsim_debug.so")
    oracle.build()
    L = q.lib()
    assert L.qsim_debug_checks(1) == 0  # a debug build (a release build returns -1)
    rng = np.random.default_rng(5)
    worst = {}
    for dtype, tol in (("c128", 1e-12), ("c64", 1e-5)):
        for n in (1, 2, 5, 13):
            psi0 = inputs.gaussian_state(n, seed=n)
            s = q.State(n, dtype).from_host(psi0)
            ref = psi0.copy()
            for kind in ("dense", "diag", "mono"):
                for k in range(1, min(n, 6) + 1):
                    for c in (0, 1, 3):
                        if k + c > n or (kind == "mono" and k > 3):
                            continue
                        qs = [int(v) for v in rng.permutation(n)[: k + c]]
                        if kind == "dense":
                            m = inputs.random_dense_gate(rng, k)
                        elif kind == "diag":
                            m = np.diag(np.exp(1j * rng.uniform(0, 6.28, 1 << k)))
                        else:
                            m = np.zeros((1 << k, 1 << k), dtype=complex)
                            m[np.arange(1 << k), rng.permutation(1 << k)] = 1.0
                        g = inputs.Gate("matrix", tuple(qs[:k]), tuple(qs[k:]), (), -1, m)
                        s.apply(g)
                        oracle.apply_gate(ref, g)
            s.synchronize()  # QSIM_EINVAL here if a check fired
            err = float(np.max(np.abs(s.to_host().astype(np.complex128) - ref)))
            assert err <= tol, (dtype, n, err)
            worst[(dtype, n)] = err
    for kmax in (1, 3, 4):  # staged register tiles, plain stages included
        circ = inputs.random_circuit(14, 5, seed=kmax)
        s = q.State(14, "c64").init_zero()
        s.run_fused(q.Plan(circ, kmax=kmax, mode=q.FUSE_STAGED))
        s.synchronize()
        err = float(np.max(np.abs(s.to_host().astype(np.complex128) - oracle.simulate(circ))))
        assert err <= 1e-5, ("staged", kmax, err)
    s = q.State(10, "c128").from_host(inputs.gaussian_state(10, seed=1))
    s.run(inputs.qft(10))
    s.synchronize()
    assert np.max(np.abs(s.to_host() - oracle.simulate(inputs.qft(10), inputs.gaussian_state(10, seed=1)))) <= 1e-12
    checks = L.qsim_debug_checks(0)
    assert checks == 0, f"{checks} indices outside their state"
    print("debug build: all cases match the oracle, 0 indices outside the state")


if __name__ == "__main__":
    main()

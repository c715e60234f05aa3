"""Write the stored oracle values that the full-size GPU parity tests and the
benchmark's error report compare against.

Calls only the CPU oracle (``oracle/``) and the seeded workload generators
(``paper_2203_08826_gb300.inputs``, which hold no simulation arithmetic).
Nothing here touches the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py random30     # ~16 GiB of host memory, ~30 min on 8 cores
    python tests/golden/make_golden.py adjoint24    # ~5 min

Files written (plain text, one value per field, full double precision):

random30_d20_seed2022.txt
    The 30-qubit, depth-20 random circuit of the benchmark (seed 2022),
    simulated gate by gate from |0...0> in complex128 by the Eq. (1) loop.
    Amplitudes at 4096 seeded indices and at the 64 indices of largest
    magnitude, <sum_i Z_i Z_{i+1}>, the squared norm and the marginal
    probabilities of qubits (29, 0).

adjoint24_tfim_grad.txt
    The 24-qubit, 10-layer variational ansatz of the gradient workload (seed 5,
    480 parameters) at the first of its 64 seeded parameter sets,
    H = sum_i (Z_i Z_{i+1} + 0.5 X_i): the energy and the gradient entries of
    a few parameters by the two-term parameter-shift rule.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2203_08826_gb300 import inputs  # noqa: E402

RANDOM30 = os.path.join(HERE, "random30_d20_seed2022.txt")
ADJOINT24 = os.path.join(HERE, "adjoint24_tfim_grad.txt")

# indices of the sampled amplitudes: seeded, so the tests draw the same ones
SAMPLE_SEED, SAMPLE_COUNT, TOP_COUNT = 30, 4096, 64
ADJ_PARAMS = (0, 1, 47, 240, 479)


def random30_indices(n: int = 30) -> np.ndarray:
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.unique(rng.integers(0, 1 << n, size=SAMPLE_COUNT, dtype=np.int64))


def make_random30():
    n = 30
    c = inputs.random_circuit(n, 20, seed=2022)
    t0 = time.time()
    psi = oracle.zero_state(n)
    for i, g in enumerate(c.gates):
        oracle.apply_gate(psi, g)
        if i % 50 == 0:
            print(f"gate {i}/{len(c)} {time.time() - t0:.0f} s", flush=True)
    idx = random30_indices(n)
    mag = np.abs(psi)
    top = np.argpartition(mag, -TOP_COUNT)[-TOP_COUNT:]
    del mag
    top = np.sort(top)
    norm2 = float(np.vdot(psi, psi).real)
    zz = oracle.expectation(psi, inputs.zz_chain(n))
    marg = oracle.probabilities(psi, (29, 0))
    with open(RANDOM30, "w") as f:
        f.write("# Written by tests/golden/make_golden.py (CPU oracle only): the 30-qubit depth-20 random\n"
                "# circuit (seed 2022) from |0...0>, complex128, gate by gate (Eq. 1).\n"
                "# norm2 <value>; zz <sum_i Z_i Z_i+1>; marginal_29_0 <p00 p01 p10 p11>;\n"
                "# then 'amp <index> <re> <im>' at the seeded indices and 'top <index> <re> <im>' at the\n"
                "# 64 indices of largest magnitude.\n")
        f.write(f"norm2 {float(norm2)!r}\n")
        f.write(f"zz {float(zz)!r}\n")
        f.write("marginal_29_0 " + " ".join(repr(float(v)) for v in marg) + "\n")
        for i in idx:
            f.write(f"amp {int(i)} {float(psi[i].real)!r} {float(psi[i].imag)!r}\n")
        for i in top:
            f.write(f"top {int(i)} {float(psi[i].real)!r} {float(psi[i].imag)!r}\n")
    print(f"wrote {RANDOM30} in {time.time() - t0:.0f} s")


def make_adjoint24():
    c = inputs.variational(24, 10, seed=5)
    ham = inputs.tfim(24)
    th = np.random.default_rng(0).uniform(0, 2 * np.pi, size=(64, c.nparams))[0]
    t0 = time.time()
    e = oracle.energy(c, ham, th)
    g = oracle.parameter_shift_gradient(c, ham, th, which=ADJ_PARAMS)
    with open(ADJOINT24, "w") as f:
        f.write("# Written by tests/golden/make_golden.py (CPU oracle only): 24-qubit 10-layer variational\n"
                "# ansatz (seed 5), parameter set 0 of default_rng(0).uniform(0, 2 pi, (64, 480)),\n"
                "# H = sum_i (Z_i Z_i+1 + 0.5 X_i); energy, then 'grad <parameter> <value>' by the\n"
                "# parameter-shift rule [E(theta + pi/2) - E(theta - pi/2)] / 2 in complex128.\n")
        f.write(f"energy {float(e)!r}\n")
        for p in ADJ_PARAMS:
            f.write(f"grad {p} {float(g[p])!r}\n")
    print(f"wrote {ADJOINT24} in {time.time() - t0:.0f} s")


def _num(tok: str) -> str:
    # values are written with repr(); numpy scalars print as np.float64(...)
    return tok[len("np.float64("):-1] if tok.startswith("np.float64(") else tok


def read(path: str) -> dict:
    """Parse one of the files above into a dict of arrays and scalars."""
    out = {"amp": [], "top": [], "grad": []}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            vals = [_num(v) for v in vals]
            if key in ("amp", "top"):
                out[key].append((int(vals[0]), complex(float(vals[1]), float(vals[2]))))
            elif key == "grad":
                out[key].append((int(vals[0]), float(vals[1])))
            else:
                v = [float(x) for x in vals]
                out[key] = v[0] if len(v) == 1 else np.array(v)
    for key in ("amp", "top"):
        out[key + "_index"] = np.array([i for i, _ in out[key]], dtype=np.int64)
        out[key + "_value"] = np.array([v for _, v in out[key]], dtype=np.complex128)
    return out


if __name__ == "__main__":
    oracle.build()
    what = sys.argv[1:] or ["random30", "adjoint24"]
    if "adjoint24" in what:
        make_adjoint24()
    if "random30" in what:
        make_random30()

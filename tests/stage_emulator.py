"""A host model of the register-tile stage kernels, for tests only.

It runs the op lists a staged plan hands to its kernels (read through
qsim_plan_stage_dump) with the kernels' data layout -- per tile, per warp
and lane, 16 registers; lanes hold qubits 0..4, registers and warps the
qubits of the current phase; exchanges re-assign them through the tile --
and each op's definition as the kernels apply it (coefficient layouts for
lane targets included), in complex128 numpy.  Comparing its result with the
oracle's gate-by-gate run checks the planner, the fusion passes and the op
lists without a GPU.  Shares no code with the library.
"""
from __future__ import annotations

import numpy as np

LANE_BITS, REG_BITS = 5, 4
POS_REG, POS_BASE = 8, 32
U1, U2, DIAG, EXCHANGE, U1R, U1L, NEG, GRAD = range(8)


def parse(dump: str) -> dict:
    st = {"phases": [], "ops": [], "pool": [], "aux": []}
    for line in dump.splitlines():
        f = line.split()
        if not f:
            continue
        if f[0] == "stage":
            st["plain"], st["W"], st["phase0"] = int(f[3]), int(f[5]), int(f[7])
        elif f[0] == "slots":
            st["slots"] = [int(x) for x in f[1:]]
        elif f[0] == "phase":
            parts = " ".join(f[1:]).split("|")
            rq, wq, rslot, wslot = ([int(x) for x in p.split()] for p in parts)
            st["phases"].append((rq, wq))
        elif f[0] == "op":
            v = [int(x) for x in f[1:]]
            st["ops"].append({"type": v[0], "a": v[1], "b": v[2], "k": v[3], "rneed": v[4], "flags": v[5],
                              "tmask": v[6], "moff": v[7], "dq": v[8:]})
        elif f[0] == "pool":
            st["pool"].append(complex(float(f[1]), float(f[2])))
        elif f[0] == "aux":
            st["aux"].append(int(f[1]))
    return st


class Tile:
    """All tiles of one stage at once: v[t, w, l, j] is register j of lane l
    of warp w in tile t."""

    def __init__(self, n: int, st: dict):
        self.n, self.st, self.W = n, st, st["W"]
        tq = list(range(LANE_BITS)) + st["slots"]
        rest = [q for q in range(n) if q not in tq]
        t = np.arange(1 << len(rest), dtype=np.uint64)
        tb = np.zeros_like(t)
        for i, q in enumerate(rest):
            tb |= ((t >> np.uint64(i)) & np.uint64(1)) << np.uint64(q)
        self.tile_base = tb[:, None, None]
        self.lane = np.arange(32, dtype=np.uint64)[None, None, :]
        self.warp = np.arange(1 << self.W, dtype=np.uint64)[None, :, None]

    def base(self, ph: int) -> np.ndarray:
        rq, wq = self.st["phases"][ph]
        b = self.tile_base | self.lane
        for i in range(self.W):
            b = b | (((self.warp >> np.uint64(i)) & np.uint64(1)) << np.uint64(wq[i]))
        return b  # [T, 2^W, 32]

    def index(self, ph: int) -> np.ndarray:
        rq, _ = self.st["phases"][ph]
        j = np.arange(1 << REG_BITS, dtype=np.uint64)
        off = np.zeros_like(j)
        for b in range(REG_BITS):
            off |= ((j >> np.uint64(b)) & np.uint64(1)) << np.uint64(rq[b])
        return self.base(ph)[..., None] | off  # [T, 2^W, 32, 16]


def _partner(v: np.ndarray, lane_mask: int) -> np.ndarray:
    return v[:, :, np.arange(32) ^ lane_mask, :]


def run_stage(psi: np.ndarray, n: int, st: dict) -> None:
    """Apply one tile stage to psi (complex128, in place)."""
    tile = Tile(n, st)
    pool, aux = np.array(st["pool"], dtype=np.complex128), st["aux"]
    ph = st["phase0"]
    idx = tile.index(ph).astype(np.int64)
    v = psi[idx]
    base = tile.base(ph)
    lane = np.arange(32)

    def tok(tmask):
        return ((base & np.uint64(tmask)) == np.uint64(tmask))[..., None]  # [T, W, 32, 1]

    def u1_reg(rb, m, rneed=0, ok=None):
        for i in range(1 << REG_BITS):
            if (i >> rb) & 1 or (i & rneed) != rneed:
                continue
            i1 = i | (1 << rb)
            a, b = v[..., i].copy(), v[..., i1].copy()
            na, nb = m[0] * a + m[1] * b, m[2] * a + m[3] * b
            if ok is not None:
                na, nb = np.where(ok[..., 0], na, a), np.where(ok[..., 0], nb, b)
            v[..., i], v[..., i1] = na, nb

    def u1_lane(l, m, rneed=0, ok=None):
        bit = ((lane >> l) & 1)[None, None, :]
        cs, co = np.where(bit == 1, m[3], m[0]), np.where(bit == 1, m[2], m[1])
        other = _partner(v, 1 << l).copy()
        for j in range(1 << REG_BITS):
            if (j & rneed) != rneed:
                continue
            new = co * other[..., j] + cs * v[..., j]
            v[..., j] = new if ok is None else np.where(ok[..., 0], new, v[..., j])

    for op in st["ops"]:
        t, a, b, k, rneed, moff = op["type"], op["a"], op["b"], op["k"], op["rneed"], op["moff"]
        ok = tok(op["tmask"])
        if t == EXCHANGE:
            # through the tile: every amplitude back to its index, then out in
            # the new phase's layout
            tmp = psi.copy()
            tmp[idx] = v
            ph = a
            idx = tile.index(ph).astype(np.int64)
            v = tmp[idx]
            base = tile.base(ph)
        elif t == U1:
            m = pool[moff:moff + 4]
            if a >= POS_REG:
                u1_reg(a - POS_REG, m, rneed, ok)
            else:
                u1_lane(a, m, rneed, ok)
        elif t == U1R:
            off = moff
            for rb in range(REG_BITS):
                if a & (1 << rb):
                    u1_reg(rb, pool[off:off + 4])
                    off += 4
        elif t == U1L:
            off = moff
            for l in range(LANE_BITS):
                if a & (1 << l):
                    u1_lane(l, pool[off:off + 4])
                    off += 4
        elif t == U2 and a >= POS_REG and b >= POS_REG:
            ja, jb = a - POS_REG, b - POS_REG
            m = pool[moff:moff + 16].reshape(4, 4)
            for i in range(1 << REG_BITS):
                if i & ((1 << ja) | (1 << jb)) or (i & rneed) != rneed:
                    continue
                ids = [i, i | (1 << jb), i | (1 << ja), i | (1 << ja) | (1 << jb)]
                x = v[..., ids].copy()
                new = x @ m.T
                v[..., ids] = np.where(ok, new, x)
        elif t == U2 and (a >= POS_REG) != (b >= POS_REG):
            la = a if a < POS_REG else b
            rb = (b if a < POS_REG else a) - POS_REG
            beta = ((lane >> la) & 1)[None, None, :]
            m = np.where(beta[..., None] == 1, pool[moff + 8:moff + 16], pool[moff:moff + 8])  # [1, 1, 32, 8]
            other = _partner(v, 1 << la).copy()
            for i in range(1 << REG_BITS):
                if (i >> rb) & 1 or (i & rneed) != rneed:
                    continue
                i1 = i | (1 << rb)
                x0, x1, y0, y1 = v[..., i].copy(), v[..., i1].copy(), other[..., i], other[..., i1]
                n0 = m[..., 0] * x0 + m[..., 1] * x1 + m[..., 2] * y0 + m[..., 3] * y1
                n1 = m[..., 4] * x0 + m[..., 5] * x1 + m[..., 6] * y0 + m[..., 7] * y1
                v[..., i], v[..., i1] = np.where(ok[..., 0], n0, x0), np.where(ok[..., 0], n1, x1)
        elif t == U2:
            sel = ((((lane >> a) & 1) << 1) | ((lane >> b) & 1))[None, None, :]
            m = np.stack([pool[moff + 4 * s:moff + 4 * s + 4] for s in range(4)])[sel]  # [1, 1, 32, 4]
            p1, p2, p3 = (_partner(v, mask).copy() for mask in (1 << a, 1 << b, (1 << a) | (1 << b)))
            for j in range(1 << REG_BITS):
                if (j & rneed) != rneed:
                    continue
                new = m[..., 0] * v[..., j] + m[..., 1] * p1[..., j] + m[..., 2] * p2[..., j] + m[..., 3] * p3[..., j]
                v[..., j] = np.where(ok[..., 0], new, v[..., j])
        elif t == DIAG:
            for j in range(1 << REG_BITS):
                if (j & rneed) != rneed:
                    continue
                if k == 0:
                    f = -1.0 if op["flags"] & 1 else pool[moff]
                else:
                    sel = np.zeros(base.shape, dtype=np.int64)
                    for q in range(k):
                        code = op["dq"][q]
                        if code >= POS_BASE:
                            bit = ((base >> np.uint64(code - POS_BASE)) & np.uint64(1)).astype(np.int64)
                        else:
                            bit = (j >> (code - POS_REG)) & 1
                        sel |= bit << (k - 1 - q)
                    f = pool[moff + sel]
                v[..., j] = np.where(ok[..., 0], f * v[..., j], v[..., j])
        elif t == NEG:
            flip = np.zeros(base.shape, dtype=np.int64)
            for e in range(k):
                tm, pat = aux[moff + 2 * e], aux[moff + 2 * e + 1]
                hit = (base & np.uint64(tm)) == np.uint64(tm)
                flip ^= np.where(hit, pat, 0)
            for j in range(1 << REG_BITS):
                v[..., j] = np.where((flip >> j) & 1 == 1, -v[..., j], v[..., j])
        elif t == GRAD:
            pass  # gradient sums; forward plans carry none
    psi[idx] = v


def run_plan(plan, circ, psi0: np.ndarray, orc) -> np.ndarray:
    """psi0 through every stage of a staged plan: tile stages by the model
    above, plain stages (one gate each) by the oracle."""
    psi = psi0.astype(np.complex128).copy()
    for i, s in enumerate(plan.stages()):
        if s["plain"]:
            for gi in s["gates"]:
                orc.apply_gate(psi, circ.gates[gi])
            continue
        run_stage(psi, circ.n, parse(plan.stage_dump(i)))
    return psi

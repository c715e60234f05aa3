// Cache-blocked multi-gate stages (QSIM_FUSE_STAGED).
//
// One stage = one HBM pass.  A CTA of 32 * 2^W threads owns a tile of
// 2^(5+4+W) amplitudes: the amplitudes whose indices agree outside the tile
// qubits.  The tile qubits are
//   - qubits 0..4, held by the 32 lanes of each warp (so every global access
//     of a warp is a contiguous run of 32 amplitudes),
//   - 4 "register" qubits: each thread holds the 16 amplitudes that differ in
//     them, in registers,
//   - W "warp" qubits, selected by the warp index.
// Gates are applied in circuit order while the tile sits in registers:
//   - a dense 1-qubit gate on a register qubit pairs registers; on a lane
//     qubit it pairs lanes through __shfl_xor_sync;
//   - a dense 2-qubit gate on two register qubits mixes groups of 4 registers;
//   - a diagonal gate (CZ, controlled phases, RZ, ...) multiplies every
//     amplitude by the entry its index selects -- its qubits may lie anywhere,
//     inside or outside the tile, because the full index of every amplitude is
//     known;
//   - controls may lie anywhere for the same reason;
//   - an EXCHANGE writes the tile to shared memory and reads it back with a
//     different choice of register and warp qubits.
// This is Eq. (1) applied gate by gate, with the amplitudes of each group
// gathered once per stage instead of once per gate.  The op list, the phase
// table and the matrices of a stage travel in the kernel parameters (constant
// bank), so every thread reads them at register speed.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"
#include "plan.h"

namespace qsim {

namespace {
constexpr int LANE_BITS = 5;
constexpr int REG_BITS = 4;  // amplitudes per thread = 16
constexpr int MAX_WARP_BITS = 4;
constexpr int MAX_SLOTS = REG_BITS + MAX_WARP_BITS;
constexpr int MAX_OPS = 192;
constexpr int MAX_PHASES = 24;
constexpr int MAX_POOL = 768;

enum SopType : int8_t { SOP_U1 = 0, SOP_U2 = 1, SOP_DIAG = 2, SOP_EXCHANGE = 3 };

// Position codes: 0..4 lane bit, 8 + b register bit b, 32 + q bit q of the
// thread's base index (lane, warp or tile qubit).
constexpr int POS_REG = 8;
constexpr int POS_BASE = 32;

struct StageOp {
    uint64_t tmask;  // control bits outside the registers: (base & tmask) == tmask
    int32_t moff;    // offset of the matrix / diagonal in the pool (complex entries)
    int8_t type;
    int8_t a, b;     // U1: target position; U2: positions (a = MSB); EXCHANGE: a = phase
    int8_t k;        // DIAG: number of selector qubits
    int8_t rneed;    // control bits on register qubits: (j & rneed) == rneed
    int8_t flags;    // DIAG k = 0: 1 when the factor is exactly -1
    int8_t dq[QSIM_MAX_TARGETS];  // DIAG selectors (position codes), dq[0] = MSB
};

struct Phase {
    int8_t rq[REG_BITS];       // global qubit of register bit b
    int8_t wq[MAX_WARP_BITS];  // global qubit of warp bit b
    int8_t rslot[REG_BITS];    // shared-memory bit (above the lane bits) of register bit b
    int8_t wslot[MAX_WARP_BITS];
};

template <typename C> struct StageParams {
    IndexMap outer;  // inserts zeros at the tile qubits (tile id -> base index)
    int nops, phase0;
    Phase phases[MAX_PHASES];
    StageOp ops[MAX_OPS];
    C pool[MAX_POOL];
};

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cmad(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

__device__ __forceinline__ uint64_t expand(uint64_t g, const IndexMap &m) {
#pragma unroll 1
    for (int i = 0; i < m.nins; ++i) {
        const uint64_t low = g & ((uint64_t(1) << m.ins[i]) - 1);
        g = ((g ^ low) << 1) | low;
    }
    return g | m.set;
}

template <typename C, int JB, bool CTRL>
__device__ __forceinline__ void u1_reg(C (&v)[1 << REG_BITS], C m00, C m01, C m10, C m11, int rneed) {
#pragma unroll
    for (int i = 0; i < (1 << REG_BITS); ++i) {
        if (i & (1 << JB)) continue;
        if (CTRL && (i & rneed) != rneed) continue;
        const C a = v[i], b = v[i | (1 << JB)];
        v[i] = cmad(m01, b, cmul(m00, a));
        v[i | (1 << JB)] = cmad(m11, b, cmul(m10, a));
    }
}

template <typename C, int JB>
__device__ __forceinline__ void u1_reg_dispatch(C (&v)[1 << REG_BITS], C m00, C m01, C m10, C m11, int rneed) {
    if (rneed) u1_reg<C, JB, true>(v, m00, m01, m10, m11, rneed);
    else u1_reg<C, JB, false>(v, m00, m01, m10, m11, 0);
}

template <typename C, int JA, int JB>
__device__ __forceinline__ void u2_reg(C (&v)[1 << REG_BITS], const C *m, int rneed) {
    // matrix index bit 1 <-> register bit JA, bit 0 <-> register bit JB
#pragma unroll
    for (int i = 0; i < (1 << REG_BITS); ++i) {
        if (i & ((1 << JA) | (1 << JB))) continue;
        if ((i & rneed) != rneed) continue;
        const int idx[4] = {i, i | (1 << JB), i | (1 << JA), i | (1 << JA) | (1 << JB)};
        C x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = v[idx[c]];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            C acc = cmul(m[r * 4], x[0]);
#pragma unroll
            for (int c = 1; c < 4; ++c) acc = cmad(m[r * 4 + c], x[c], acc);
            v[idx[r]] = acc;
        }
    }
}

__device__ __forceinline__ float2 shfl_c(float2 a, int mask) {
    a.x = __shfl_xor_sync(0xffffffffu, a.x, mask);
    a.y = __shfl_xor_sync(0xffffffffu, a.y, mask);
    return a;
}
__device__ __forceinline__ double2 shfl_c(double2 a, int mask) {
    a.x = __shfl_xor_sync(0xffffffffu, a.x, mask);
    a.y = __shfl_xor_sync(0xffffffffu, a.y, mask);
    return a;
}

// Global index of register 0 of this thread in phase P.
template <int W>
__device__ __forceinline__ uint64_t thread_base(const Phase &P, uint64_t tile_base, int lane, int warp) {
    uint64_t b = tile_base | uint64_t(lane);
#pragma unroll
    for (int i = 0; i < W; ++i)
        if ((warp >> i) & 1) b |= uint64_t(1) << P.wq[i];
    return b;
}

template <typename C, int W, bool STORE>
__device__ __forceinline__ void tile_global(C *__restrict__ psi, C (&v)[1 << REG_BITS], const Phase &P,
                                            uint64_t base) {
    uint64_t rm[REG_BITS];
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) rm[b] = uint64_t(1) << P.rq[b];
#pragma unroll
    for (int j = 0; j < (1 << REG_BITS); ++j) {
        uint64_t x = base;
#pragma unroll
        for (int b = 0; b < REG_BITS; ++b)
            if ((j >> b) & 1) x |= rm[b];
        if (STORE) psi[x] = v[j];
        else v[j] = psi[x];
    }
}

template <typename C, int W, bool STORE>
__device__ __forceinline__ void tile_shared(C *tile, C (&v)[1 << REG_BITS], const Phase &P, int lane, int warp) {
    uint32_t lb = uint32_t(lane), lm[REG_BITS];
#pragma unroll
    for (int i = 0; i < W; ++i)
        if ((warp >> i) & 1) lb |= uint32_t(1) << (LANE_BITS + P.wslot[i]);
#pragma unroll
    for (int b = 0; b < REG_BITS; ++b) lm[b] = uint32_t(1) << (LANE_BITS + P.rslot[b]);
#pragma unroll
    for (int j = 0; j < (1 << REG_BITS); ++j) {
        uint32_t l = lb;
#pragma unroll
        for (int b = 0; b < REG_BITS; ++b)
            if ((j >> b) & 1) l |= lm[b];
        if (STORE) tile[l] = v[j];
        else v[j] = tile[l];
    }
}

template <typename R, int W>
__global__ void __launch_bounds__(32 << W, (sizeof(R) == 4 ? (W <= 3 ? 3 : 2) : 1))
    k_stage(typename CT<R>::T *__restrict__ psi, const __grid_constant__ StageParams<typename CT<R>::T> p) {
    using C = typename CT<R>::T;
    constexpr int NR = 1 << REG_BITS;
    extern __shared__ unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t tile_base = expand(blockIdx.x, p.outer);

    int ph = p.phase0;
    uint64_t base = thread_base<W>(p.phases[ph], tile_base, lane, warp);
    C v[NR];
    tile_global<C, W, false>(psi, v, p.phases[ph], base);

    for (int o = 0; o < p.nops; ++o) {
        const StageOp &op = p.ops[o];
        const int type = op.type;
        if (type == SOP_EXCHANGE) {
            tile_shared<C, W, true>(tile, v, p.phases[ph], lane, warp);
            __syncthreads();
            ph = op.a;
            base = thread_base<W>(p.phases[ph], tile_base, lane, warp);
            tile_shared<C, W, false>(tile, v, p.phases[ph], lane, warp);
            __syncthreads();
            continue;
        }
        // controls on lane / warp / tile qubits: one test per thread (a lane
        // gate still takes part in the shuffles when its controls are not met)
        const bool tok = (base & op.tmask) == op.tmask;
        if (!tok && !(type == SOP_U1 && op.a < POS_REG)) continue;
        const int rneed = op.rneed;
        if (type == SOP_U1) {
            const C m00 = p.pool[op.moff], m01 = p.pool[op.moff + 1];
            const C m10 = p.pool[op.moff + 2], m11 = p.pool[op.moff + 3];
            if (op.a >= POS_REG) {
                switch (op.a - POS_REG) {
                    case 0: u1_reg_dispatch<C, 0>(v, m00, m01, m10, m11, rneed); break;
                    case 1: u1_reg_dispatch<C, 1>(v, m00, m01, m10, m11, rneed); break;
                    case 2: u1_reg_dispatch<C, 2>(v, m00, m01, m10, m11, rneed); break;
                    default: u1_reg_dispatch<C, 3>(v, m00, m01, m10, m11, rneed); break;
                }
            } else {
                const int bit = (lane >> op.a) & 1;
                const C cs = bit ? m11 : m00, co = bit ? m10 : m01;
                const int lm = 1 << op.a;
                if (tok && rneed == 0) {
#pragma unroll
                    for (int j = 0; j < NR; ++j) v[j] = cmad(co, shfl_c(v[j], lm), cmul(cs, v[j]));
                } else {
#pragma unroll
                    for (int j = 0; j < NR; ++j) {
                        const C other = shfl_c(v[j], lm);
                        if (tok && (j & rneed) == rneed) v[j] = cmad(co, other, cmul(cs, v[j]));
                    }
                }
            }
        } else if (type == SOP_U2) {
            const C *m = p.pool + op.moff;
            switch ((op.a - POS_REG) * 4 + (op.b - POS_REG)) {
                case 1: u2_reg<C, 0, 1>(v, m, rneed); break;
                case 2: u2_reg<C, 0, 2>(v, m, rneed); break;
                case 3: u2_reg<C, 0, 3>(v, m, rneed); break;
                case 4: u2_reg<C, 1, 0>(v, m, rneed); break;
                case 6: u2_reg<C, 1, 2>(v, m, rneed); break;
                case 7: u2_reg<C, 1, 3>(v, m, rneed); break;
                case 8: u2_reg<C, 2, 0>(v, m, rneed); break;
                case 9: u2_reg<C, 2, 1>(v, m, rneed); break;
                case 11: u2_reg<C, 2, 3>(v, m, rneed); break;
                case 12: u2_reg<C, 3, 0>(v, m, rneed); break;
                case 13: u2_reg<C, 3, 1>(v, m, rneed); break;
                default: u2_reg<C, 3, 2>(v, m, rneed); break;
            }
        } else if (op.k == 0) {  // SOP_DIAG, one factor on the control subspace
            if (op.flags & 1) {
                if (rneed == 0) {
#pragma unroll
                    for (int j = 0; j < NR; ++j) {
                        v[j].x = -v[j].x;
                        v[j].y = -v[j].y;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < NR; ++j)
                        if ((j & rneed) == rneed) {
                            v[j].x = -v[j].x;
                            v[j].y = -v[j].y;
                        }
                }
            } else {
                const C f = p.pool[op.moff];
#pragma unroll
                for (int j = 0; j < NR; ++j)
                    if ((j & rneed) == rneed) v[j] = cmul(f, v[j]);
            }
        } else {  // SOP_DIAG with selector qubits
            int sel_t = 0, regsel[QSIM_MAX_TARGETS];
            const int k = op.k;
            for (int t = 0; t < k; ++t) {
                const int code = op.dq[t];
                const int sh = k - 1 - t;
                if (code >= POS_BASE) {
                    sel_t |= int((base >> (code - POS_BASE)) & 1) << sh;
                    regsel[t] = 0;
                } else {
                    regsel[t] = code - POS_REG + 1;  // register bit + 1
                }
            }
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                if ((j & rneed) != rneed) continue;
                int sel = sel_t;
                for (int t = 0; t < k; ++t)
                    if (regsel[t]) sel |= ((j >> (regsel[t] - 1)) & 1) << (k - 1 - t);
                v[j] = cmul(p.pool[op.moff + sel], v[j]);
            }
        }
    }
    tile_global<C, W, true>(psi, v, p.phases[ph], base);
}

// ------------------------------------------------------------------ host plan
struct GateClass {
    enum { DIAG, DENSE1, DENSE2, OTHER } kind;
    Op op;  // classified form (targets reduced, controls extended)
};

struct Stage {
    bool plain = false;
    Op op;                   // plain: one sweep
    std::vector<int> slots;  // tile qubits outside the lanes (slot s <-> slots[s])
    std::vector<StageOp> ops;
    std::vector<Phase> phases;
    std::vector<cd> pool;
    int phase0 = 0;
};

uint64_t qmask(const int *q, int n) {
    uint64_t m = 0;
    for (int i = 0; i < n; ++i) m |= uint64_t(1) << q[i];
    return m;
}

// Build the op list of one tile stage from its gates (circuit order).
// Returns QSIM_EUNSUPPORTED (without error text) when the stage outgrows the
// parameter-block limits; the caller then splits it.
int emit_stage_ops(Stage &st, const std::vector<const GateClass *> &gates, int W) {
    const int nslots = REG_BITS + W;
    auto slot_of = [&](int q) {
        for (int s = 0; s < nslots; ++s)
            if (st.slots[s] == q) return s;
        return -1;
    };
    std::vector<std::vector<int>> need(gates.size());
    for (size_t i = 0; i < gates.size(); ++i) {
        const GateClass &g = *gates[i];
        if (g.kind == GateClass::DIAG) continue;
        for (int t = 0; t < g.op.k; ++t)
            if (g.op.targets[t] >= LANE_BITS) need[i].push_back(g.op.targets[t]);
    }
    // register set for the window starting at gate `from`: the next distinct
    // qubits the dense gates need, as many as fit
    auto pick = [&](size_t from) {
        std::vector<int> regs;
        for (size_t i = from; i < gates.size() && int(regs.size()) < REG_BITS; ++i) {
            std::vector<int> add;
            for (int q : need[i])
                if (std::find(regs.begin(), regs.end(), q) == regs.end()) add.push_back(q);
            if (int(regs.size() + add.size()) > REG_BITS) break;
            for (int q : add) regs.push_back(q);
        }
        for (int q : st.slots) {
            if (int(regs.size()) >= REG_BITS) break;
            if (std::find(regs.begin(), regs.end(), q) == regs.end()) regs.push_back(q);
        }
        Phase P{};
        int wi = 0;
        for (int b = 0; b < REG_BITS; ++b) {
            P.rq[b] = int8_t(regs[b]);
            P.rslot[b] = int8_t(slot_of(regs[b]));
        }
        for (int q : st.slots)
            if (std::find(regs.begin(), regs.end(), q) == regs.end()) {
                P.wq[wi] = int8_t(q);
                P.wslot[wi] = int8_t(slot_of(q));
                ++wi;
            }
        st.phases.push_back(P);
        return int(st.phases.size()) - 1;
    };
    int cur = pick(0);
    st.phase0 = cur;
    size_t phase_first_op = 0;
    auto reg_bit = [&](int q) -> int {  // register bit of q in the current phase, or -1
        const Phase &P = st.phases[cur];
        for (int b = 0; b < REG_BITS; ++b)
            if (P.rq[b] == q) return b;
        return -1;
    };
    auto pos_of = [&](int q) -> int {  // U1/U2 target position
        if (q < LANE_BITS) return q;
        const int b = reg_bit(q);
        return b < 0 ? -1 : POS_REG + b;
    };
    auto split_controls = [&](const Op &op, StageOp &so) {
        so.tmask = 0;
        so.rneed = 0;
        for (int i = 0; i < op.c; ++i) {
            const int q = op.controls[i];
            const int b = reg_bit(q);
            if (b >= 0) so.rneed |= int8_t(1 << b);
            else so.tmask |= uint64_t(1) << q;
        }
    };
    auto add_pool = [&](const std::vector<cd> &m) {
        const int off = int(st.pool.size());
        st.pool.insert(st.pool.end(), m.begin(), m.end());
        return off;
    };
    // does op `so` read or write qubit q (current phase)?
    auto touches = [&](const StageOp &so, int q) {
        const int b = reg_bit(q);
        if (b >= 0 && (so.rneed >> b & 1)) return true;
        if (so.tmask >> q & 1) return true;
        if (so.type == SOP_U1) return so.a == pos_of(q);
        if (so.type == SOP_U2) return so.a == pos_of(q) || so.b == pos_of(q);
        if (so.type == SOP_DIAG)
            for (int t = 0; t < so.k; ++t)
                if (so.dq[t] == (b >= 0 ? POS_REG + b : POS_BASE + q)) return true;
        return false;
    };
    // index of a preceding uncontrolled U1 on q that nothing after it touches, or -1
    auto mergeable_u1 = [&](int q) -> int {
        for (size_t o = st.ops.size(); o-- > phase_first_op;) {
            const StageOp &prev = st.ops[o];
            if (!touches(prev, q)) continue;
            if (prev.type == SOP_U1 && prev.a == pos_of(q) && prev.tmask == 0 && prev.rneed == 0) return int(o);
            return -1;
        }
        return -1;
    };
    for (size_t i = 0; i < gates.size(); ++i) {
        const GateClass &g = *gates[i];
        if (g.kind == GateClass::DIAG) {
            if (g.op.k == 1 && g.op.c == 0) {
                // fold an uncontrolled 1-qubit diagonal into a preceding U1 on its qubit
                const int mi = pos_of(g.op.targets[0]) >= 0 ? mergeable_u1(g.op.targets[0]) : -1;
                if (mi >= 0) {
                    StageOp &prev = st.ops[mi];
                    std::vector<cd> old(st.pool.begin() + prev.moff, st.pool.begin() + prev.moff + 4);
                    std::vector<cd> dm = {g.op.m[0], 0.0, 0.0, g.op.m[1]};
                    std::vector<cd> nw = matmul(dm, old, 2);
                    std::copy(nw.begin(), nw.end(), st.pool.begin() + prev.moff);
                    continue;
                }
            }
            StageOp so{};
            so.type = SOP_DIAG;
            so.k = int8_t(g.op.k);
            split_controls(g.op, so);
            for (int t = 0; t < g.op.k; ++t) {
                const int q = g.op.targets[t];
                const int b = reg_bit(q);
                so.dq[t] = int8_t(b >= 0 ? POS_REG + b : POS_BASE + q);
            }
            if (g.op.k == 0 && g.op.m[0] == cd(-1.0)) so.flags = 1;
            so.moff = add_pool(g.op.m);
            st.ops.push_back(so);
            continue;
        }
        bool ok = true;
        for (int t = 0; t < g.op.k; ++t)
            if (pos_of(g.op.targets[t]) < 0) ok = false;
        if (!ok) {
            cur = pick(i);
            StageOp ex{};
            ex.type = SOP_EXCHANGE;
            ex.a = int8_t(cur);
            st.ops.push_back(ex);
            phase_first_op = st.ops.size();
            for (int t = 0; t < g.op.k; ++t)
                if (pos_of(g.op.targets[t]) < 0) return set_error(QSIM_EINVAL, "staged planner: register window");
        }
        StageOp so{};
        split_controls(g.op, so);
        if (g.kind == GateClass::DENSE1) {
            so.type = SOP_U1;
            so.a = int8_t(pos_of(g.op.targets[0]));
            if (so.tmask == 0 && so.rneed == 0) {
                const int mi = mergeable_u1(g.op.targets[0]);
                if (mi >= 0) {
                    StageOp &prev = st.ops[mi];
                    std::vector<cd> old(st.pool.begin() + prev.moff, st.pool.begin() + prev.moff + 4);
                    std::vector<cd> nw = matmul(g.op.m, old, 2);
                    std::copy(nw.begin(), nw.end(), st.pool.begin() + prev.moff);
                    continue;
                }
            }
        } else {
            so.type = SOP_U2;
            so.a = int8_t(pos_of(g.op.targets[0]));
            so.b = int8_t(pos_of(g.op.targets[1]));
        }
        so.moff = add_pool(g.op.m);
        st.ops.push_back(so);
    }
    if (st.ops.size() > size_t(MAX_OPS) || st.phases.size() > size_t(MAX_PHASES) ||
        st.pool.size() > size_t(MAX_POOL))
        return QSIM_EUNSUPPORTED;
    return QSIM_OK;
}

}  // namespace

struct StagedPlan {
    int W = 4;
    std::vector<Stage> stages;
    struct Dev {
        bool ready = false;
        std::vector<void *> plain_mats;
        std::vector<unsigned char> params;  // packed StageParams per tile stage
        std::vector<size_t> param_off;
    } dev[2];
    ~StagedPlan() {
        for (Dev &d : dev)
            for (void *m : d.plain_mats)
                if (m) cudaFree(m);
    }
};

int build_staged(const qsim_circuit &c, qsim_plan &p) {
    const int n = c.n;
    if (n < LANE_BITS + REG_BITS) {
        // too small for a tile: the paper's greedy fusion plan serves
        p.mode = QSIM_FUSE_GREEDY2;
        return build_greedy2(c, p);
    }
    StagedPlan *sp = new StagedPlan();
    p.staged = sp;
    // kmax selects the tile: 2^(9 + W) amplitudes with W = min(kmax, 4) warp qubits
    const int W = std::min(std::min(p.kmax, MAX_WARP_BITS), n - LANE_BITS - REG_BITS);
    sp->W = W;
    const int cap = REG_BITS + W;
    std::vector<GateClass> cls(c.gates.size());
    for (size_t i = 0; i < c.gates.size(); ++i) {
        const GateRec &g = c.gates[i];
        QSIM_TRY(classify(g.m, g.targets, g.k, g.controls, g.nc, cls[i].op));
        Op &op = cls[i].op;
        if (op.type == Op::IDENTITY || op.type == Op::DIAG) {
            cls[i].kind = GateClass::DIAG;
            if (op.type == Op::IDENTITY) {
                op.type = Op::DIAG;
                op.k = 0;
                op.c = 0;
                op.m = {cd(1.0)};
            }
        } else {
            if (op.type == Op::MONO) {  // the stage applies the full matrix
                const size_t d = size_t(1) << op.k;
                op.m.assign(d * d, cd(0.0));
                for (size_t r = 0; r < d; ++r) op.m[r * d + op.perm[r]] = op.phase[r];
                op.type = Op::DENSE;
            }
            bool lane_target = false;
            for (int t = 0; t < op.k; ++t) lane_target |= op.targets[t] < LANE_BITS;
            if (op.k == 1) cls[i].kind = GateClass::DENSE1;
            else if (op.k == 2 && !lane_target) cls[i].kind = GateClass::DENSE2;
            else cls[i].kind = GateClass::OTHER;
        }
    }
    std::vector<int> remaining(c.gates.size());
    for (size_t i = 0; i < remaining.size(); ++i) remaining[i] = int(i);
    size_t limit = remaining.size();  // largest number of gates one stage may take
    while (!remaining.empty()) {
        uint64_t blocked = 0;
        std::vector<int> tile;
        std::vector<int> sched, rest;
        bool plain_emitted = false;
        for (size_t r = 0; r < remaining.size(); ++r) {
            const int gi = remaining[r];
            const GateClass &g = cls[gi];
            const uint64_t qs = qmask(g.op.targets, g.op.k) | qmask(g.op.controls, g.op.c);
            if ((qs & blocked) || sched.size() >= limit) {
                blocked |= qs;
                rest.push_back(gi);
                continue;
            }
            if (g.kind == GateClass::DIAG) {
                sched.push_back(gi);
                continue;
            }
            if (g.kind == GateClass::OTHER) {
                if (sched.empty() && !plain_emitted && r == 0) {
                    Stage st;
                    st.plain = true;
                    st.op = g.op;
                    sp->stages.push_back(std::move(st));
                    plain_emitted = true;
                    continue;
                }
                blocked |= qs;
                rest.push_back(gi);
                continue;
            }
            std::vector<int> add;
            for (int t = 0; t < g.op.k; ++t) {
                const int q = g.op.targets[t];
                if (q >= LANE_BITS && std::find(tile.begin(), tile.end(), q) == tile.end()) add.push_back(q);
            }
            if (int(tile.size() + add.size()) <= cap) {
                tile.insert(tile.end(), add.begin(), add.end());
                sched.push_back(gi);
            } else {
                blocked |= qs;
                rest.push_back(gi);
            }
        }
        if (sched.empty()) {
            remaining.swap(rest);
            limit = remaining.size();
            continue;
        }
        for (int q = LANE_BITS; q < n && int(tile.size()) < cap; ++q)
            if (std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
        Stage st;
        st.slots = tile;
        std::vector<const GateClass *> gl;
        for (int gi : sched) gl.push_back(&cls[gi]);
        const int rc = emit_stage_ops(st, gl, W);
        if (rc == QSIM_EUNSUPPORTED) {
            // too many ops for one parameter block: retry with half the gates
            // (any prefix of an order-respecting schedule is one too); a plain
            // stage emitted in this scan stays, its gate is not in `merged`
            limit = std::max<size_t>(1, sched.size() / 2);
            std::vector<int> merged(sched);
            merged.insert(merged.end(), rest.begin(), rest.end());
            std::sort(merged.begin(), merged.end());
            remaining.swap(merged);
            continue;
        }
        QSIM_TRY(rc);
        sp->stages.push_back(std::move(st));
        remaining.swap(rest);
        limit = remaining.size();
    }
    return QSIM_OK;
}

template <typename C> static void make_params(const Stage &st, StageParams<C> &prm) {
    memset(&prm, 0, sizeof prm);
    int tq[LANE_BITS + MAX_SLOTS];
    int nt = 0;
    for (int q = 0; q < LANE_BITS; ++q) tq[nt++] = q;
    for (int q : st.slots) tq[nt++] = q;
    prm.outer = make_index_map(tq, nt, nullptr, 0);
    prm.nops = int(st.ops.size());
    prm.phase0 = st.phase0;
    for (size_t i = 0; i < st.phases.size(); ++i) prm.phases[i] = st.phases[i];
    for (size_t i = 0; i < st.ops.size(); ++i) prm.ops[i] = st.ops[i];
    for (size_t i = 0; i < st.pool.size(); ++i) {
        prm.pool[i].x = decltype(prm.pool[i].x)(st.pool[i].real());
        prm.pool[i].y = decltype(prm.pool[i].y)(st.pool[i].imag());
    }
}

static int prepare_staged(qsim_plan &p, int dtype) {
    StagedPlan &sp = *p.staged;
    StagedPlan::Dev &d = sp.dev[dtype];
    if (d.ready) return QSIM_OK;
    const size_t eb = dtype == QSIM_C64 ? 8 : 16;
    d.plain_mats.assign(sp.stages.size(), nullptr);
    d.param_off.assign(sp.stages.size(), 0);
    const size_t psz = dtype == QSIM_C64 ? sizeof(StageParams<float2>) : sizeof(StageParams<double2>);
    d.params.clear();
    for (size_t i = 0; i < sp.stages.size(); ++i) {
        const Stage &st = sp.stages[i];
        if (st.plain) {
            if (st.op.type != Op::DENSE || st.op.k < 2) continue;
            const size_t D = size_t(1) << st.op.k;
            std::vector<unsigned char> buf(D * D * eb);
            for (size_t e = 0; e < D * D; ++e) {
                if (dtype == QSIM_C64) {
                    float v[2] = {float(st.op.m[e].real()), float(st.op.m[e].imag())};
                    memcpy(&buf[e * eb], v, 8);
                } else {
                    double v[2] = {st.op.m[e].real(), st.op.m[e].imag()};
                    memcpy(&buf[e * eb], v, 16);
                }
            }
            QSIM_CUDA_TRY(cudaMalloc(&d.plain_mats[i], buf.size()), "stage plain matrix");
            QSIM_CUDA_TRY(cudaMemcpy(d.plain_mats[i], buf.data(), buf.size(), cudaMemcpyHostToDevice),
                          "stage plain matrix upload");
            continue;
        }
        d.param_off[i] = d.params.size();
        d.params.resize(d.params.size() + psz);
        if (dtype == QSIM_C64)
            make_params<float2>(st, *reinterpret_cast<StageParams<float2> *>(&d.params[d.param_off[i]]));
        else
            make_params<double2>(st, *reinterpret_cast<StageParams<double2> *>(&d.params[d.param_off[i]]));
    }
    d.ready = true;
    return QSIM_OK;
}

template <typename R, int W>
static int launch_stage_w(void *psi, int n, const StageParams<typename CT<R>::T> &prm, cudaStream_t s) {
    using C = typename CT<R>::T;
    const int nt = LANE_BITS + REG_BITS + W;
    const uint64_t ntiles = uint64_t(1) << (n - nt);
    const size_t smem = (size_t(1) << nt) * sizeof(C);
    static bool attr_set = false;
    if (!attr_set) {
        QSIM_CUDA_TRY(cudaFuncSetAttribute(k_stage<R, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                      "stage smem attribute");
        attr_set = true;
    }
    LaunchScope ls(K_STAGE, s, 2.0 * double(uint64_t(1) << n) * sizeof(C));
    k_stage<R, W><<<unsigned(ntiles), 32 << W, smem, s>>>(static_cast<C *>(psi), prm);
    QSIM_CUDA_TRY(cudaGetLastError(), "stage launch");
    return QSIM_OK;
}

template <typename R>
static int launch_stage(void *psi, int n, int W, const void *params, cudaStream_t s) {
    using C = typename CT<R>::T;
    const StageParams<C> &prm = *static_cast<const StageParams<C> *>(params);
    switch (W) {
        case 0: return launch_stage_w<R, 0>(psi, n, prm, s);
        case 1: return launch_stage_w<R, 1>(psi, n, prm, s);
        case 2: return launch_stage_w<R, 2>(psi, n, prm, s);
        case 3: return launch_stage_w<R, 3>(psi, n, prm, s);
        default: return launch_stage_w<R, 4>(psi, n, prm, s);
    }
}

int run_staged(qsim_state *s, qsim_plan &p) {
    if (!p.staged) return run_block_plan(s, p);
    QSIM_TRY(prepare_staged(p, s->dtype));
    StagedPlan &sp = *p.staged;
    const StagedPlan::Dev &d = sp.dev[s->dtype];
    for (size_t i = 0; i < sp.stages.size(); ++i) {
        const Stage &st = sp.stages[i];
        if (st.plain) {
            QSIM_TRY(launch_op(s->amps, s->n, s->dtype, st.op, s->stream, d.plain_mats[i]));
            continue;
        }
        const void *prm = &d.params[d.param_off[i]];
        if (s->dtype == QSIM_C64)
            QSIM_TRY(launch_stage<float>(s->amps, s->n, sp.W, prm, s->stream));
        else
            QSIM_TRY(launch_stage<double>(s->amps, s->n, sp.W, prm, s->stream));
    }
    return QSIM_OK;
}

void staged_describe(const qsim_plan &p, std::string &out) {
    if (!p.staged) return;
    char buf[256];
    const StagedPlan &sp = *p.staged;
    snprintf(buf, sizeof buf, "staged plan: %zu stages, tile 2^%d amplitudes (W=%d)\n", sp.stages.size(),
             LANE_BITS + REG_BITS + sp.W, sp.W);
    out += buf;
    for (size_t i = 0; i < sp.stages.size(); ++i) {
        const Stage &st = sp.stages[i];
        if (st.plain) {
            snprintf(buf, sizeof buf, "  %3zu plain sweep: k=%d c=%d\n", i, st.op.k, st.op.c);
            out += buf;
            continue;
        }
        int cnt[4] = {0, 0, 0, 0}, lane_u1 = 0;
        for (const StageOp &o : st.ops) {
            cnt[int(o.type)]++;
            if (o.type == SOP_U1 && o.a < POS_REG) ++lane_u1;
        }
        std::string sl;
        for (int q : st.slots) sl += std::to_string(q) + " ";
        snprintf(buf, sizeof buf, "  %3zu tile [%s]: u1=%d (lane %d) u2=%d diag=%d exchange=%d\n", i, sl.c_str(),
                 cnt[SOP_U1], lane_u1, cnt[SOP_U2], cnt[SOP_DIAG], cnt[SOP_EXCHANGE]);
        out += buf;
    }
}

int staged_nsweeps(const qsim_plan &p) { return p.staged ? int(p.staged->stages.size()) : int(p.blocks.size()); }

}  // namespace qsim

void qsim_plan::release_staged() {
    delete staged;
    staged = nullptr;
}

int qsim_plan::nsweeps() const {
    if (mode == QSIM_FUSE_STAGED) return qsim::staged_nsweeps(*this);
    if (mode == QSIM_FUSE_TC) return qsim::tc_nsweeps(*this);
    return int(blocks.size());
}

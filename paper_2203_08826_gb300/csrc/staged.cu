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
#include <cstdlib>
#include <cstring>
#include <string>

#include "internal.h"
#include "plan.h"
#include "stage_common.cuh"

namespace qsim {

namespace stage {

namespace {

template <typename C> struct ParamSrc {
    const StageParams<C> &p;
    __device__ const StageOp &op(int o) const { return p.ops[o]; }
    __device__ const Phase &phase(int i) const { return p.phases[i]; }
    __device__ C pool(int i) const { return p.pool[i]; }
    __device__ uint64_t aux(int i) const { return p.aux[i]; }
};

#ifdef QSIM_DEBUG
static __device__ unsigned long long g_staged_oob;
#endif

template <typename R, int W>
__global__ void __launch_bounds__(32 << W, (sizeof(R) == 4 ? (W <= 3 ? 3 : 2) : 1))
    k_stage(typename CT<R>::T *__restrict__ psi, const __grid_constant__ StageParams<typename CT<R>::T> p) {
    using C = typename CT<R>::T;
    extern __shared__ unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint64_t tile_base = expand(blockIdx.x, p.outer);
    int ph = p.phase0;
    uint64_t base = thread_base<W>(p.phases[ph], tile_base, lane, warp);
    C v[1 << REG_BITS];
#ifdef QSIM_DEBUG
    // every index this thread loads and stores (the same set: the final
    // phase permutes registers within the tile) must lie inside the state;
    // a thread with one outside computes on zeros and stores nothing, but
    // still takes part in the CTA's exchanges
    bool inside = true;
    {
        uint64_t hi = base;
        for (int b = 0; b < REG_BITS; ++b) hi |= uint64_t(1) << p.phases[ph].rq[b];
        if (p.outer.limit && hi >= p.outer.limit) {
            atomicAdd(&g_staged_oob, 1ull);
            inside = false;
        }
    }
    if (inside) tile_global<C, W, false>(psi, v, p.phases[ph], base);
    else
        for (int j = 0; j < (1 << REG_BITS); ++j) v[j] = C{0, 0};
#else
    tile_global<C, W, false>(psi, v, p.phases[ph], base);
#endif
    const ParamSrc<C> src{p};
    stage_exec<C, W>(src, p.nops, v, ph, base, tile_base, tile, lane, warp);
#ifdef QSIM_DEBUG
    if (inside)
#endif
        tile_global<C, W, true>(psi, v, p.phases[ph], base);
}

// ------------------------------------------------------------------ host plan
uint64_t qmask(const int *q, int n) {
    uint64_t m = 0;
    for (int i = 0; i < n; ++i) m |= uint64_t(1) << q[i];
    return m;
}

// Merge adjacent ops that need no ordering among themselves: uncontrolled
// 1-qubit gates on distinct register bits (or distinct lane bits) commute, and
// so do sign flips.  One merged op costs one dispatch instead of several.
void batch_ops(Stage &st) {
    std::vector<StageOp> out;
    std::vector<cd> pool;
    const auto &in = st.ops;
    size_t i = 0;
    auto plain_u1 = [](const StageOp &o) { return o.type == SOP_U1 && o.tmask == 0 && o.rneed == 0; };
    while (i < in.size()) {
        const StageOp &o = in[i];
        if (plain_u1(o) || o.type == SOP_GRAD) {
            // a run of uncontrolled 1-qubit gates on distinct positions
            // commutes: one batched op for its register targets, one for its
            // lane targets.  Gradient ops in the run go first (each commutes
            // with the gates on other positions; the run ends before one
            // whose position a gate of the run already touched).
            size_t j = i;
            int rmask = 0, lmask = 0;
            while (j < in.size() && (plain_u1(in[j]) || in[j].type == SOP_GRAD)) {
                const bool reg = in[j].a >= POS_REG;
                const int b = reg ? in[j].a - POS_REG : in[j].a;
                int &mask = reg ? rmask : lmask;
                if (mask & (1 << b)) break;
                if (in[j].type != SOP_GRAD) mask |= 1 << b;
                ++j;
            }
            for (size_t t = i; t < j; ++t)
                if (in[t].type == SOP_GRAD) out.push_back(in[t]);
            for (int cls = 0; cls < 2; ++cls) {
                const bool reg = cls == 0;
                const int mask = reg ? rmask : lmask;
                if (!mask) continue;
                if (__builtin_popcount(unsigned(mask)) == 1) {
                    for (size_t t = i; t < j; ++t)
                        if (in[t].type == SOP_U1 && (in[t].a >= POS_REG) == reg) {
                            StageOp c = in[t];
                            c.moff = int(pool.size());
                            pool.insert(pool.end(), st.pool.begin() + in[t].moff, st.pool.begin() + in[t].moff + 4);
                            out.push_back(c);
                        }
                    continue;
                }
                StageOp m{};
                m.type = reg ? SOP_U1R : SOP_U1L;
                m.a = int8_t(mask);
                m.moff = int(pool.size());
                // matrices in increasing bit order
                for (int b = 0; b < 8; ++b)
                    for (size_t t = i; t < j; ++t) {
                        if (in[t].type != SOP_U1 || (in[t].a >= POS_REG) != reg) continue;
                        const int tb = reg ? in[t].a - POS_REG : in[t].a;
                        if (tb == b) pool.insert(pool.end(), st.pool.begin() + in[t].moff, st.pool.begin() + in[t].moff + 4);
                    }
                out.push_back(m);
            }
            i = j;
            continue;
        }
        if (o.type == SOP_DIAG && o.k == 0 && (o.flags & 1)) {
            size_t j = i;
            while (j < in.size() && in[j].type == SOP_DIAG && in[j].k == 0 && (in[j].flags & 1)) ++j;
            if (j - i >= 2) {
                StageOp m{};
                m.type = SOP_NEG;
                m.k = int8_t(std::min<size_t>(j - i, 127));
                j = i + size_t(m.k);
                m.moff = int(st.aux.size());
                for (size_t t = i; t < j; ++t) {
                    uint64_t pat = 0;
                    for (int r = 0; r < (1 << REG_BITS); ++r)
                        if ((r & in[t].rneed) == in[t].rneed) pat |= uint64_t(1) << r;
                    st.aux.push_back(in[t].tmask);
                    st.aux.push_back(pat);
                }
                out.push_back(m);
                i = j;
                continue;
            }
        }
        StageOp c = o;
        if (o.type == SOP_U1 || o.type == SOP_U2 || o.type == SOP_DIAG) {
            const int cnt = o.type == SOP_U1 ? 4 : o.type == SOP_U2 ? 16 : (1 << o.k);
            c.moff = int(pool.size());
            pool.insert(pool.end(), st.pool.begin() + o.moff, st.pool.begin() + o.moff + cnt);
        }
        out.push_back(c);
        ++i;
    }
    st.ops.swap(out);
    st.pool.swap(pool);
}

// Coefficients of a dense 4x4 U (row-major, index (bit A << 1) | bit B, A =
// the first target) with a target on a lane, in the order the kernel reads
// them (each thread holds its own amplitudes and gets its partner lanes' by
// shuffle):
//   one lane target: for lane-bit value beta = 0, 1 and the thread's output
//     register value r = 0, 1: the coefficients of (own, register 0), (own,
//     register 1), (partner, register 0), (partner, register 1);
//   two lane targets: for the lane's values (bit A, bit B) = 00, 01, 10, 11:
//     the coefficients of its own amplitude and of the lanes across bit A,
//     across bit B and across both.
static std::vector<cd> lane_u2_layout(const std::vector<cd> &U, bool lane_a, bool lane_b) {
    std::vector<cd> out;
    out.reserve(16);
    if (lane_a && lane_b) {
        for (int r = 0; r < 4; ++r)
            for (int flip : {0, 2, 1, 3}) out.push_back(U[size_t(r * 4 + (r ^ flip))]);
        return out;
    }
    // idx(beta, rho): matrix index of lane-bit value beta and register-bit value rho
    auto idx = [&](int beta, int rho) { return lane_a ? (beta << 1) | rho : (rho << 1) | beta; };
    for (int beta = 0; beta < 2; ++beta)
        for (int rho = 0; rho < 2; ++rho) {
            const int row = idx(beta, rho);
            for (int c : {idx(beta, 0), idx(beta, 1), idx(1 - beta, 0), idx(1 - beta, 1)})
                out.push_back(U[size_t(row * 4 + c)]);
        }
    return out;
}

// Build the op list of one tile stage from its gates (circuit order).
// Returns QSIM_EUNSUPPORTED (without error text) when the stage outgrows the
// parameter-block limits; the caller then splits it.
int emit_stage_ops(Stage &st, const std::vector<const GateClass *> &gates, int W, bool limits) {
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
        if (so.type == SOP_U1 || so.type == SOP_GRAD) return so.a == pos_of(q);
        if (so.type == SOP_U2) return so.a == pos_of(q) || so.b == pos_of(q);
        if (so.type == SOP_DIAG)
            for (int t = 0; t < so.k; ++t)
                if (so.dq[t] == (b >= 0 ? POS_REG + b : POS_BASE + q)) return true;
        return false;
    };
    // index of a preceding uncontrolled U1 on q (or, with `diag`, an
    // uncontrolled 1-qubit diagonal on q) that nothing after it touches, or -1
    auto mergeable_u1 = [&](int q, bool diag) -> int {
        const int b = reg_bit(q);
        const int8_t dpos = int8_t(b >= 0 ? POS_REG + b : POS_BASE + q);
        for (size_t o = st.ops.size(); o-- > phase_first_op;) {
            const StageOp &prev = st.ops[o];
            if (!touches(prev, q)) continue;
            if (prev.tmask != 0 || prev.rneed != 0) return -1;
            if (prev.type == SOP_U1 && prev.a == pos_of(q)) return int(o);
            if (diag && prev.type == SOP_DIAG && prev.k == 1 && prev.dq[0] == dpos) return int(o);
            return -1;
        }
        return -1;
    };
    for (size_t i = 0; i < gates.size(); ++i) {
        const GateClass &g = *gates[i];
        if (g.kind == GateClass::DIAG) {
            if (g.op.k == 1 && g.op.c == 0) {
                // fold an uncontrolled 1-qubit diagonal into a preceding U1 on its qubit
                const int mi = pos_of(g.op.targets[0]) >= 0 ? mergeable_u1(g.op.targets[0], false) : -1;
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
            // register selector bits: nibble r of (b:a) holds 1 + the selector
            // bit that register bit r feeds (0: none)
            uint32_t pk = 0;
            for (int t = 0; t < g.op.k; ++t) {
                const int q = g.op.targets[t];
                const int b = reg_bit(q);
                so.dq[t] = int8_t(b >= 0 ? POS_REG + b : POS_BASE + q);
                if (b >= 0) pk |= uint32_t(g.op.k - t) << (4 * b);
            }
            so.a = int8_t(pk & 0xFF);
            so.b = int8_t((pk >> 8) & 0xFF);
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
        if (g.grad_slot >= 0) {
            // terms on one qubit with nothing touching it in between share one op
            const int q = g.op.targets[0];
            int gop = -1;
            for (size_t o = st.ops.size(); o-- > phase_first_op;) {
                const StageOp &prev = st.ops[o];
                if (prev.type == SOP_GRAD && prev.a == pos_of(q) && prev.tmask == 0 && prev.rneed == 0) {
                    gop = prev.k;
                    break;
                }
                if (touches(prev, q)) break;
            }
            if (gop < 0) {
                so.type = SOP_GRAD;
                so.a = int8_t(pos_of(q));
                so.k = int8_t(std::min(st.ngradops, 127));
                gop = st.ngradops++;
                st.ops.push_back(so);
            }
            st.grads.push_back({g.grad_slot, gop, {g.grad_v[0], g.grad_v[1], g.grad_v[2]}});
            continue;
        }
        if (g.kind == GateClass::DENSE1) {
            so.type = SOP_U1;
            so.a = int8_t(pos_of(g.op.targets[0]));
            if (so.tmask == 0 && so.rneed == 0) {
                const int mi = mergeable_u1(g.op.targets[0], true);
                if (mi >= 0) {
                    StageOp &prev = st.ops[mi];
                    if (prev.type == SOP_DIAG) {  // U diag(d0, d1) becomes one U1
                        const cd d0 = st.pool[prev.moff], d1 = st.pool[prev.moff + 1];
                        const std::vector<cd> &u = g.op.m;
                        StageOp m1 = so;
                        m1.moff = add_pool({u[0] * d0, u[1] * d1, u[2] * d0, u[3] * d1});
                        prev = m1;
                        continue;
                    }
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
            if (so.a < POS_REG || so.b < POS_REG) {
                so.moff = add_pool(lane_u2_layout(g.op.m, so.a < POS_REG, so.b < POS_REG));
                st.ops.push_back(so);
                continue;
            }
        }
        so.moff = add_pool(g.op.m);
        st.ops.push_back(so);
    }
    batch_ops(st);
    if (limits && (st.ops.size() > size_t(MAX_OPS) || st.phases.size() > size_t(MAX_PHASES) ||
                   st.pool.size() > size_t(MAX_POOL) || st.aux.size() > size_t(2 * MAX_AUX) ||
                   st.grads.size() > size_t(MAX_GRAD)))
        return QSIM_EUNSUPPORTED;
    return QSIM_OK;
}

}  // namespace

// Algorithmic flops per amplitude of a stage: those of the circuit's gates it
// applies, each counted as one sweep would apply it (a dense k-qubit gate with
// c controls: 2^k complex multiply-adds of 8 flops on 1/2^c of the
// amplitudes; a diagonal or permutation gate: one complex multiply of 6 flops
// per amplitude it touches, none when every factor is +-1 or 1).  Fused
// 4x4 blocks and merged diagonals do fewer flops than this; the count is
// the workload's, not the plan's.
// Flops per amplitude a stage's ops execute (a complex multiply-add is 8
// flops; a controlled op counts for the fraction of amplitudes it touches;
// sign flips and exchanges none): the work of the plan as fused.
double stage_exec_flops_per_amp(const Stage &st) {
    if (st.plain) return st.op.type == Op::DENSE ? 8.0 * double(1 << st.op.k) / double(1ull << st.op.c) : 0.0;
    double f = 0;
    for (const StageOp &o : st.ops) {
        const double frac = 1.0 / double(1ull << (__builtin_popcountll(o.tmask) + __builtin_popcount(o.rneed)));
        if (o.type == SOP_U1) f += 16.0 * frac;
        else if (o.type == SOP_U1R || o.type == SOP_U1L) f += 16.0 * __builtin_popcount(unsigned(o.a));
        else if (o.type == SOP_U2) f += 32.0 * frac;
        else if (o.type == SOP_DIAG && !(o.flags & 1)) f += 6.0 * frac;
    }
    return f;
}

double stage_flops_per_amp(const qsim_circuit &c, const Stage &st) {
    double f = 0;
    for (int gi : st.gates) {
        const GateRec &g = c.gates[size_t(gi)];
        if (g.grad_slot >= 0) continue;
        Op op;
        if (classify(g.m, g.targets, g.k, g.controls, g.nc, op) != QSIM_OK) continue;
        const double frac = 1.0 / double(1ull << op.c);
        if (op.type == Op::DENSE) {
            f += 8.0 * double(1 << op.k) * frac;
        } else if (op.type == Op::DIAG || op.type == Op::MONO) {
            const std::vector<cd> &e = op.type == Op::DIAG ? op.m : op.phase;
            bool sign_only = true;
            for (const cd &x : e) sign_only &= x.imag() == 0.0 && (x.real() == 1.0 || x.real() == -1.0);
            if (!sign_only) f += 6.0 * frac;
        }
    }
    return f;
}

// Pair fusion before staging: an uncontrolled 2-qubit gate M on qubits a, b
// absorbs the run of uncontrolled 1-qubit gates just before it on a (every
// gate on a between the previous multi-qubit gate on a and M), the same run
// on b, and the runs just after it on a and on b.  Each run touches only its
// own qubit, so moving it next to M crosses only gates it commutes with, and
// its product is one 2x2: U = (Ha x Hb) M (Ga x Gb) is one dense 4x4 at M's
// place.  A 4x4 costs 16 multiply-adds per amplitude, a 1-qubit op 8, and a
// 1-qubit diagonal merges into a neighbouring 1-qubit op for nothing; so M is
// fused only when at least three of its four runs hold a non-diagonal gate.
// Gates are taken greedily in circuit order, each 1-qubit gate absorbed at
// most once.  src[i] lists the source gates of fused gate i in an order that
// applies them correctly (the runs before M in circuit order, M, the runs
// after M in circuit order).
static void pair_fuse(const qsim_circuit &c, std::vector<GateRec> &gates, std::vector<std::vector<int>> &src) {
    const size_t G = c.gates.size();
    auto touches = [&](size_t i, int q) {
        const GateRec &g = c.gates[i];
        for (int t = 0; t < g.k; ++t)
            if (g.targets[t] == q) return true;
        for (int t = 0; t < g.nc; ++t)
            if (g.controls[t] == q) return true;
        return false;
    };
    auto plain1 = [&](size_t i) {
        const GateRec &g = c.gates[i];
        return g.k == 1 && g.nc == 0 && g.grad_slot < 0;
    };
    auto diagonal = [&](size_t i) { return c.gates[i].m[1] == cd(0.0) && c.gates[i].m[2] == cd(0.0); };
    const std::vector<cd> I2 = {1.0, 0.0, 0.0, 1.0};
    std::vector<char> absorbed(G, 0);
    std::vector<std::vector<int>> parts(G);  // fused 2-qubit gate -> its source gates
    std::vector<std::vector<cd>> fusedm(G);
    for (size_t i = 0; i < G; ++i) {
        const GateRec &g = c.gates[i];
        if (g.k != 2 || g.nc != 0 || g.grad_slot >= 0) continue;
        std::vector<int> prev[2], next[2];  // circuit order
        int have = 0;
        for (int t = 0; t < 2; ++t) {
            const int q = g.targets[t];
            for (size_t j = i; j-- > 0;) {
                if (!touches(j, q)) continue;
                if (!plain1(j) || absorbed[j]) break;
                prev[t].insert(prev[t].begin(), int(j));
            }
            for (size_t j = i + 1; j < G; ++j) {
                if (!touches(j, q)) continue;
                if (!plain1(j)) break;
                next[t].push_back(int(j));
            }
            for (const std::vector<int> *run : {&prev[t], &next[t]}) {
                bool dense = false;
                for (int j : *run) dense |= !diagonal(size_t(j));
                have += dense;
            }
        }
        if (have < 3) continue;
        auto product = [&](const std::vector<int> &run) {  // later gates on the left
            std::vector<cd> P = I2;
            for (int j : run) P = matmul(c.gates[size_t(j)].m, P, 2);
            return P;
        };
        auto kron = [](const std::vector<cd> &A, const std::vector<cd> &B) {  // A on the MSB
            std::vector<cd> K(16);
            for (int r = 0; r < 4; ++r)
                for (int q = 0; q < 4; ++q) K[size_t(r * 4 + q)] = A[size_t((r >> 1) * 2 + (q >> 1))] * B[size_t((r & 1) * 2 + (q & 1))];
            return K;
        };
        std::vector<cd> U = matmul(g.m, kron(product(prev[0]), product(prev[1])), 4);
        U = matmul(kron(product(next[0]), product(next[1])), U, 4);
        fusedm[i] = U;
        std::vector<int> before(prev[0]), after(next[0]);
        before.insert(before.end(), prev[1].begin(), prev[1].end());
        after.insert(after.end(), next[1].begin(), next[1].end());
        std::sort(before.begin(), before.end());
        std::sort(after.begin(), after.end());
        parts[i] = before;
        parts[i].push_back(int(i));
        parts[i].insert(parts[i].end(), after.begin(), after.end());
        for (const std::vector<int> &run : {prev[0], prev[1], next[0], next[1]})
            for (int j : run) absorbed[size_t(j)] = 1;
    }
    gates.clear();
    src.clear();
    for (size_t i = 0; i < G; ++i) {
        if (absorbed[i]) continue;
        GateRec r = c.gates[i];
        if (!parts[i].empty()) {
            r.kind = QSIM_GATE_MATRIX;
            r.pindex = -1;
            r.m = fusedm[i];
            src.push_back(parts[i]);
        } else {
            src.push_back({int(i)});
        }
        gates.push_back(std::move(r));
    }
}

int plan_stage_list(const qsim_circuit &c0, int W, bool limits, std::vector<Stage> &out, bool lookahead) {
    // pair fusion first, except for the reverse sweep of the adjoint method,
    // whose gradient markers must stay between the gates they sit between
    qsim_circuit fused;
    std::vector<std::vector<int>> src;
    const bool use_fused = [&] {
        for (const GateRec &g : c0.gates)
            if (g.grad_slot >= 0) return false;
        return true;
    }();
    if (use_fused) {
        fused.n = c0.n;
        fused.nparams = c0.nparams;
        pair_fuse(c0, fused.gates, src);
    }
    const qsim_circuit &c = use_fused ? fused : c0;
    auto source = [&](int gi, std::vector<int> &dst) {
        if (use_fused) dst.insert(dst.end(), src[size_t(gi)].begin(), src[size_t(gi)].end());
        else dst.push_back(gi);
    };
    const int n = c.n;
    const int cap = REG_BITS + W;
    std::vector<GateClass> cls(c.gates.size());
    for (size_t i = 0; i < c.gates.size(); ++i) {
        const GateRec &g = c.gates[i];
        if (g.grad_slot >= 0) {
            // adjoint gradient marker: needs its qubit in the tile like a 1-qubit gate
            cls[i].kind = GateClass::DENSE1;
            cls[i].op = Op{};
            cls[i].op.type = Op::DENSE;
            cls[i].op.k = 1;
            cls[i].op.targets[0] = g.targets[0];
            cls[i].op.m = {1.0, 0.0, 0.0, 1.0};
            cls[i].grad_slot = g.grad_slot;
            for (int t = 0; t < 3; ++t) cls[i].grad_v[t] = g.grad_v[t];
            continue;
        }
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
            if (op.k == 1) cls[i].kind = GateClass::DENSE1;
            else if (op.k == 2) cls[i].kind = GateClass::DENSE2;
            else cls[i].kind = GateClass::OTHER;
        }
    }
    std::vector<int> remaining(c.gates.size());
    for (size_t i = 0; i < remaining.size(); ++i) remaining[i] = int(i);
    size_t limit = remaining.size();  // largest number of gates one stage may take
    while (!remaining.empty()) {
        // a leading gate no tile holds (more than two dense targets) runs as a
        // plain sweep of its own
        if (cls[size_t(remaining[0])].kind == GateClass::OTHER) {
            const int g0 = remaining[0];
            Stage st;
            st.plain = true;
            st.op = cls[size_t(g0)].op;
            source(g0, st.gates);
            out.push_back(std::move(st));
            remaining.erase(remaining.begin());
            limit = remaining.size();
            continue;
        }
        // Fill the tile (lookahead): repeatedly take, among the gates that
        // commute with every earlier gate not yet taken (none of those touches
        // their qubits), the one that adds the fewest new tile qubits (gates
        // already inside the tile and diagonal gates first, in circuit order).
        // Any prefix of the picks is an order-respecting schedule.
        std::vector<int> tile, sched, rest;
        if (!lookahead) {
            // one pass in circuit order: each gate that fits joins the tile;
            // one that does not is deferred and blocks its qubits
            uint64_t blocked = 0;
            for (int gi : remaining) {
                const GateClass &g = cls[size_t(gi)];
                const uint64_t qs = qmask(g.op.targets, g.op.k) | qmask(g.op.controls, g.op.c);
                bool take = !(qs & blocked) && sched.size() < limit && g.kind != GateClass::OTHER;
                std::vector<int> add;
                if (take && g.kind != GateClass::DIAG) {
                    for (int t = 0; t < g.op.k; ++t) {
                        const int q = g.op.targets[t];
                        if (q >= LANE_BITS && std::find(tile.begin(), tile.end(), q) == tile.end()) add.push_back(q);
                    }
                    take = int(tile.size() + add.size()) <= cap;
                }
                if (take) {
                    tile.insert(tile.end(), add.begin(), add.end());
                    sched.push_back(gi);
                } else {
                    blocked |= qs;
                    rest.push_back(gi);
                }
            }
        } else {
            rest = remaining;
        }
        while (lookahead && sched.size() < limit) {
            uint64_t blocked = 0;
            int best = -1, best_add = 1 << 30;
            for (size_t r = 0; r < rest.size(); ++r) {
                const GateClass &g = cls[size_t(rest[r])];
                const uint64_t qs = qmask(g.op.targets, g.op.k) | qmask(g.op.controls, g.op.c);
                if (qs & blocked) {
                    blocked |= qs;
                    continue;
                }
                blocked |= qs;  // later gates on these qubits wait for this one
                if (g.kind == GateClass::OTHER) continue;
                int add = 0;
                if (g.kind != GateClass::DIAG)
                    for (int t = 0; t < g.op.k; ++t) {
                        const int q = g.op.targets[t];
                        if (q >= LANE_BITS && std::find(tile.begin(), tile.end(), q) == tile.end()) ++add;
                    }
                if (int(tile.size()) + add > cap || add >= best_add) continue;
                best = int(r);
                best_add = add;
                if (add == 0) break;
            }
            if (best < 0) break;
            const int gi = rest[size_t(best)];
            rest.erase(rest.begin() + best);
            const GateClass &g = cls[size_t(gi)];
            if (g.kind != GateClass::DIAG)
                for (int t = 0; t < g.op.k; ++t) {
                    const int q = g.op.targets[t];
                    if (q >= LANE_BITS && std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
                }
            sched.push_back(gi);
        }
        if (sched.empty()) return set_error(QSIM_EINVAL, "staged planner: no gate fits a tile");
        for (int q = LANE_BITS; q < n && int(tile.size()) < cap; ++q)
            if (std::find(tile.begin(), tile.end(), q) == tile.end()) tile.push_back(q);
        Stage st;
        st.slots = tile;
        for (int gi : sched) source(gi, st.gates);
        std::vector<const GateClass *> gl;
        for (int gi : sched) gl.push_back(&cls[gi]);
        const int rc = emit_stage_ops(st, gl, W, limits);
        if (rc == QSIM_EUNSUPPORTED) {
            // too many ops for one parameter block: retry with half the gates
            // (the same picks, cut short: a prefix of the picks is an
            // order-respecting schedule too)
            limit = std::max<size_t>(1, sched.size() / 2);
            std::vector<int> merged(sched);
            merged.insert(merged.end(), rest.begin(), rest.end());
            std::sort(merged.begin(), merged.end());
            remaining.swap(merged);
            continue;
        }
        QSIM_TRY(rc);
        out.push_back(std::move(st));
        remaining.swap(rest);
        limit = remaining.size();
    }
    return QSIM_OK;
}

}  // namespace stage

using namespace stage;

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
    sp->W = std::min(std::min(p.kmax, MAX_WARP_BITS), n - LANE_BITS - REG_BITS);
    QSIM_TRY(plan_stage_list(c, sp->W, true, sp->stages));
    for (const Stage &st : sp->stages) {
        sp->flops_per_amp.push_back(stage_exec_flops_per_amp(st));
        sp->circuit_flops_per_amp += stage_flops_per_amp(c, st);
    }
    return QSIM_OK;
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
            QSIM_CUDA_TRY(dev_alloc(&d.plain_mats[i], buf.size()), "stage plain matrix");
            QSIM_CUDA_TRY(cudaMemcpy(d.plain_mats[i], buf.data(), buf.size(), cudaMemcpyHostToDevice),
                          "stage plain matrix upload");
            continue;
        }
        d.param_off[i] = d.params.size();
        d.params.resize(d.params.size() + psz);
        if (dtype == QSIM_C64) {
            auto &prm = *reinterpret_cast<StageParams<float2> *>(&d.params[d.param_off[i]]);
            make_params<float2>(st, prm);
            prm.outer.limit = uint64_t(1) << p.n;
        } else {
            auto &prm = *reinterpret_cast<StageParams<double2> *>(&d.params[d.param_off[i]]);
            make_params<double2>(st, prm);
            prm.outer.limit = uint64_t(1) << p.n;
        }
    }
    d.ready = true;
    return QSIM_OK;
}

template <typename R, int W>
static int launch_stage_w(void *psi, int n, const StageParams<typename CT<R>::T> &prm, cudaStream_t s, double fpa) {
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
    LaunchScope ls(K_STAGE, s, 2.0 * double(uint64_t(1) << n) * sizeof(C), fpa * double(uint64_t(1) << n));
    k_stage<R, W><<<unsigned(ntiles), 32 << W, smem, s>>>(static_cast<C *>(psi), prm);
    QSIM_CUDA_TRY(cudaGetLastError(), "stage launch");
    return QSIM_OK;
}

template <typename R>
static int launch_stage(void *psi, int n, int W, const void *params, cudaStream_t s, double fpa) {
    using C = typename CT<R>::T;
    const StageParams<C> &prm = *static_cast<const StageParams<C> *>(params);
    switch (W) {
        case 0: return launch_stage_w<R, 0>(psi, n, prm, s, fpa);
        case 1: return launch_stage_w<R, 1>(psi, n, prm, s, fpa);
        case 2: return launch_stage_w<R, 2>(psi, n, prm, s, fpa);
        case 3: return launch_stage_w<R, 3>(psi, n, prm, s, fpa);
        default: return launch_stage_w<R, 4>(psi, n, prm, s, fpa);
    }
}

int run_staged(qsim_state *s, qsim_plan &p) {
    if (!p.staged) return run_block_plan(s, p);
    QSIM_TRY(prepare_staged(p, s->dtype));
    if (p.staged->specialized) QSIM_TRY(spec_prepare(*p.staged, s->dtype));
    StagedPlan &sp = *p.staged;
    const StagedPlan::Dev &d = sp.dev[s->dtype];
    for (size_t i = 0; i < sp.stages.size(); ++i) {
        const Stage &st = sp.stages[i];
        if (st.plain) {
            QSIM_TRY(launch_op(s->amps, s->n, s->dtype, st.op, s->stream, d.plain_mats[i]));
            continue;
        }
        if (sp.specialized) {
            QSIM_TRY(spec_launch(sp, s->dtype, i, s->amps, s->n, s->stream));
            continue;
        }
        const void *prm = &d.params[d.param_off[i]];
        if (s->dtype == QSIM_C64)
            QSIM_TRY(launch_stage<float>(s->amps, s->n, sp.W, prm, s->stream, sp.flops_per_amp[i]));
        else
            QSIM_TRY(launch_stage<double>(s->amps, s->n, sp.W, prm, s->stream, sp.flops_per_amp[i]));
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
        int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lane_u1 = 0;
        for (const StageOp &o : st.ops) {
            cnt[int(o.type)]++;
            if (o.type == SOP_U1 && o.a < POS_REG) ++lane_u1;
        }
        std::string sl;
        for (int q : st.slots) sl += std::to_string(q) + " ";
        snprintf(buf, sizeof buf,
                 "  %3zu tile [%s]: u1=%d (lane %d) u1-batches reg=%d lane=%d u2=%d diag=%d sign-batches=%d exchange=%d\n",
                 i, sl.c_str(), cnt[SOP_U1], lane_u1, cnt[SOP_U1R], cnt[SOP_U1L], cnt[SOP_U2], cnt[SOP_DIAG], cnt[SOP_NEG],
                 cnt[SOP_EXCHANGE]);
        out += buf;
    }
}

void staged_set_specialized(qsim_plan &p) {
    if (p.staged) p.staged->specialized = true;  // narrower circuits got a greedy plan
}
bool staged_specialized(const qsim_plan &p) { return p.staged && p.staged->specialized; }

extern "C" QSIM_API int qsim_plan_flops(const qsim_plan *p, double *executed, double *circuit) {
    if (!p || !p->staged) return qsim::set_error(QSIM_EINVAL, "not a staged plan");
    double e = 0;
    for (double f : p->staged->flops_per_amp) e += f;
    if (executed) *executed = e;
    if (circuit) *circuit = p->staged->circuit_flops_per_amp;
    return QSIM_OK;
}

int staged_nsweeps(const qsim_plan &p) { return p.staged ? int(p.staged->stages.size()) : int(p.blocks.size()); }

unsigned long long staged_debug_oob(bool clear) {
#ifdef QSIM_DEBUG
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, stage::g_staged_oob, sizeof v);
    if (clear) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(stage::g_staged_oob, &z, sizeof z);
    }
    return v;
#else
    (void)clear;
    return 0;
#endif
}

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

// ------------------------------------------------------------------ host inspection
extern "C" QSIM_API int qsim_plan_stage(const qsim_plan *p, int i, int *plain, int *ngates, int *gates, int *nslots,
                                        int *slots) {
    using namespace qsim;
    if (!p || !p->staged) return set_error(QSIM_EINVAL, "not a staged plan");
    const std::vector<stage::Stage> &stages = p->staged->stages;
    if (i < 0 || i >= int(stages.size())) return set_error(QSIM_EINVAL, "stage %d outside the plan", i);
    const stage::Stage &st = stages[size_t(i)];
    if (plain) *plain = st.plain ? 1 : 0;
    if (ngates) *ngates = int(st.gates.size());
    if (gates)
        for (size_t j = 0; j < st.gates.size(); ++j) gates[j] = st.gates[j];
    if (nslots) *nslots = int(st.slots.size());
    if (slots)
        for (size_t j = 0; j < st.slots.size(); ++j) slots[j] = st.slots[j];
    return QSIM_OK;
}

// Stage i of a staged plan as text: the op list the kernels run (for
// checking the planner and the op lists against the gate-by-gate result on
// the host).  Lines:
//   stage <i> plain <0|1> W <W> phase0 <p>
//   slots <q ...>
//   phase <rq0..rq3> | <wq0..wq{W-1}> | <rslot0..3> | <wslot0..>
//   op <type> <a> <b> <k> <rneed> <flags> <tmask> <moff> <dq0..dq5>
//   pool <re> <im>
//   aux <u64>
extern "C" QSIM_API int qsim_plan_stage_dump(const qsim_plan *p, int i, char *buf, size_t len, size_t *needed) {
    using namespace qsim;
    if (!p || !p->staged) return set_error(QSIM_EINVAL, "not a staged plan");
    const std::vector<stage::Stage> &stages = p->staged->stages;
    if (i < 0 || i >= int(stages.size())) return set_error(QSIM_EINVAL, "stage %d outside the plan", i);
    const stage::Stage &st = stages[size_t(i)];
    const int W = p->staged->W;
    std::string o;
    char line[512];
    snprintf(line, sizeof line, "stage %d plain %d W %d phase0 %d\nslots", i, st.plain ? 1 : 0, W, st.phase0);
    o += line;
    for (int q : st.slots) o += " " + std::to_string(q);
    o += "\n";
    for (const stage::Phase &P : st.phases) {
        o += "phase";
        for (int b = 0; b < stage::REG_BITS; ++b) o += " " + std::to_string(int(P.rq[b]));
        o += " |";
        for (int b = 0; b < W; ++b) o += " " + std::to_string(int(P.wq[b]));
        o += " |";
        for (int b = 0; b < stage::REG_BITS; ++b) o += " " + std::to_string(int(P.rslot[b]));
        o += " |";
        for (int b = 0; b < W; ++b) o += " " + std::to_string(int(P.wslot[b]));
        o += "\n";
    }
    for (const stage::StageOp &op : st.ops) {
        snprintf(line, sizeof line, "op %d %d %d %d %d %d %llu %d", int(op.type), int(op.a), int(op.b), int(op.k),
                 int(op.rneed), int(op.flags), (unsigned long long)op.tmask, op.moff);
        o += line;
        for (int t = 0; t < QSIM_MAX_TARGETS; ++t) o += " " + std::to_string(int(op.dq[t]));
        o += "\n";
    }
    for (const cd &c : st.pool) {
        snprintf(line, sizeof line, "pool %.17g %.17g\n", c.real(), c.imag());
        o += line;
    }
    for (uint64_t a : st.aux) o += "aux " + std::to_string((unsigned long long)a) + "\n";
    if (needed) *needed = o.size() + 1;
    if (buf && len) {
        const size_t m = std::min(len - 1, o.size());
        memcpy(buf, o.data(), m);
        buf[m] = 0;
    }
    return QSIM_OK;
}

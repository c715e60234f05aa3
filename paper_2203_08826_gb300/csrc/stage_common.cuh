// Register-tile stage interpreter shared by the staged fusion kernel and the
// batched persistent kernel (see staged.cu for the scheme).
#pragma once

#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace qsim {
namespace stage {

constexpr int LANE_BITS = 5;
constexpr int REG_BITS = 4;  // amplitudes per thread = 16
constexpr int MAX_WARP_BITS = 4;
constexpr int MAX_SLOTS = REG_BITS + MAX_WARP_BITS;
constexpr int MAX_OPS = 192;
constexpr int MAX_PHASES = 24;
constexpr int MAX_POOL = 768;
constexpr int MAX_AUX = 192;  // (thread mask, register pattern) pairs of batched sign flips
constexpr int MAX_GRAD = 96;  // gradient terms (and SOP_GRAD ops) of one reverse-sweep stage

// SOP_U2 on a lane position (a or b < POS_REG): the pool holds the matrix
// rearranged per lane-bit value (lane_u2_layout), 16 entries as for two
// register targets.
// SOP_U1R / SOP_U1L: uncontrolled 1-qubit gates on distinct register / lane
// bits (mask in a, matrices consecutive in the pool, lowest bit first);
// SOP_NEG: sign flips (k pairs in aux from moff): amplitude j of a thread
// flips once per pair with (base & mask) == mask and bit j of the pattern.
// SOP_GRAD: the sums from which the adjoint gradient terms Im<lambda|P|psi> on
// one qubit follow (a = position, k = local index); only the two-state
// executor runs it.
enum SopType : int8_t { SOP_U1 = 0, SOP_U2 = 1, SOP_DIAG = 2, SOP_EXCHANGE = 3, SOP_U1R = 4, SOP_U1L = 5, SOP_NEG = 6, SOP_GRAD = 7 };

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
    uint64_t aux[2 * MAX_AUX];
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

// A dense 4x4 on one lane bit (partner lane = lane ^ lmask) and register bit
// JB: for each register pair the thread's two amplitudes (x0, x1: register
// bit 0, 1) and its partner's (y0, y1) give the thread's two outputs,
// out_r = m[4r] x0 + m[4r+1] x1 + m[4r+2] y0 + m[4r+3] y1, with m the eight
// coefficients the host laid out for this thread's lane-bit value.  Every
// lane takes part in the shuffles; ok / rneed only gate the update.
template <typename C, int JB>
__device__ __forceinline__ void u2_lane_reg(C (&v)[1 << REG_BITS], const C (&m)[8], int lmask, bool ok, int rneed) {
#pragma unroll
    for (int i = 0; i < (1 << REG_BITS); ++i) {
        if (i & (1 << JB)) continue;
        const C x0 = v[i], x1 = v[i | (1 << JB)];
        const C y0 = shfl_c(x0, lmask), y1 = shfl_c(x1, lmask);
        if (!ok || (i & rneed) != rneed) continue;
        v[i] = cmad(m[3], y1, cmad(m[2], y0, cmad(m[1], x1, cmul(m[0], x0))));
        v[i | (1 << JB)] = cmad(m[7], y1, cmad(m[6], y0, cmad(m[5], x1, cmul(m[4], x0))));
    }
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


// One non-exchange op on the 16 amplitudes of a thread whose register 0
// sits at global index `base`, applied to NS tiles at once (v, and w when
// NS = 2: the op is decoded once for both).
#define QSIM_EACH(S, X) for (int S = 0; S < NS; ++S) if (auto &X = S ? w : v; true)
template <typename C, int NS, typename Src>
__device__ __forceinline__ void apply_op2(const StageOp &op, const Src &src, C (&v)[1 << REG_BITS],
                                          C (&w)[1 << REG_BITS], uint64_t base, int lane) {
    constexpr int NR = 1 << REG_BITS;
    const int type = op.type;
    if (type == SOP_U1R) {
        int off = op.moff;
        const int mask = op.a;
#define QSIM_U1R_BIT(J)                                                                                        \
if (mask & (1 << J)) {                                                                                     \
    const C m00 = src.pool(off), m01 = src.pool(off + 1), m10 = src.pool(off + 2), m11 = src.pool(off + 3);  \
    _Pragma("unroll") QSIM_EACH(s, x) u1_reg<C, J, false>(x, m00, m01, m10, m11, 0);                         \
    off += 4;                                                                                              \
}
        QSIM_U1R_BIT(0)
        QSIM_U1R_BIT(1)
        QSIM_U1R_BIT(2)
        QSIM_U1R_BIT(3)
#undef QSIM_U1R_BIT
        return;
    }
    if (type == SOP_U1L) {
        int off = op.moff;
        for (int l = 0; l < LANE_BITS; ++l) {
            if (!(op.a & (1 << l))) continue;
            const int bit = (lane >> l) & 1;
            const C cs = bit ? src.pool(off + 3) : src.pool(off), co = bit ? src.pool(off + 2) : src.pool(off + 1);
            off += 4;
#pragma unroll
            QSIM_EACH(s, x) {
#pragma unroll
                for (int j = 0; j < NR; ++j) x[j] = cmad(co, shfl_c(x[j], 1 << l), cmul(cs, x[j]));
            }
        }
        return;
    }
    if (type == SOP_NEG) {
        uint32_t flip = 0;
        for (int e = 0; e < op.k; ++e) {
            const uint64_t tm = src.aux(op.moff + 2 * e);
            if ((base & tm) == tm) flip ^= uint32_t(src.aux(op.moff + 2 * e + 1));
        }
#pragma unroll
        QSIM_EACH(s, x) {
#pragma unroll
            for (int j = 0; j < NR; ++j)
                if ((flip >> j) & 1) {
                    x[j].x = -x[j].x;
                    x[j].y = -x[j].y;
                }
        }
        return;
    }
    // controls on lane / warp / tile qubits: one test per thread (a lane
    // gate still takes part in the shuffles when its controls are not met)
    const bool tok = (base & op.tmask) == op.tmask;
    const bool on_lanes = op.a < POS_REG || (type == SOP_U2 && op.b < POS_REG);
    if (!tok && !((type == SOP_U1 || type == SOP_U2) && on_lanes)) return;
    const int rneed = op.rneed;
    if (type == SOP_U1) {
        const C m00 = src.pool(op.moff), m01 = src.pool(op.moff + 1);
        const C m10 = src.pool(op.moff + 2), m11 = src.pool(op.moff + 3);
        if (op.a >= POS_REG) {
#pragma unroll
            QSIM_EACH(s, x) {
                switch (op.a - POS_REG) {
                    case 0: u1_reg_dispatch<C, 0>(x, m00, m01, m10, m11, rneed); break;
                    case 1: u1_reg_dispatch<C, 1>(x, m00, m01, m10, m11, rneed); break;
                    case 2: u1_reg_dispatch<C, 2>(x, m00, m01, m10, m11, rneed); break;
                    default: u1_reg_dispatch<C, 3>(x, m00, m01, m10, m11, rneed); break;
                }
            }
        } else {
            const int bit = (lane >> op.a) & 1;
            const C cs = bit ? m11 : m00, co = bit ? m10 : m01;
            const int lm = 1 << op.a;
            if (tok && rneed == 0) {
#pragma unroll
                QSIM_EACH(s, x) {
#pragma unroll
                    for (int j = 0; j < NR; ++j) x[j] = cmad(co, shfl_c(x[j], lm), cmul(cs, x[j]));
                }
            } else {
#pragma unroll
                QSIM_EACH(s, x) {
#pragma unroll
                    for (int j = 0; j < NR; ++j) {
                        const C other = shfl_c(x[j], lm);
                        if (tok && (j & rneed) == rneed) x[j] = cmad(co, other, cmul(cs, x[j]));
                    }
                }
            }
        }
    } else if (type == SOP_U2 && on_lanes && (op.a >= POS_REG || op.b >= POS_REG)) {
        // one lane and one register target: the host stores the 8 coefficients
        // of lane-bit value 0, then those of value 1
        const int la = op.a < POS_REG ? op.a : op.b;
        const int rb = (op.a < POS_REG ? op.b : op.a) - POS_REG;
        const int off = op.moff + 8 * ((lane >> la) & 1);
        C m[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) m[e] = src.pool(off + e);
#pragma unroll
        QSIM_EACH(s, x) {
            switch (rb) {
                case 0: u2_lane_reg<C, 0>(x, m, 1 << la, tok, rneed); break;
                case 1: u2_lane_reg<C, 1>(x, m, 1 << la, tok, rneed); break;
                case 2: u2_lane_reg<C, 2>(x, m, 1 << la, tok, rneed); break;
                default: u2_lane_reg<C, 3>(x, m, 1 << la, tok, rneed); break;
            }
        }
    } else if (type == SOP_U2 && on_lanes) {
        // two lane targets: each amplitude takes its own value and those of
        // the lanes across bit a, bit b and both, with the 4 coefficients
        // the host stored for this lane's (bit a, bit b) values
        const int ma = 1 << op.a, mb = 1 << op.b;
        const int off = op.moff + 4 * ((((lane >> op.a) & 1) << 1) | ((lane >> op.b) & 1));
        const C m0 = src.pool(off), m1 = src.pool(off + 1), m2 = src.pool(off + 2), m3 = src.pool(off + 3);
#pragma unroll
        QSIM_EACH(s, x) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const C p1 = shfl_c(x[j], ma), p2 = shfl_c(x[j], mb), p3 = shfl_c(x[j], ma | mb);
                if (tok && (j & rneed) == rneed) x[j] = cmad(m3, p3, cmad(m2, p2, cmad(m1, p1, cmul(m0, x[j]))));
            }
        }
    } else if (type == SOP_U2) {
        C m[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) m[e] = src.pool(op.moff + e);
#pragma unroll
        QSIM_EACH(s, x) {
            switch ((op.a - POS_REG) * 4 + (op.b - POS_REG)) {
                case 1: u2_reg<C, 0, 1>(x, m, rneed); break;
                case 2: u2_reg<C, 0, 2>(x, m, rneed); break;
                case 3: u2_reg<C, 0, 3>(x, m, rneed); break;
                case 4: u2_reg<C, 1, 0>(x, m, rneed); break;
                case 6: u2_reg<C, 1, 2>(x, m, rneed); break;
                case 7: u2_reg<C, 1, 3>(x, m, rneed); break;
                case 8: u2_reg<C, 2, 0>(x, m, rneed); break;
                case 9: u2_reg<C, 2, 1>(x, m, rneed); break;
                case 11: u2_reg<C, 2, 3>(x, m, rneed); break;
                case 12: u2_reg<C, 3, 0>(x, m, rneed); break;
                case 13: u2_reg<C, 3, 1>(x, m, rneed); break;
                default: u2_reg<C, 3, 2>(x, m, rneed); break;
            }
        }
    } else if (op.k == 0) {  // SOP_DIAG, one factor on the control subspace
        if (op.flags & 1) {
#pragma unroll
            QSIM_EACH(s, x) {
#pragma unroll
                for (int j = 0; j < NR; ++j)
                    if ((j & rneed) == rneed) {
                        x[j].x = -x[j].x;
                        x[j].y = -x[j].y;
                    }
            }
        } else {
            const C f = src.pool(op.moff);
#pragma unroll
            QSIM_EACH(s, x) {
#pragma unroll
                for (int j = 0; j < NR; ++j)
                    if ((j & rneed) == rneed) x[j] = cmul(f, x[j]);
            }
        }
    } else {  // SOP_DIAG with selector qubits
        // selector bits from the thread's base index (lane / warp / tile
        // qubits), then per register index j the bits its register qubits add
        const int k = op.k;
        int sel_t = 0;
        for (int t = 0; t < k; ++t) {
            const int code = op.dq[t];
            if (code >= POS_BASE) sel_t |= int((base >> (code - POS_BASE)) & 1) << (k - 1 - t);
        }
        const uint32_t pk = uint32_t(uint8_t(op.a)) | (uint32_t(uint8_t(op.b)) << 8);
        int rm[REG_BITS];
#pragma unroll
        for (int r = 0; r < REG_BITS; ++r) {
            const int f = int(pk >> (4 * r)) & 15;
            rm[r] = f ? 1 << (f - 1) : 0;
        }
        if (k <= 2) {
            const C f0 = src.pool(op.moff), f1 = src.pool(op.moff + 1);
            const C f2 = k == 2 ? src.pool(op.moff + 2) : f0, f3 = k == 2 ? src.pool(op.moff + 3) : f1;
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                if ((j & rneed) != rneed) continue;
                int sel = sel_t;
#pragma unroll
                for (int r = 0; r < REG_BITS; ++r)
                    if ((j >> r) & 1) sel |= rm[r];
                const C f = (sel & 2) ? ((sel & 1) ? f3 : f2) : ((sel & 1) ? f1 : f0);
#pragma unroll
                QSIM_EACH(s, x) x[j] = cmul(f, x[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                if ((j & rneed) != rneed) continue;
                int sel = sel_t;
#pragma unroll
                for (int r = 0; r < REG_BITS; ++r)
                    if ((j >> r) & 1) sel |= rm[r];
                const C f = src.pool(op.moff + sel);
#pragma unroll
                QSIM_EACH(s, x) x[j] = cmul(f, x[j]);
            }
        }
    }
}
#undef QSIM_EACH

template <typename C, typename Src>
__device__ __forceinline__ void apply_op(const StageOp &op, const Src &src, C (&v)[1 << REG_BITS], uint64_t base,
                                         int lane) {
    apply_op2<C, 1>(op, src, v, v, base, lane);
}

// One pass of the op list over the tile held in v (16 amplitudes per thread).
// Src supplies op(o), phase(i), pool(i) and aux(i); ph / base are the current
// phase and the thread's base index, updated by EXCHANGE ops.
template <typename C, int W, typename Src>
__device__ __forceinline__ void stage_exec(const Src &src, int nops, C (&v)[1 << REG_BITS], int &ph, uint64_t &base,
                                           uint64_t tile_base, C *tile, int lane, int warp) {
    for (int o = 0; o < nops; ++o) {
        const StageOp &op = src.op(o);
        if (op.type == SOP_EXCHANGE) {
            tile_shared<C, W, true>(tile, v, src.phase(ph), lane, warp);
            __syncthreads();
            ph = op.a;
            base = thread_base<W>(src.phase(ph), tile_base, lane, warp);
            tile_shared<C, W, false>(tile, v, src.phase(ph), lane, warp);
            __syncthreads();
            continue;
        }
        apply_op<C>(op, src, v, base, lane);
    }
}

// For a gradient term on qubit position a: with M[r][c] = sum conj(w_r) v_c
// over the pairs (r, c = the qubit's value), Im<w| px X + py Y + pz Z |v> =
// px Sx + py Sy + pz Sz with
//   Sx = Im M01 + Im M10,  Sy = Re M10 - Re M01,  Sz = Im M00 - Im M11.
// This adds the thread's share of (Sx, Sy, Sz) over its 16 amplitudes
// (register bit RB; RB < 0: lane bit a, each lane taking the terms whose w
// it holds).  Every term on one qubit at one point of the sweep shares the
// three sums, whatever its Pauli vector.
template <typename C, int RB>
__device__ __forceinline__ void grad3_t(const C (&v)[1 << REG_BITS], const C (&w)[1 << REG_BITS], int a, int lane,
                                        float &sx, float &sy, float &sz) {
    constexpr int NR = 1 << REG_BITS;
    if constexpr (RB >= 0) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            if (j & (1 << RB)) continue;
            const C p0 = v[j], p1 = v[j | (1 << RB)], l0 = w[j], l1 = w[j | (1 << RB)];
            sz += float(l0.x) * float(p0.y) - float(l0.y) * float(p0.x) - float(l1.x) * float(p1.y) +
                  float(l1.y) * float(p1.x);
            sx += float(l0.x) * float(p1.y) - float(l0.y) * float(p1.x) + float(l1.x) * float(p0.y) -
                  float(l1.y) * float(p0.x);
            sy += float(l1.x) * float(p0.x) + float(l1.y) * float(p0.y) - float(l0.x) * float(p1.x) -
                  float(l0.y) * float(p1.y);
        }
    } else {
        float tx = 0.f, ty = 0.f, tz = 0.f;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const C p = v[j], l = w[j], q = shfl_c(v[j], 1 << a);  // q: the partner's amplitude
            tz += float(l.x) * float(p.y) - float(l.y) * float(p.x);
            tx += float(l.x) * float(q.y) - float(l.y) * float(q.x);
            ty += float(l.x) * float(q.x) + float(l.y) * float(q.y);
        }
        const bool one = (lane >> a) & 1;
        sx += tx;
        sy += one ? ty : -ty;
        sz += one ? -tz : tz;
    }
}

// position a: lane bit a < 8, register bit a - 8
template <typename C>
__device__ __forceinline__ void grad3(const C (&v)[1 << REG_BITS], const C (&w)[1 << REG_BITS], int a, int lane,
                                      float &sx, float &sy, float &sz) {
    switch (a - POS_REG) {
        case 0: grad3_t<C, 0>(v, w, a, lane, sx, sy, sz); break;
        case 1: grad3_t<C, 1>(v, w, a, lane, sx, sy, sz); break;
        case 2: grad3_t<C, 2>(v, w, a, lane, sx, sy, sz); break;
        case 3: grad3_t<C, 3>(v, w, a, lane, sx, sy, sz); break;
        default: grad3_t<C, -1>(v, w, a, lane, sx, sy, sz); break;
    }
}

// The reverse sweep of the adjoint gradient: the same op list applied to two
// tiles (psi in v, lambda in w); a SOP_GRAD op (a = position, k = its local
// index) adds the warp's share of (Sx, Sy, Sz) to gw[(3k + c) * 2^W + warp]
// (shared; each entry belongs to one warp, so no atomics).  The sums stay in
// fp32 up to the warp: fp64 runs at 1/64 of the fp32 rate here.
template <typename C, int W, typename Src>
__device__ __forceinline__ void stage_exec2(const Src &src, int nops, C (&v)[1 << REG_BITS], C (&w)[1 << REG_BITS],
                                            int &ph, uint64_t &base, uint64_t tile_base, C *tile, int lane, int warp,
                                            float *gw) {
    for (int o = 0; o < nops; ++o) {
        const StageOp &op = src.op(o);
        if (op.type == SOP_EXCHANGE) {
            tile_shared<C, W, true>(tile, v, src.phase(ph), lane, warp);
            __syncthreads();
            const int nph = op.a;
            tile_shared<C, W, false>(tile, v, src.phase(nph), lane, warp);
            __syncthreads();
            tile_shared<C, W, true>(tile, w, src.phase(ph), lane, warp);
            __syncthreads();
            tile_shared<C, W, false>(tile, w, src.phase(nph), lane, warp);
            __syncthreads();
            ph = nph;
            base = thread_base<W>(src.phase(ph), tile_base, lane, warp);
            continue;
        }
        if (op.type == SOP_GRAD) {
            float sx = 0.f, sy = 0.f, sz = 0.f;
            grad3<C>(v, w, op.a, lane, sx, sy, sz);
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, s);
                sy += __shfl_xor_sync(0xffffffffu, sy, s);
                sz += __shfl_xor_sync(0xffffffffu, sz, s);
            }
            if (lane == 0) {
                float *g = gw + ((3 * op.k) << W) + warp;
                g[0] += sx;
                g[1 << W] += sy;
                g[2 << W] += sz;
            }
            continue;
        }
        apply_op2<C, 2>(op, src, v, w, base, lane);
    }
}

// ------------------------------------------------------------------ host planner
struct GateClass {
    enum { DIAG, DENSE1, DENSE2, OTHER } kind;
    Op op;            // classified form (targets reduced, controls extended)
    int grad_slot = -1;  // >= 0: an adjoint gradient marker on op.targets[0]
    double grad_v[3] = {0, 0, 0};  // its operator px X + py Y + pz Z
};

struct Stage {
    bool plain = false;
    Op op;                   // plain: one sweep
    std::vector<int> slots;  // tile qubits outside the lanes (slot s <-> slots[s])
    std::vector<StageOp> ops;
    std::vector<Phase> phases;
    std::vector<cd> pool;
    std::vector<uint64_t> aux;
    struct GradRef {
        int slot;     // global gradient slot
        int op;       // local SOP_GRAD index whose (Sx, Sy, Sz) it combines
        double v[3];  // its Pauli vector
    };
    std::vector<GradRef> grads;
    int ngradops = 0;
    int phase0 = 0;
    std::vector<int> gates;  // source gates the stage applies, in schedule order (before merging / batching)
};

// flops per amplitude of a planned stage (host): those of the circuit's gates
// it applies, one sweep each; and those its ops execute after fusion
double stage_flops_per_amp(const qsim_circuit &c, const Stage &st);
double stage_exec_flops_per_amp(const Stage &st);
// Split a circuit into stages for tiles of 2^(9 + W) amplitudes (after pair
// fusion, when the circuit has no gradient markers).  With `limits` the op,
// phase and pool counts of a stage stay within one kernel parameter block.
// With `lookahead` each stage repeatedly takes the gate that adds the fewest
// new tile qubits (fewer stages on random circuits); without it, one pass in
// circuit order (the batch kernel's plans, where it measured faster).
int plan_stage_list(const qsim_circuit &c, int W, bool limits, std::vector<Stage> &out, bool lookahead = true);

// Kernel parameter block of one tile stage.
template <typename C> inline void make_params(const Stage &st, StageParams<C> &prm) {
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
    for (size_t i = 0; i < st.aux.size(); ++i) prm.aux[i] = st.aux[i];
}

}  // namespace stage

struct SpecLib;  // specialize.cu
// A staged plan: its stages, the interpreter's parameter blocks per dtype
// and, for specialised plans (QSIM_PLAN_SPECIALIZE), the compiled stage
// kernels with their coefficient blocks.
struct StagedPlan {
    int W = 4;
    bool specialized = false;
    std::vector<stage::Stage> stages;
    struct Dev {
        bool ready = false;
        std::vector<void *> plain_mats;
        std::vector<unsigned char> params;  // packed StageParams per tile stage
        std::vector<size_t> param_off;
    } dev[2];
    struct Spec {
        bool ready = false;
        std::vector<std::shared_ptr<SpecLib>> libs;     // compiled groups of stages
        std::vector<cudaKernel_t> kern;                  // per stage (plain stages: null)
        std::vector<std::vector<unsigned char>> params;  // per stage coefficient block
    } spec[2];
    std::vector<double> flops_per_amp;   // flops per amplitude each stage executes
    double circuit_flops_per_amp = 0.0;  // the circuit's gates, one sweep each, summed
    ~StagedPlan() {
        for (Dev &d : dev)
            for (void *m : d.plain_mats)
                if (m) cudaFree(m);
    }
};
// specialize.cu: compile (or find cached) the kernels of every tile stage
// for one dtype; launch tile stage i on psi
int spec_prepare(StagedPlan &sp, int dtype);
int spec_launch(StagedPlan &sp, int dtype, size_t i, void *psi, int n, cudaStream_t s);
std::string spec_source(const StagedPlan &sp, int dtype, size_t i0, size_t i1);
// specialize.cu: the two-state stages of the adjoint reverse sweep
struct DualSpec {
    std::vector<std::shared_ptr<SpecLib>> libs;
    std::vector<cudaKernel_t> kern;  // per stage (plain stages: null)
};
int spec_dual_prepare(const std::vector<stage::Stage> &stages, int n, int W, DualSpec &out);
int spec_dual_launch(const DualSpec &d, const stage::Stage &st, size_t i, float2 *psi, float2 *lam, double *partial,
                     int n, int W, cudaStream_t s);
}  // namespace qsim

// Stage kernels specialised per plan (QSIM_PLAN_SPECIALIZE).
//
// The register-tile interpreter (staged.cu, stage_common.cuh) decodes each
// stage's op list at run time: every thread loads an op's type, positions,
// masks and coefficients from the parameter block and branches on them, and
// on the fused random-circuit plan about half of its instructions are that
// decoding.  Here the host writes each tile stage of a plan out as its own
// CUDA kernel instead -- the same tile, phases, exchanges and arithmetic, but
// every position, control mask, register index and coefficient offset a
// constant of the source -- and compiles the plan's kernels with NVRTC for
// sm_103a.  The coefficients stay out of the source: each kernel takes them
// as a by-value parameter block (scalar FP64 / lane ops read them from the
// constant bank; the complex64 register ops read host-made coefficient pairs
// for the paired FP32 instructions), so two circuits of the same structure
// with other angles share one compiled module.  Modules are cached by a
// structural fingerprint of their stages.  The adjoint method's reverse
// sweep gets two-state kernels from the same generator (dual).
//
// The arithmetic per op is the interpreter's (same products, same order), so
// both executors give the same amplitudes up to the compiler's contraction
// choices.
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "plan.h"
#include "stage_common.cuh"

namespace qsim {
using namespace stage;

// A compiled group of stage kernels (one NVRTC program, one CUDA library).
struct SpecLib {
    cudaLibrary_t lib = nullptr;
    ~SpecLib() {
        if (lib) cudaLibraryUnload(lib);
    }
};

namespace {

const char *kPrelude = R"(
typedef unsigned long long u64;
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
__device__ __forceinline__ float2 shfl_c(float2 a, int m) {
    a.x = __shfl_xor_sync(0xffffffffu, a.x, m);
    a.y = __shfl_xor_sync(0xffffffffu, a.y, m);
    return a;
}
__device__ __forceinline__ double2 shfl_c(double2 a, int m) {
    a.x = __shfl_xor_sync(0xffffffffu, a.x, m);
    a.y = __shfl_xor_sync(0xffffffffu, a.y, m);
    return a;
}
// 2x2 on a register pair
template <typename C> __device__ __forceinline__ void u1(C &a, C &b, C m00, C m01, C m10, C m11) {
    const C x = a, y = b;
    a = cmad(m01, y, cmul(m00, x));
    b = cmad(m11, y, cmul(m10, x));
}
// 4x4 on four registers (index bit 1 = first target)
template <typename C> __device__ __forceinline__ void u2(C &a0, C &a1, C &a2, C &a3, const C *m) {
    const C x0 = a0, x1 = a1, x2 = a2, x3 = a3;
    a0 = cmad(m[3], x3, cmad(m[2], x2, cmad(m[1], x1, cmul(m[0], x0))));
    a1 = cmad(m[7], x3, cmad(m[6], x2, cmad(m[5], x1, cmul(m[4], x0))));
    a2 = cmad(m[11], x3, cmad(m[10], x2, cmad(m[9], x1, cmul(m[8], x0))));
    a3 = cmad(m[15], x3, cmad(m[14], x2, cmad(m[13], x1, cmul(m[12], x0))));
}
template <typename C> __device__ __forceinline__ C neg(C a) {
    a.x = -a.x;
    a.y = -a.y;
    return a;
}
// paired FP32 arithmetic (fma.rn.f32x2): two lanes of a 64-bit register
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up2(u64 r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// complex products with each coefficient m given as the pairs (m.x, m.x) and
// (-m.y, m.y) (cc[2e], cc[2e + 1]): m x = (m.x, m.x) (x.x, x.y) + (-m.y, m.y) (x.y, x.x),
// in the order of cmul / cmad above
__device__ __forceinline__ void u1p(float2 &a, float2 &b, const u64 *cc) {
    const u64 X = pk2(a.x, a.y), Xs = pk2(a.y, a.x), Y = pk2(b.x, b.y), Ys = pk2(b.y, b.x);
    a = up2(fma2(cc[3], Ys, fma2(cc[2], Y, fma2(cc[1], Xs, mul2(cc[0], X)))));
    b = up2(fma2(cc[7], Ys, fma2(cc[6], Y, fma2(cc[5], Xs, mul2(cc[4], X)))));
}
__device__ __forceinline__ void u2p(float2 &a0, float2 &a1, float2 &a2, float2 &a3, const u64 *cc) {
    const u64 X0 = pk2(a0.x, a0.y), S0 = pk2(a0.y, a0.x), X1 = pk2(a1.x, a1.y), S1 = pk2(a1.y, a1.x);
    const u64 X2 = pk2(a2.x, a2.y), S2 = pk2(a2.y, a2.x), X3 = pk2(a3.x, a3.y), S3 = pk2(a3.y, a3.x);
#define QSIM_U2P_ROW(R, OUT)                                   \
    {                                                          \
        const u64 *m = cc + 8 * R;                             \
        u64 t = fma2(m[1], S0, mul2(m[0], X0));                \
        t = fma2(m[3], S1, fma2(m[2], X1, t));                 \
        t = fma2(m[5], S2, fma2(m[4], X2, t));                 \
        OUT = up2(fma2(m[7], S3, fma2(m[6], X3, t)));          \
    }
    QSIM_U2P_ROW(0, a0)
    QSIM_U2P_ROW(1, a1)
    QSIM_U2P_ROW(2, a2)
    QSIM_U2P_ROW(3, a3)
#undef QSIM_U2P_ROW
}
// a with its sign flipped where sb (0 or 0x80000000) says so
__device__ __forceinline__ float2 xsign(float2 a, unsigned sb) {
    a.x = __uint_as_float(__float_as_uint(a.x) ^ sb);
    a.y = __uint_as_float(__float_as_uint(a.y) ^ sb);
    return a;
}
__device__ __forceinline__ double2 xsign(double2 a, unsigned sb) {
    a.x = __hiloint2double(__double2hiint(a.x) ^ int(sb), __double2loint(a.x));
    a.y = __hiloint2double(__double2hiint(a.y) ^ int(sb), __double2loint(a.y));
    return a;
}
)";

// Writes the source of tile-stage kernels.  Every op is emitted for the
// tile in `v` and, for the two-state stages of the adjoint reverse sweep
// (dual), once more for the tile in `w`, as the interpreter's apply_op2
// applies one decoded op to both.
struct Gen {
    std::ostringstream o;
    const char *C;  // "float2" / "double2"
    int W;
    bool paired = false;  // register ops in paired FP32 (complex64 single-state stages)

    // global index bits of register index j in phase P
    static uint64_t reg_offset(const Phase &P, int j) {
        uint64_t off = 0;
        for (int b = 0; b < REG_BITS; ++b)
            if ((j >> b) & 1) off |= uint64_t(1) << P.rq[b];
        return off;
    }
    static uint32_t smem_offset(const Phase &P, int j) {
        uint32_t off = 0;
        for (int b = 0; b < REG_BITS; ++b)
            if ((j >> b) & 1) off |= uint32_t(1) << (LANE_BITS + P.rslot[b]);
        return off;
    }
    void set_base(const Phase &P) {
        o << "    base = tbase | (u64)lane";
        for (int i = 0; i < W; ++i) o << " | ((u64)((warp >> " << i << ") & 1) << " << int(P.wq[i]) << ")";
        o << ";\n";
    }
    std::string tcond(uint64_t tm) const {
        std::ostringstream c;
        c << "(base & 0x" << std::hex << tm << "ull) == 0x" << tm << "ull";
        return c.str();
    }
    void ctrl_open(const StageOp &op) {
        if (op.tmask) o << "    if (" << tcond(op.tmask) << ") {\n";
        else o << "    {\n";
    }
    static bool rok(int j, int rneed) { return (j & rneed) == rneed; }
    std::string coef(int i) const { return "p.c[" + std::to_string(i) + "]"; }

    void u1_reg(const char *A, int rb, int moff, int rneed) {
        for (int i = 0; i < (1 << REG_BITS); ++i) {
            if ((i >> rb) & 1 || !rok(i, rneed)) continue;
            if (paired)
                o << "        u1p(" << A << "[" << i << "], " << A << "[" << (i | (1 << rb)) << "], &p.cc["
                  << 2 * moff << "]);\n";
            else
            o << "        u1(" << A << "[" << i << "], " << A << "[" << (i | (1 << rb)) << "], " << coef(moff) << ", "
              << coef(moff + 1) << ", " << coef(moff + 2) << ", " << coef(moff + 3) << ");\n";
        }
    }
    // 1-qubit gate on lane bit l; `ok` guards the update (every lane shuffles)
    void u1_lane(const char *A, int l, int moff, int rneed, bool guarded) {
        o << "    {\n        const bool hi = (lane >> " << l << ") & 1;\n";
        o << "        const " << C << " cs = hi ? " << coef(moff + 3) << " : " << coef(moff) << ";\n";
        o << "        const " << C << " co = hi ? " << coef(moff + 2) << " : " << coef(moff + 1) << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j) {
            if (!rok(j, rneed)) continue;
            o << "        { const " << C << " t = shfl_c(" << A << "[" << j << "], " << (1 << l) << "); ";
            if (guarded) o << "if (ok) ";
            o << A << "[" << j << "] = cmad(co, t, cmul(cs, " << A << "[" << j << "])); }\n";
        }
        o << "    }\n";
    }
    void op_u2(const char *A, const StageOp &op) {
        const bool la = op.a < POS_REG, lb = op.b < POS_REG;
        const int m = op.moff;
        if (!la && !lb) {  // two register targets: the interpreter's u2_reg
            const int JA = op.a - POS_REG, JB = op.b - POS_REG;
            ctrl_open(op);
            if (paired) o << "        const u64 *m = &p.cc[" << 2 * m << "];\n";
            else o << "        const " << C << " *m = &" << coef(m) << ";\n";
            for (int i = 0; i < (1 << REG_BITS); ++i) {
                if (i & ((1 << JA) | (1 << JB)) || !rok(i, op.rneed)) continue;
                o << "        " << (paired ? "u2p(" : "u2(") << A << "[" << i << "], " << A << "[" << (i | (1 << JB))
                  << "], " << A << "[" << (i | (1 << JA)) << "], " << A << "[" << (i | (1 << JA) | (1 << JB))
                  << "], m);\n";
            }
            o << "    }\n";
            return;
        }
        o << "    {\n        const bool ok = " << (op.tmask ? tcond(op.tmask) : std::string("true")) << ";\n";
        if (la != lb) {
            // one lane bit and one register bit (coefficients per lane-bit value)
            const int l = la ? op.a : op.b, rb = (la ? op.b : op.a) - POS_REG;
            o << "        const bool hi = (lane >> " << l << ") & 1;\n";
            for (int e = 0; e < 8; ++e)
                o << "        const " << C << " m" << e << " = hi ? " << coef(m + 8 + e) << " : " << coef(m + e)
                  << ";\n";
            for (int i = 0; i < (1 << REG_BITS); ++i) {
                if ((i >> rb) & 1 || !rok(i, op.rneed)) continue;
                const int i1 = i | (1 << rb);
                o << "        { const " << C << " x0 = " << A << "[" << i << "], x1 = " << A << "[" << i1 << "];\n";
                o << "          const " << C << " y0 = shfl_c(x0, " << (1 << l) << "), y1 = shfl_c(x1, " << (1 << l)
                  << ");\n";
                o << "          if (ok) { " << A << "[" << i
                  << "] = cmad(m3, y1, cmad(m2, y0, cmad(m1, x1, cmul(m0, x0))));\n";
                o << "                    " << A << "[" << i1
                  << "] = cmad(m7, y1, cmad(m6, y0, cmad(m5, x1, cmul(m4, x0)))); } }\n";
            }
        } else {
            // two lane bits: own amplitude and the lanes across a, b and both
            const int ma = 1 << op.a, mb = 1 << op.b;
            o << "        const int sel = (((lane >> " << int(op.a) << ") & 1) << 1) | ((lane >> " << int(op.b)
              << ") & 1);\n";
            for (int e = 0; e < 4; ++e)
                o << "        const " << C << " m" << e << " = sel == 0 ? " << coef(m + e) << " : sel == 1 ? "
                  << coef(m + 4 + e) << " : sel == 2 ? " << coef(m + 8 + e) << " : " << coef(m + 12 + e) << ";\n";
            for (int j = 0; j < (1 << REG_BITS); ++j) {
                if (!rok(j, op.rneed)) continue;
                o << "        { const " << C << " p1 = shfl_c(" << A << "[" << j << "], " << ma << "), p2 = shfl_c("
                  << A << "[" << j << "], " << mb << "), p3 = shfl_c(" << A << "[" << j << "], " << (ma | mb)
                  << ");\n";
                o << "          if (ok) " << A << "[" << j << "] = cmad(m3, p3, cmad(m2, p2, cmad(m1, p1, cmul(m0, "
                  << A << "[" << j << "])))); }\n";
            }
        }
        o << "    }\n";
    }

    void op_diag(const char *A, const StageOp &op) {
        if (op.k == 0 && (op.flags & 1)) {  // a sign flip: branch free, the control as a sign mask
            o << "    {\n        const unsigned sb = " << (op.tmask ? "(" + tcond(op.tmask) + ") ? 0x80000000u : 0u"
                                                           : std::string("0x80000000u")) << ";\n";
            for (int j = 0; j < (1 << REG_BITS); ++j)
                if (rok(j, op.rneed)) o << "        " << A << "[" << j << "] = xsign(" << A << "[" << j << "], sb);\n";
            o << "    }\n";
            return;
        }
        ctrl_open(op);
        if (op.k == 0) {
            for (int j = 0; j < (1 << REG_BITS); ++j)
                if (rok(j, op.rneed))
                    o << "        " << A << "[" << j << "] = cmul(" << coef(op.moff) << ", " << A << "[" << j << "]);\n";
            o << "    }\n";
            return;
        }
        // selector: bits from the thread's base index, then per register index
        const int k = op.k;
        o << "        const int st = 0";
        int rsel[REG_BITS] = {0, 0, 0, 0};  // selector bit each register bit feeds
        for (int t = 0; t < k; ++t) {
            const int code = op.dq[t];
            if (code >= POS_BASE) o << " | (int((base >> " << (code - POS_BASE) << ") & 1) << " << (k - 1 - t) << ")";
            else rsel[code - POS_REG] = 1 << (k - 1 - t);
        }
        o << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j) {
            if (!rok(j, op.rneed)) continue;
            int sj = 0;
            for (int r = 0; r < REG_BITS; ++r)
                if ((j >> r) & 1) sj |= rsel[r];
            o << "        " << A << "[" << j << "] = cmul(p.c[" << op.moff << " + (st | " << sj << ")], " << A << "["
              << j << "]);\n";
        }
        o << "    }\n";
    }

    void op_neg(const Stage &st, const StageOp &op, bool dual) {
        o << "    {\n        unsigned flip = 0u;\n";
        for (int e = 0; e < op.k; ++e) {
            const uint64_t tm = st.aux[size_t(op.moff + 2 * e)];
            const uint32_t pat = uint32_t(st.aux[size_t(op.moff + 2 * e + 1)]);
            if (tm == 0) o << "        flip ^= " << pat << "u;\n";
            else o << "        if (" << tcond(tm) << ") flip ^= " << pat << "u;\n";
        }
        // branch free: flip's bit j moved to the sign bit and XORed in (the
        // lanes of a warp flip different registers)
        for (int j = 0; j < (1 << REG_BITS); ++j) {
            o << "        { const unsigned sb = (flip << " << (31 - j) << ") & 0x80000000u; v[" << j << "] = xsign(v["
              << j << "], sb);";
            if (dual) o << " w[" << j << "] = xsign(w[" << j << "], sb);";
            o << " }\n";
        }
        o << "    }\n";
    }

    void exchange_one(const char *A, const Phase &from, const Phase &to) {
        o << "    {\n        unsigned lb = (unsigned)lane";
        for (int i = 0; i < W; ++i) o << " | (((unsigned)warp >> " << i << " & 1u) << " << (LANE_BITS + from.wslot[i]) << ")";
        o << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j)
            o << "        tile[lb | " << smem_offset(from, j) << "u] = " << A << "[" << j << "];\n";
        o << "        __syncthreads();\n        lb = (unsigned)lane";
        for (int i = 0; i < W; ++i) o << " | (((unsigned)warp >> " << i << " & 1u) << " << (LANE_BITS + to.wslot[i]) << ")";
        o << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j)
            o << "        " << A << "[" << j << "] = tile[lb | " << smem_offset(to, j) << "u];\n";
        o << "        __syncthreads();\n    }\n";
    }
    // adjoint gradient op: the warp's share of (Sx, Sy, Sz) over the pairs
    // of position a (as grad3_t in stage_common.cuh), added to gw
    void op_grad(const StageOp &op) {
        o << "    {\n        float sx = 0.f, sy = 0.f, sz = 0.f;\n";
        if (op.a >= POS_REG) {
            const int rb = op.a - POS_REG;
            for (int j = 0; j < (1 << REG_BITS); ++j) {
                if ((j >> rb) & 1) continue;
                const int j1 = j | (1 << rb);
                o << "        { const " << C << " p0 = v[" << j << "], p1 = v[" << j1 << "], l0 = w[" << j
                  << "], l1 = w[" << j1 << "];\n";
                o << "          sz += float(l0.x) * float(p0.y) - float(l0.y) * float(p0.x) - float(l1.x) * float(p1.y) + "
                     "float(l1.y) * float(p1.x);\n";
                o << "          sx += float(l0.x) * float(p1.y) - float(l0.y) * float(p1.x) + float(l1.x) * float(p0.y) - "
                     "float(l1.y) * float(p0.x);\n";
                o << "          sy += float(l1.x) * float(p0.x) + float(l1.y) * float(p0.y) - float(l0.x) * float(p1.x) - "
                     "float(l0.y) * float(p1.y); }\n";
            }
        } else {
            o << "        float tx = 0.f, ty = 0.f, tz = 0.f;\n";
            for (int j = 0; j < (1 << REG_BITS); ++j) {
                o << "        { const " << C << " pp = v[" << j << "], l = w[" << j << "], qq = shfl_c(v[" << j << "], "
                  << (1 << op.a) << ");\n";
                o << "          tz += float(l.x) * float(pp.y) - float(l.y) * float(pp.x);\n";
                o << "          tx += float(l.x) * float(qq.y) - float(l.y) * float(qq.x);\n";
                o << "          ty += float(l.x) * float(qq.x) + float(l.y) * float(qq.y); }\n";
            }
            o << "        const bool one = (lane >> " << int(op.a) << ") & 1;\n";
            o << "        sx += tx;\n        sy += one ? ty : -ty;\n        sz += one ? -tz : tz;\n";
        }
        o << "        for (int s = 16; s > 0; s >>= 1) {\n"
             "            sx += __shfl_xor_sync(0xffffffffu, sx, s);\n"
             "            sy += __shfl_xor_sync(0xffffffffu, sy, s);\n"
             "            sz += __shfl_xor_sync(0xffffffffu, sz, s);\n"
             "        }\n";
        o << "        if (lane == 0) {\n            float *g = gw + " << ((3 * int(op.k)) << W) << " + warp;\n"
          << "            g[0] += sx;\n            g[" << (1 << W) << "] += sy;\n            g[" << (2 << W)
          << "] += sz;\n        }\n    }\n";
    }

    void op_any(const Stage &st, const StageOp &op, bool dual) {
        const char *arrs[2] = {"v", "w"};
        const int na = dual ? 2 : 1;
        switch (op.type) {
            case SOP_U1:
                for (int t = 0; t < na; ++t) {
                    if (op.a >= POS_REG) {
                        ctrl_open(op);
                        u1_reg(arrs[t], op.a - POS_REG, op.moff, op.rneed);
                        o << "    }\n";
                    } else {
                        o << "    {\n        const bool ok = " << (op.tmask ? tcond(op.tmask) : std::string("true"))
                          << ";\n";
                        u1_lane(arrs[t], op.a, op.moff, op.rneed, op.tmask != 0);
                        o << "    }\n";
                    }
                }
                break;
            case SOP_U1R:
                for (int t = 0; t < na; ++t) {
                    int off = op.moff;
                    o << "    {\n";
                    for (int b = 0; b < REG_BITS; ++b)
                        if (op.a & (1 << b)) {
                            u1_reg(arrs[t], b, off, 0);
                            off += 4;
                        }
                    o << "    }\n";
                }
                break;
            case SOP_U1L:
                for (int t = 0; t < na; ++t) {
                    int off = op.moff;
                    for (int l = 0; l < LANE_BITS; ++l)
                        if (op.a & (1 << l)) {
                            u1_lane(arrs[t], l, off, 0, false);
                            off += 4;
                        }
                }
                break;
            case SOP_U2:
                for (int t = 0; t < na; ++t) op_u2(arrs[t], op);
                break;
            case SOP_DIAG:
                for (int t = 0; t < na; ++t) op_diag(arrs[t], op);
                break;
            case SOP_NEG: op_neg(st, op, dual); break;
            case SOP_GRAD:
                if (dual) op_grad(op);
                break;
            default: break;
        }
    }
    // the kernel of one tile stage; its parameter block holds ncoef
    // coefficients (at least one) and, for a dual stage, the Pauli vectors of
    // its gradient terms.  A dual stage (n qubits, ntiles tiles) writes each
    // gradient term's per-tile sum to partial[slot * ntiles + tile].
    void stage(const Stage &st, const std::string &name, int ncoef, int min_blocks, bool dual, uint64_t ntiles) {
        const int ng = std::max<int>(1, int(st.grads.size()));
        o << "struct P_" << name << " { " << C << " c[" << ncoef << "];";
        if (paired) o << " u64 cc[" << 2 * ncoef << "];";
        if (dual) o << " float gv[" << ng << "][3];";
        o << " };\n";
        if (dual) {
            o << "__constant__ int " << name << "_gslot[" << ng << "] = {";
            for (size_t g = 0; g < st.grads.size(); ++g) o << (g ? ", " : "") << st.grads[g].slot;
            if (st.grads.empty()) o << "0";
            o << "};\n__constant__ int " << name << "_gop[" << ng << "] = {";
            for (size_t g = 0; g < st.grads.size(); ++g) o << (g ? ", " : "") << st.grads[g].op;
            if (st.grads.empty()) o << "0";
            o << "};\n";
        }
        o << "extern \"C\" __global__ void __launch_bounds__(" << (32 << W) << ", " << min_blocks << ") " << name
          << "(" << C << " *__restrict__ psi, ";
        if (dual) o << C << " *__restrict__ lam, double *__restrict__ partial, ";
        o << "const __grid_constant__ P_" << name << " p) {\n";
        o << "    extern __shared__ " << C << " tile[];\n";
        o << "    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;\n";
        const int gwn = (3 * std::max(1, st.ngradops)) << W;
        if (dual) {
            o << "    __shared__ float gw[" << gwn << "];\n";
            o << "    for (int g = threadIdx.x; g < " << gwn << "; g += blockDim.x) gw[g] = 0.f;\n";
            o << "    __syncthreads();\n";
        }
        // tile id -> base index: a zero inserted at every tile qubit (ascending)
        std::vector<int> tq;
        for (int q = 0; q < LANE_BITS; ++q) tq.push_back(q);
        for (int q : st.slots) tq.push_back(q);
        std::sort(tq.begin(), tq.end());
        o << "    u64 tbase = (u64)blockIdx.x;\n";
        for (int q : tq)
            o << "    tbase = ((tbase >> " << q << ") << " << (q + 1) << ") | (tbase & 0x" << std::hex
              << ((uint64_t(1) << q) - 1) << std::dec << "ull);\n";
        o << "    u64 base;\n";
        int ph = st.phase0;
        set_base(st.phases[size_t(ph)]);
        o << "    " << C << " v[" << (1 << REG_BITS) << "];\n";
        if (dual) o << "    " << C << " w[" << (1 << REG_BITS) << "];\n";
        auto io = [&](const char *ptr, const char *A, bool store) {
            o << "    {\n        " << (store ? "" : "const ") << C << " *g = " << ptr << " + base;\n";
            for (int j = 0; j < (1 << REG_BITS); ++j) {
                const uint64_t off = reg_offset(st.phases[size_t(ph)], j);
                if (store) o << "        g[0x" << std::hex << off << std::dec << "ull] = " << A << "[" << j << "];\n";
                else o << "        " << A << "[" << j << "] = g[0x" << std::hex << off << std::dec << "ull];\n";
            }
            o << "    }\n";
        };
        io("psi", "v", false);
        if (dual) io("lam", "w", false);
        for (const StageOp &op : st.ops) {
            if (op.type == SOP_EXCHANGE) {
                exchange_one("v", st.phases[size_t(ph)], st.phases[size_t(op.a)]);
                if (dual) exchange_one("w", st.phases[size_t(ph)], st.phases[size_t(op.a)]);
                ph = op.a;
                set_base(st.phases[size_t(ph)]);
                continue;
            }
            op_any(st, op, dual);
        }
        io("psi", "v", true);
        if (dual) {
            io("lam", "w", true);
            o << "    __syncthreads();\n";
            o << "    for (int g = threadIdx.x; g < " << int(st.grads.size()) << "; g += blockDim.x) {\n";
            o << "        const float *s = gw + ((3 * " << name << "_gop[g]) << " << W << ");\n";
            o << "        double t = 0.0;\n";
            o << "        for (int i = 0; i < " << (1 << W) << "; ++i)\n";
            o << "            t += double(p.gv[g][0]) * s[i] + double(p.gv[g][1]) * s[" << (1 << W)
              << " + i] + double(p.gv[g][2]) * s[" << (2 << W) << " + i];\n";
            o << "        partial[(u64)" << name << "_gslot[g] * " << ntiles << "ull + blockIdx.x] = t;\n    }\n";
        }
        o << "}\n";
    }
};

std::mutex g_cache_mu;
std::map<std::string, std::shared_ptr<SpecLib>> g_cache;  // structural key -> library
constexpr size_t CACHE_MAX = 64;
double g_compile_s = 0.0;  // seconds spent in NVRTC since load
uint64_t g_compiles = 0, g_hits = 0;

int compile(const std::string &src, std::string &cubin, std::string &log) {
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "qsim_stage.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        log = "nvrtcCreateProgram failed";
        return QSIM_ECUDA;
    }
    const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-default-device"};
    const nvrtcResult rc = nvrtcCompileProgram(prog, 3, opts);
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    log.assign(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    if (rc == NVRTC_SUCCESS) {
        nvrtcGetCUBINSize(prog, &n);
        cubin.assign(n, '\0');
        nvrtcGetCUBIN(prog, &cubin[0]);
    }
    nvrtcDestroyProgram(&prog);
    return rc == NVRTC_SUCCESS ? QSIM_OK : QSIM_ECUDA;
}

std::string kernel_name(size_t i) { return "qsim_spec_stage_" + std::to_string(i); }
std::string dual_kernel_name(size_t i) { return "qsim_spec_dual_" + std::to_string(i); }

// Structural fingerprint of a stage: everything its generated source depends
// on, and nothing of the coefficient values (cache key; far cheaper to form
// than the source).
template <typename T> void put(std::string &k, const T &v) { k.append(reinterpret_cast<const char *>(&v), sizeof v); }
void put_stage(std::string &k, const Stage &st) {
    put(k, int(st.plain));
    if (st.plain) return;
    put(k, int(st.slots.size()));
    for (int q : st.slots) put(k, q);
    put(k, st.phase0);
    put(k, int(st.phases.size()));
    for (const Phase &P : st.phases) put(k, P);  // int8 arrays only
    put(k, int(st.ops.size()));
    for (const StageOp &op : st.ops) {
        put(k, op.tmask);
        put(k, op.moff);
        const int8_t f[6] = {op.type, op.a, op.b, op.k, op.rneed, op.flags};
        put(k, f);
        put(k, op.dq);
    }
    put(k, int(st.aux.size()));
    for (uint64_t a : st.aux) put(k, a);
    put(k, int(st.pool.size()));
    put(k, st.ngradops);
    put(k, int(st.grads.size()));
    for (const Stage::GradRef &g : st.grads) {
        put(k, g.slot);
        put(k, g.op);
    }
}

// The libraries for groups of stages [first, second): looked up by key,
// the missing ones generated and compiled in parallel host threads.
int get_libs(const std::vector<std::pair<size_t, size_t>> &groups, const std::vector<std::string> &keys,
             const std::function<std::string(size_t)> &source_of, std::vector<std::shared_ptr<SpecLib>> &libs) {
    libs.assign(groups.size(), nullptr);
    std::vector<size_t> todo;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            auto it = g_cache.find(keys[gi]);
            if (it != g_cache.end()) {
                libs[gi] = it->second;
                ++g_hits;
            } else {
                todo.push_back(gi);
            }
        }
    }
    if (todo.empty()) return QSIM_OK;
    std::vector<std::string> cubins(groups.size()), logs(groups.size());
    std::vector<int> rcs(groups.size(), QSIM_OK);
    const auto t0 = std::chrono::steady_clock::now();
    {
        std::vector<std::thread> th;
        const size_t nthreads =
            std::max<size_t>(1, std::min<size_t>(todo.size(), std::max(1u, std::thread::hardware_concurrency())));
        std::atomic<size_t> next{0};
        for (size_t t = 0; t < nthreads; ++t)
            th.emplace_back([&] {
                for (size_t k; (k = next.fetch_add(1)) < todo.size();) {
                    const size_t gi = todo[k];
                    rcs[gi] = compile(source_of(gi), cubins[gi], logs[gi]);
                }
            });
        for (std::thread &t : th) t.join();
    }
    for (size_t gi : todo)
        if (rcs[gi] != QSIM_OK)
            return set_error(QSIM_ECUDA, "specialised stage compile failed: %.400s", logs[gi].c_str());
    for (size_t gi : todo) {
        auto L = std::make_shared<SpecLib>();
        QSIM_CUDA_TRY(cudaLibraryLoadData(&L->lib, cubins[gi].data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
                      "load specialised stages");
        libs[gi] = L;
        std::lock_guard<std::mutex> lk(g_cache_mu);
        if (g_cache.size() >= CACHE_MAX) g_cache.erase(g_cache.begin());
        g_cache[keys[gi]] = L;
        ++g_compiles;
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_compile_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return QSIM_OK;
}

std::vector<std::pair<size_t, size_t>> stage_groups(size_t ns) {
    // stages per program: programs compile in parallel host threads and are
    // cached separately; two keeps a 26-stage plan's 13 programs within the
    // host's cores
    const size_t per = 2;
    std::vector<std::pair<size_t, size_t>> groups;
    for (size_t i = 0; i < ns; i += per) groups.push_back({i, std::min(ns, i + per)});
    return groups;
}

void pack_coefficients(const Stage &st, int dtype, std::vector<unsigned char> &b, size_t extra) {
    const size_t eb = dtype == QSIM_C64 ? 8 : 16;
    const size_t nc = std::max<size_t>(1, st.pool.size());
    b.assign(nc * eb + extra, 0);
    for (size_t e = 0; e < st.pool.size(); ++e) {
        if (dtype == QSIM_C64) {
            const float v[2] = {float(st.pool[e].real()), float(st.pool[e].imag())};
            memcpy(&b[e * eb], v, 8);
        } else {
            const double v[2] = {st.pool[e].real(), st.pool[e].imag()};
            memcpy(&b[e * eb], v, 16);
        }
    }
}

// Resident CTAs per SM the kernels are compiled for.  With scalar FMAs four
// CTAs of 256 (64 registers; the coefficients are constant-bank operands)
// measured best (random 30-qubit circuit, one-pass plan: 3.56 ms per stage,
// 3.81 ms at three CTAs, 3.86 ms at five).  The complex64 single-state
// stages run their register ops in paired FP32 (fma.rn.f32x2 on (re, im)
// pairs, the coefficients as host-made pairs in the parameter block), which
// wants more registers: 768 resident threads per SM for tiles of up to 2^12
// (lookahead plan: three CTAs of 256, 3.79 ms per stage, against 3.94 ms at
// four CTAs with spills and 3.98 ms for the scalar FMAs at four), 1024 for
// tiles of 2^13.
int min_blocks_single(int dtype, int W) {
    if (dtype != QSIM_C64) return 1;
    return W >= 4 ? 2 : 24 >> W;
}

}  // namespace

// Source of the tile stages [i0, i1) of a staged plan for one dtype.
std::string spec_source(const StagedPlan &sp, int dtype, size_t i0, size_t i1) {
    Gen g;
    g.C = dtype == QSIM_C64 ? "float2" : "double2";
    g.W = sp.W;
    g.paired = dtype == QSIM_C64;
    g.o << kPrelude;
    for (size_t i = i0; i < i1; ++i) {
        const Stage &st = sp.stages[i];
        if (st.plain) continue;
        g.stage(st, kernel_name(i), std::max<int>(1, int(st.pool.size())), min_blocks_single(dtype, sp.W), false, 0);
    }
    return g.o.str();
}

// Compiles (or finds in the cache) the kernels of every tile stage and
// packs each stage's coefficient block.
int spec_prepare(StagedPlan &sp, int dtype) {
    StagedPlan::Spec &S = sp.spec[dtype];
    if (S.ready) return QSIM_OK;
    const size_t ns = sp.stages.size();
    const auto groups = stage_groups(ns);
    std::vector<std::string> keys(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        std::string &k = keys[gi];
        k = "single";
        put(k, dtype);
        put(k, sp.W);
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            put(k, i);
            put_stage(k, sp.stages[i]);
        }
    }
    std::vector<std::shared_ptr<SpecLib>> libs;
    QSIM_TRY(get_libs(groups, keys,
                      [&](size_t gi) { return spec_source(sp, dtype, groups[gi].first, groups[gi].second); }, libs));
    S.libs.assign(libs.begin(), libs.end());
    S.kern.assign(ns, nullptr);
    S.params.assign(ns, {});
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            const Stage &st = sp.stages[i];
            if (st.plain) continue;
            cudaKernel_t k = nullptr;
            QSIM_CUDA_TRY(cudaLibraryGetKernel(&k, libs[gi]->lib, kernel_name(i).c_str()), "specialised stage kernel");
            S.kern[i] = k;
            pack_coefficients(st, dtype, S.params[i], 0);
            if (dtype == QSIM_C64) {  // the coefficient pairs of the paired register ops
                std::vector<unsigned char> &b = S.params[i];
                const size_t nc = std::max<size_t>(1, st.pool.size());
                b.resize(nc * 8 + nc * 16, 0);
                for (size_t e = 0; e < st.pool.size(); ++e) {
                    const float mx = float(st.pool[e].real()), my = float(st.pool[e].imag());
                    const float pr[4] = {mx, mx, -my, my};
                    memcpy(&b[nc * 8 + e * 16], pr, 16);
                }
            }
        }
    S.ready = true;
    return QSIM_OK;
}

int spec_launch(StagedPlan &sp, int dtype, size_t i, void *psi, int n, cudaStream_t s) {
    const StagedPlan::Spec &S = sp.spec[dtype];
    const size_t eb = dtype == QSIM_C64 ? 8 : 16;
    const int nt = LANE_BITS + REG_BITS + sp.W;
    const uint64_t ntiles = uint64_t(1) << (n - nt);
    const size_t smem = (size_t(1) << nt) * eb;
    const void *f = reinterpret_cast<const void *>(S.kern[i]);
    if (smem > 48 * 1024)
        QSIM_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                      "specialised stage smem attribute");
    void *args[2] = {&psi, const_cast<unsigned char *>(S.params[i].data())};
    LaunchScope ls(K_STAGE, s, 2.0 * double(uint64_t(1) << n) * double(eb), sp.flops_per_amp[i] * double(uint64_t(1) << n));
    QSIM_CUDA_TRY(cudaLaunchKernel(f, dim3(unsigned(ntiles)), dim3(32u << sp.W), args, smem, s),
                  "specialised stage launch");
    return QSIM_OK;
}


// Two-state stages of the adjoint reverse sweep (complex64, tiles of
// 2^(9 + W)): kernels for every tile stage, compiled or found in the cache.
int spec_dual_prepare(const std::vector<Stage> &stages, int n, int W, DualSpec &out) {
    const auto groups = stage_groups(stages.size());
    const uint64_t ntiles = uint64_t(1) << (n - (LANE_BITS + REG_BITS + W));
    std::vector<std::string> keys(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        std::string &k = keys[gi];
        k = "dual";
        put(k, n);
        put(k, W);
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            put(k, i);
            put_stage(k, stages[i]);
        }
    }
    auto source_of = [&](size_t gi) {
        Gen g;
        g.C = "float2";
        g.W = W;
        g.o << kPrelude;
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            const Stage &st = stages[i];
            if (st.plain) continue;
            g.stage(st, dual_kernel_name(i), std::max<int>(1, int(st.pool.size())), 2, true, ntiles);
        }
        return g.o.str();
    };
    std::vector<std::shared_ptr<SpecLib>> libs;
    QSIM_TRY(get_libs(groups, keys, source_of, libs));
    out.libs.assign(libs.begin(), libs.end());
    out.kern.assign(stages.size(), nullptr);
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            if (stages[i].plain) continue;
            cudaKernel_t k = nullptr;
            QSIM_CUDA_TRY(cudaLibraryGetKernel(&k, libs[gi]->lib, dual_kernel_name(i).c_str()),
                          "specialised two-state stage kernel");
            out.kern[i] = k;
        }
    return QSIM_OK;
}

int spec_dual_launch(const DualSpec &d, const Stage &st, size_t i, float2 *psi, float2 *lam, double *partial, int n,
                     int W, cudaStream_t s) {
    // parameter block: { float2 c[max(1, pool)]; float gv[max(1, grads)][3]; }
    std::vector<unsigned char> b;
    const size_t ng = std::max<size_t>(1, st.grads.size());
    pack_coefficients(st, QSIM_C64, b, ng * 12);
    const size_t off = std::max<size_t>(1, st.pool.size()) * 8;
    for (size_t g = 0; g < st.grads.size(); ++g) {
        const float gv[3] = {float(st.grads[g].v[0]), float(st.grads[g].v[1]), float(st.grads[g].v[2])};
        memcpy(&b[off + g * 12], gv, 12);
    }
    b.resize((b.size() + 7) / 8 * 8, 0);  // the struct's size: a multiple of its 8-byte alignment
    const int nt = LANE_BITS + REG_BITS + W;
    const uint64_t ntiles = uint64_t(1) << (n - nt);
    const size_t smem = (size_t(1) << nt) * sizeof(float2);
    const void *f = reinterpret_cast<const void *>(d.kern[i]);
    void *args[4] = {&psi, &lam, &partial, b.data()};
    QSIM_CUDA_TRY(cudaLaunchKernel(f, dim3(unsigned(ntiles)), dim3(32u << W), args, smem, s),
                  "specialised two-state stage launch");
    return QSIM_OK;
}

}  // namespace qsim

extern "C" QSIM_API int qsim_spec_stats(double *compile_s, uint64_t *compiles, uint64_t *cache_hits) {
    std::lock_guard<std::mutex> lk(qsim::g_cache_mu);
    if (compile_s) *compile_s = qsim::g_compile_s;
    if (compiles) *compiles = qsim::g_compiles;
    if (cache_hits) *cache_hits = qsim::g_hits;
    return QSIM_OK;
}

extern "C" QSIM_API int qsim_plan_source(const qsim_plan *p, int dtype, char *buf, size_t len, size_t *needed) {
    using namespace qsim;
    if (!p || !p->staged) return set_error(QSIM_EINVAL, "not a staged plan");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return set_error(QSIM_EINVAL, "dtype %d", dtype);
    const std::string src = spec_source(*p->staged, dtype, 0, p->staged->stages.size());
    if (needed) *needed = src.size() + 1;
    if (buf && len) {
        const size_t n = std::min(len - 1, src.size());
        memcpy(buf, src.data(), n);
        buf[n] = 0;
    }
    return QSIM_OK;
}

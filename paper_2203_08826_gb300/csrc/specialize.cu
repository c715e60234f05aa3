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
// as a by-value parameter block (read straight from the constant bank by the
// FMAs), so two circuits of the same structure with other angles share one
// compiled module.  Modules are cached by their source text.
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
)";

// Writes the source of one tile stage as kernel `name`.
struct Gen {
    std::ostringstream o;
    const char *C;  // "float2" / "double2"
    int W;

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
    void ctrl_open(const StageOp &op) {
        if (op.tmask) o << "    if ((base & 0x" << std::hex << op.tmask << std::dec << "ull) == 0x" << std::hex
                        << op.tmask << std::dec << "ull) {\n";
        else o << "    {\n";
    }
    static bool rok(int j, int rneed) { return (j & rneed) == rneed; }
    std::string coef(int i) const { return "p.c[" + std::to_string(i) + "]"; }

    void u1_reg(int rb, int moff, int rneed) {
        for (int i = 0; i < (1 << REG_BITS); ++i) {
            if ((i >> rb) & 1 || !rok(i, rneed)) continue;
            o << "        u1(v[" << i << "], v[" << (i | (1 << rb)) << "], " << coef(moff) << ", " << coef(moff + 1)
              << ", " << coef(moff + 2) << ", " << coef(moff + 3) << ");\n";
        }
    }
    // 1-qubit gate on lane bit l; `ok` guards the update (every lane shuffles)
    void u1_lane(int l, int moff, int rneed, bool guarded) {
        o << "    {\n        const bool hi = (lane >> " << l << ") & 1;\n";
        o << "        const " << C << " cs = hi ? " << coef(moff + 3) << " : " << coef(moff) << ";\n";
        o << "        const " << C << " co = hi ? " << coef(moff + 2) << " : " << coef(moff + 1) << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j) {
            if (!rok(j, rneed)) continue;
            o << "        { const " << C << " t = shfl_c(v[" << j << "], " << (1 << l) << "); ";
            if (guarded) o << "if (ok) ";
            o << "v[" << j << "] = cmad(co, t, cmul(cs, v[" << j << "])); }\n";
        }
        o << "    }\n";
    }

    void op_u2(const StageOp &op) {
        const bool la = op.a < POS_REG, lb = op.b < POS_REG;
        const int m = op.moff;
        if (!la && !lb) {  // two register targets: the interpreter's u2_reg
            const int JA = op.a - POS_REG, JB = op.b - POS_REG;
            ctrl_open(op);
            o << "        const " << C << " *m = &" << coef(m) << ";\n";
            for (int i = 0; i < (1 << REG_BITS); ++i) {
                if (i & ((1 << JA) | (1 << JB)) || !rok(i, op.rneed)) continue;
                o << "        u2(v[" << i << "], v[" << (i | (1 << JB)) << "], v[" << (i | (1 << JA)) << "], v["
                  << (i | (1 << JA) | (1 << JB)) << "], m);\n";
            }
            o << "    }\n";
            return;
        }
        o << "    {\n";
        o << "        const bool ok = " << (op.tmask ? "" : "true") ;
        if (op.tmask) o << "(base & 0x" << std::hex << op.tmask << "ull) == 0x" << op.tmask << std::dec << "ull";
        o << ";\n";
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
                o << "        { const " << C << " x0 = v[" << i << "], x1 = v[" << i1 << "];\n";
                o << "          const " << C << " y0 = shfl_c(x0, " << (1 << l) << "), y1 = shfl_c(x1, " << (1 << l)
                  << ");\n";
                o << "          if (ok) { v[" << i << "] = cmad(m3, y1, cmad(m2, y0, cmad(m1, x1, cmul(m0, x0))));\n";
                o << "                    v[" << i1 << "] = cmad(m7, y1, cmad(m6, y0, cmad(m5, x1, cmul(m4, x0)))); } }\n";
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
                o << "        { const " << C << " p1 = shfl_c(v[" << j << "], " << ma << "), p2 = shfl_c(v[" << j
                  << "], " << mb << "), p3 = shfl_c(v[" << j << "], " << (ma | mb) << ");\n";
                o << "          if (ok) v[" << j << "] = cmad(m3, p3, cmad(m2, p2, cmad(m1, p1, cmul(m0, v[" << j
                  << "])))); }\n";
            }
        }
        o << "    }\n";
    }

    void op_diag(const StageOp &op) {
        ctrl_open(op);
        if (op.k == 0) {
            for (int j = 0; j < (1 << REG_BITS); ++j) {
                if (!rok(j, op.rneed)) continue;
                if (op.flags & 1) o << "        v[" << j << "] = neg(v[" << j << "]);\n";
                else o << "        v[" << j << "] = cmul(" << coef(op.moff) << ", v[" << j << "]);\n";
            }
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
            o << "        v[" << j << "] = cmul(p.c[" << op.moff << " + (st | " << sj << ")], v[" << j << "]);\n";
        }
        o << "    }\n";
    }

    void op_neg(const Stage &st, const StageOp &op) {
        o << "    {\n        unsigned flip = 0u;\n";
        for (int e = 0; e < op.k; ++e) {
            const uint64_t tm = st.aux[size_t(op.moff + 2 * e)];
            const uint32_t pat = uint32_t(st.aux[size_t(op.moff + 2 * e + 1)]);
            if (tm == 0) o << "        flip ^= " << pat << "u;\n";
            else o << "        if ((base & 0x" << std::hex << tm << "ull) == 0x" << tm << std::dec << "ull) flip ^= " << pat
                   << "u;\n";
        }
        for (int j = 0; j < (1 << REG_BITS); ++j)
            o << "        if (flip & " << (1u << j) << "u) v[" << j << "] = neg(v[" << j << "]);\n";
        o << "    }\n";
    }

    void exchange(const Phase &from, const Phase &to) {
        o << "    {\n        unsigned lb = (unsigned)lane";
        for (int i = 0; i < W; ++i) o << " | (((unsigned)warp >> " << i << " & 1u) << " << (LANE_BITS + from.wslot[i]) << ")";
        o << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j) o << "        tile[lb | " << smem_offset(from, j) << "u] = v[" << j << "];\n";
        o << "        __syncthreads();\n        lb = (unsigned)lane";
        for (int i = 0; i < W; ++i) o << " | (((unsigned)warp >> " << i << " & 1u) << " << (LANE_BITS + to.wslot[i]) << ")";
        o << ";\n";
        for (int j = 0; j < (1 << REG_BITS); ++j) o << "        v[" << j << "] = tile[lb | " << smem_offset(to, j) << "u];\n";
        o << "        __syncthreads();\n    }\n";
        set_base(to);
    }

    // the whole kernel of one tile stage; its parameter block holds ncoef
    // coefficients (at least one)
    void stage(const Stage &st, const std::string &name, int ncoef, int min_blocks) {
        o << "struct P_" << name << " { " << C << " c[" << ncoef << "]; };\n";
        o << "extern \"C\" __global__ void __launch_bounds__(" << (32 << W) << ", " << min_blocks << ") " << name
          << "(" << C << " *__restrict__ psi, const __grid_constant__ P_" << name << " p) {\n";
        o << "    extern __shared__ " << C << " tile[];\n";
        o << "    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;\n";
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
        o << "    {\n        const " << C << " *g = psi + base;\n";
        for (int j = 0; j < (1 << REG_BITS); ++j)
            o << "        v[" << j << "] = g[0x" << std::hex << reg_offset(st.phases[size_t(ph)], j) << std::dec << "ull];\n";
        o << "    }\n";
        for (const StageOp &op : st.ops) {
            switch (op.type) {
                case SOP_EXCHANGE:
                    exchange(st.phases[size_t(ph)], st.phases[size_t(op.a)]);
                    ph = op.a;
                    break;
                case SOP_U1:
                    if (op.a >= POS_REG) {
                        ctrl_open(op);
                        u1_reg(op.a - POS_REG, op.moff, op.rneed);
                        o << "    }\n";
                    } else {
                        o << "    {\n        const bool ok = ";
                        if (op.tmask) o << "(base & 0x" << std::hex << op.tmask << "ull) == 0x" << op.tmask << std::dec << "ull";
                        else o << "true";
                        o << ";\n";
                        u1_lane(op.a, op.moff, op.rneed, op.tmask != 0);
                        o << "    }\n";
                    }
                    break;
                case SOP_U1R: {
                    int off = op.moff;
                    o << "    {\n";
                    for (int b = 0; b < REG_BITS; ++b)
                        if (op.a & (1 << b)) {
                            u1_reg(b, off, 0);
                            off += 4;
                        }
                    o << "    }\n";
                    break;
                }
                case SOP_U1L: {
                    int off = op.moff;
                    for (int l = 0; l < LANE_BITS; ++l)
                        if (op.a & (1 << l)) {
                            u1_lane(l, off, 0, false);
                            off += 4;
                        }
                    break;
                }
                case SOP_U2: op_u2(op); break;
                case SOP_DIAG: op_diag(op); break;
                case SOP_NEG: op_neg(st, op); break;
                default: break;  // gradient ops never reach a specialised plan
            }
        }
        o << "    {\n        " << C << " *g = psi + base;\n";
        for (int j = 0; j < (1 << REG_BITS); ++j)
            o << "        g[0x" << std::hex << reg_offset(st.phases[size_t(ph)], j) << std::dec << "ull] = v[" << j << "];\n";
        o << "    }\n}\n";
    }
};

std::mutex g_cache_mu;
std::map<std::string, std::shared_ptr<SpecLib>> g_cache;  // program source -> library
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

}  // namespace

// Source of the tile stages [i0, i1) of a staged plan for one dtype.
std::string spec_source(const StagedPlan &sp, int dtype, size_t i0, size_t i1) {
    Gen g;
    g.C = dtype == QSIM_C64 ? "float2" : "double2";
    g.W = sp.W;
    g.o << kPrelude;
    const int min_blocks = dtype == QSIM_C64 ? (sp.W <= 3 ? 3 : 2) : 1;
    for (size_t i = i0; i < i1; ++i) {
        const Stage &st = sp.stages[i];
        if (st.plain) continue;
        g.stage(st, kernel_name(i), std::max<int>(1, int(st.pool.size())), min_blocks);
    }
    return g.o.str();
}

// Compiles (or finds in the cache) the kernels of every tile stage and
// packs each stage's coefficient block.
int spec_prepare(StagedPlan &sp, int dtype) {
    StagedPlan::Spec &S = sp.spec[dtype];
    if (S.ready) return QSIM_OK;
    const size_t ns = sp.stages.size();
    // groups of about 4 stages: compiled in parallel, cached separately
    const size_t per = 4;
    std::vector<std::pair<size_t, size_t>> groups;
    for (size_t i = 0; i < ns; i += per) groups.push_back({i, std::min(ns, i + per)});
    std::vector<std::string> srcs(groups.size());
    std::vector<std::shared_ptr<SpecLib>> libs(groups.size());
    std::vector<size_t> todo;
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        srcs[gi] = spec_source(sp, dtype, groups[gi].first, groups[gi].second);
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(srcs[gi]);
        if (it != g_cache.end()) {
            libs[gi] = it->second;
            ++g_hits;
        } else {
            todo.push_back(gi);
        }
    }
    std::vector<std::string> cubins(groups.size()), logs(groups.size());
    std::vector<int> rcs(groups.size(), QSIM_OK);
    const auto t0 = std::chrono::steady_clock::now();
    {
        std::vector<std::thread> th;
        const size_t nthreads = std::max<size_t>(1, std::min<size_t>(todo.size(), std::thread::hardware_concurrency()));
        std::atomic<size_t> next{0};
        for (size_t t = 0; t < nthreads; ++t)
            th.emplace_back([&] {
                for (size_t k; (k = next.fetch_add(1)) < todo.size();) {
                    const size_t gi = todo[k];
                    rcs[gi] = compile(srcs[gi], cubins[gi], logs[gi]);
                }
            });
        for (std::thread &t : th) t.join();
    }
    for (size_t gi : todo) {
        if (rcs[gi] != QSIM_OK)
            return set_error(QSIM_ECUDA, "specialised stage compile failed: %.400s", logs[gi].c_str());
        auto L = std::make_shared<SpecLib>();
        QSIM_CUDA_TRY(cudaLibraryLoadData(&L->lib, cubins[gi].data(), nullptr, nullptr, 0, nullptr, nullptr, 0),
                      "load specialised stages");
        libs[gi] = L;
        std::lock_guard<std::mutex> lk(g_cache_mu);
        if (g_cache.size() >= CACHE_MAX) g_cache.erase(g_cache.begin());
        g_cache[srcs[gi]] = L;
        ++g_compiles;
    }
    if (!todo.empty())
        g_compile_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    S.libs.assign(libs.begin(), libs.end());
    S.kern.assign(ns, nullptr);
    S.params.assign(ns, {});
    const size_t eb = dtype == QSIM_C64 ? 8 : 16;
    for (size_t gi = 0; gi < groups.size(); ++gi)
        for (size_t i = groups[gi].first; i < groups[gi].second; ++i) {
            const Stage &st = sp.stages[i];
            if (st.plain) continue;
            cudaKernel_t k = nullptr;
            QSIM_CUDA_TRY(cudaLibraryGetKernel(&k, libs[gi]->lib, kernel_name(i).c_str()), "specialised stage kernel");
            S.kern[i] = k;
            std::vector<unsigned char> &b = S.params[i];
            b.assign(std::max<size_t>(1, st.pool.size()) * eb, 0);
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

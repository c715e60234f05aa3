// Fusion planning (Sec. 3.2) and plan execution.
//
// QSIM_FUSE_GREEDY2 is the paper's fusion: walk the gate list and multiply
// each 1- or 2-qubit gate into the most recent fused gate on its qubits when
// the union stays within two qubits and no later fused gate on those qubits
// would be overtaken.  The other modes live in their own translation units
// and share the block bookkeeping defined here.
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "plan.h"

namespace qsim {

// Matrix of a gate (targets + controls) on the ordered qubit list `qs`
// (qs[0] = most significant bit of the result's index).
std::vector<cd> embed_gate(const GateRec &g, const std::vector<int> &qs) {
    const int b = int(qs.size());
    const size_t D = size_t(1) << b;
    auto pos = [&](int q) {
        for (int i = 0; i < b; ++i)
            if (qs[i] == q) return b - 1 - i;  // bit position within the block index
        return -1;
    };
    std::vector<int> tpos(g.k), cpos(g.nc);
    for (int i = 0; i < g.k; ++i) tpos[i] = pos(g.targets[i]);
    for (int i = 0; i < g.nc; ++i) cpos[i] = pos(g.controls[i]);
    const size_t d = size_t(1) << g.k;
    std::vector<cd> out(D * D, cd(0.0));
    for (size_t col = 0; col < D; ++col) {
        bool active = true;
        for (int i = 0; i < g.nc; ++i)
            if (!((col >> cpos[i]) & 1)) active = false;
        if (!active) {
            out[col * D + col] = 1.0;
            continue;
        }
        size_t jc = 0;  // gate column index read from the block column
        for (int i = 0; i < g.k; ++i) jc = (jc << 1) | ((col >> tpos[i]) & 1);
        size_t rest = col;
        for (int i = 0; i < g.k; ++i) rest &= ~(size_t(1) << tpos[i]);
        for (size_t jr = 0; jr < d; ++jr) {
            size_t row = rest;
            for (int i = 0; i < g.k; ++i)
                if ((jr >> (g.k - 1 - i)) & 1) row |= size_t(1) << tpos[i];
            out[row * D + col] += g.m[jr * d + jc];
        }
    }
    return out;
}

// C = A * B for D x D row-major matrices
std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, size_t D) {
    std::vector<cd> C(D * D, cd(0.0));
    for (size_t i = 0; i < D; ++i)
        for (size_t k = 0; k < D; ++k) {
            const cd a = A[i * D + k];
            if (a == cd(0.0)) continue;
            for (size_t j = 0; j < D; ++j) C[i * D + j] += a * B[k * D + j];
        }
    return C;
}

// Re-express a block matrix on a larger ordered qubit list.
std::vector<cd> widen(const std::vector<cd> &m, const std::vector<int> &from, const std::vector<int> &to) {
    GateRec g;
    g.k = int(from.size());
    g.nc = 0;
    for (int i = 0; i < g.k; ++i) g.targets[i] = from[i];
    g.m = m;
    return embed_gate(g, to);
}

int build_greedy2(const qsim_circuit &c, qsim_plan &p) {
    std::vector<int> last(c.n, -1);  // index of the latest block touching each qubit
    for (size_t gi = 0; gi < c.gates.size(); ++gi) {
        const GateRec &g = c.gates[gi];
        std::vector<int> gq;
        for (int i = 0; i < g.k; ++i) gq.push_back(g.targets[i]);
        for (int i = 0; i < g.nc; ++i) gq.push_back(g.controls[i]);
        int F = -1;
        for (int q : gq) F = std::max(F, last[q]);
        bool merged = false;
        if (F >= 0 && gq.size() <= 2) {
            Block &B = p.blocks[F];
            std::vector<int> uni = B.qubits;
            for (int q : gq)
                if (std::find(uni.begin(), uni.end(), q) == uni.end()) uni.push_back(q);
            if (int(uni.size()) <= std::min(p.kmax, 2)) {
                // the qubits the gate adds must not have a block after F
                bool ok = true;
                for (int q : gq)
                    if (last[q] > F) ok = false;
                if (ok) {
                    std::sort(uni.begin(), uni.end(), std::greater<int>());
                    const size_t D = size_t(1) << uni.size();
                    std::vector<cd> bm = widen(B.m, B.qubits, uni);
                    B.m = matmul(embed_gate(g, uni), bm, D);
                    B.qubits = uni;
                    B.gates.push_back(int(gi));
                    // qubits of B outside the gate may already have later blocks
                    for (int q : gq) last[q] = F;
                    merged = true;
                }
            }
        }
        if (!merged) {
            Block B;
            B.qubits = gq;
            std::sort(B.qubits.begin(), B.qubits.end(), std::greater<int>());
            B.m = embed_gate(g, B.qubits);
            B.gates.push_back(int(gi));
            p.blocks.push_back(std::move(B));
            for (int q : gq) last[q] = int(p.blocks.size()) - 1;
        }
    }
    return QSIM_OK;
}

// Per-dtype device copies of the dense matrices of a block-list plan.
static int prepare_ops(qsim_plan &p, int dtype, cudaStream_t st) {
    PlanDev &dv = p.dev[dtype];
    if (dv.ready) return QSIM_OK;
    dv.ops.clear();
    dv.mat_off.clear();
    std::vector<unsigned char> host;
    const size_t eb = dtype == QSIM_C64 ? 8 : 16;
    for (const Block &B : p.blocks) {
        Op op;
        std::vector<int> t(B.qubits.begin(), B.qubits.end());
        QSIM_TRY(classify(B.m, t.data(), int(t.size()), nullptr, 0, op));
        size_t off = size_t(-1);
        if (op.type == Op::DENSE && op.k >= 2) {
            off = host.size();
            const size_t d = size_t(1) << op.k;
            host.resize(off + d * d * eb);
            for (size_t i = 0; i < d * d; ++i) {
                if (dtype == QSIM_C64) {
                    float v[2] = {float(op.m[i].real()), float(op.m[i].imag())};
                    memcpy(&host[off + i * eb], v, 8);
                } else {
                    double v[2] = {op.m[i].real(), op.m[i].imag()};
                    memcpy(&host[off + i * eb], v, 16);
                }
            }
        }
        dv.ops.push_back(std::move(op));
        dv.mat_off.push_back(off);
    }
    if (!host.empty()) {
        QSIM_CUDA_TRY(dev_alloc(&dv.mats, host.size()), "plan matrices");
        QSIM_CUDA_TRY(cudaMemcpyAsync(dv.mats, host.data(), host.size(), cudaMemcpyHostToDevice, st),
                      "plan matrices upload");
        QSIM_CUDA_TRY(cudaStreamSynchronize(st), "plan upload sync");
    }
    dv.ready = true;
    return QSIM_OK;
}

int run_block_plan(qsim_state *s, qsim_plan &p) {
    QSIM_TRY(prepare_ops(p, s->dtype, s->stream));
    PlanDev &dv = p.dev[s->dtype];
    for (size_t i = 0; i < dv.ops.size(); ++i) {
        void *mat = dv.mat_off[i] == size_t(-1) ? nullptr : static_cast<char *>(dv.mats) + dv.mat_off[i];
        QSIM_TRY(launch_op(s->amps, s->n, s->dtype, dv.ops[i], s->stream, mat));
    }
    return QSIM_OK;
}

}  // namespace qsim

using namespace qsim;

qsim_plan::~qsim_plan() {
    for (PlanDev &d : dev)
        if (d.mats) cudaFree(d.mats);
    release_staged();
    release_tc();
}

extern "C" {

int qsim_plan_build(const qsim_circuit *c, int kmax, int mode, qsim_plan **out) {
    if (!c || !out) return set_error(QSIM_EINVAL, "NULL argument");
    *out = nullptr;
    if (kmax < 1 || kmax > QSIM_MAX_TARGETS) return set_error(QSIM_EINVAL, "kmax=%d outside 1..6", kmax);
    if (c->n > 34) return set_error(QSIM_EINVAL, "plans act on states of at most 34 qubits (circuit has %d)", c->n);
    const bool specialize = (mode & QSIM_PLAN_SPECIALIZE) != 0;
    mode &= ~QSIM_PLAN_SPECIALIZE;
    if (specialize && mode != QSIM_FUSE_STAGED)
        return set_error(QSIM_EINVAL, "QSIM_PLAN_SPECIALIZE applies to staged plans only");
    qsim_plan *p = new qsim_plan();
    p->n = c->n;
    p->mode = mode;
    p->kmax = kmax;
    p->ngates = int(c->gates.size());
    int rc = QSIM_OK;
    switch (mode) {
        case QSIM_FUSE_GREEDY2: rc = build_greedy2(*c, *p); break;
        case QSIM_FUSE_STAGED: rc = build_staged(*c, *p); break;
        case QSIM_FUSE_TC: rc = build_tc(*c, *p); break;
        default: rc = set_error(QSIM_EINVAL, "unknown fusion mode %d", mode);
    }
    if (rc == QSIM_OK && specialize) staged_set_specialized(*p);
    if (rc != QSIM_OK) {
        delete p;
        return rc;
    }
    *out = p;
    return QSIM_OK;
}

int qsim_plan_destroy(qsim_plan *p) {
    delete p;
    return QSIM_OK;
}

int qsim_plan_info(const qsim_plan *p, int *nsweeps, int *ngates, int *mode) {
    if (!p) return set_error(QSIM_EINVAL, "plan is NULL");
    if (nsweeps) *nsweeps = p->nsweeps();
    if (ngates) *ngates = p->ngates;
    if (mode) *mode = p->mode | (staged_specialized(*p) ? QSIM_PLAN_SPECIALIZE : 0);
    return QSIM_OK;
}

int qsim_plan_describe(const qsim_plan *p, char *buf, size_t len) {
    if (!p || !buf || len == 0) return set_error(QSIM_EINVAL, "NULL argument");
    std::string out;
    if (p->mode == QSIM_FUSE_STAGED) {
        staged_describe(*p, out);
    } else if (p->mode == QSIM_FUSE_TC) {
        tc_describe(*p, out);
    } else {
        out = "greedy2 plan: " + std::to_string(p->blocks.size()) + " fused gates\n";
        for (size_t i = 0; i < p->blocks.size(); ++i) {
            out += "  " + std::to_string(i) + " [";
            for (int q : p->blocks[i].qubits) out += std::to_string(q) + " ";
            out += "] gates=" + std::to_string(p->blocks[i].gates.size()) + "\n";
        }
    }
    const size_t n = std::min(len - 1, out.size());
    memcpy(buf, out.data(), n);
    buf[n] = 0;
    return QSIM_OK;
}

int qsim_plan_block(const qsim_plan *p, int i, int *k, int *targets, double *matrix_out) {
    if (!p) return set_error(QSIM_EINVAL, "plan is NULL");
    if (i < 0 || i >= int(p->blocks.size())) return set_error(QSIM_EINVAL, "block %d outside the plan", i);
    const Block &B = p->blocks[i];
    if (k) *k = int(B.qubits.size());
    if (targets)
        for (size_t j = 0; j < B.qubits.size(); ++j) targets[j] = B.qubits[j];
    if (matrix_out)
        for (size_t j = 0; j < B.m.size(); ++j) {
            matrix_out[2 * j] = B.m[j].real();
            matrix_out[2 * j + 1] = B.m[j].imag();
        }
    return QSIM_OK;
}

// Candidates: complex64 -- staged tiles (FP32 on the CUDA cores, tiles of
// 2^12 and 2^13 amplitudes) and tensor-core plans with every pass in BF16x3
// (6-qubit windows), 3xTF32 (5-qubit windows) or FP32 on the CUDA cores
// (6-qubit windows); complex128 -- staged tiles against one sweep per gate
// (greedy fusion limited to 1 qubit).  Each runs once from |0...0> (warm-up,
// and the state whose error is measured when max_err > 0 or a table is
// asked for), then `reps` timed times.
// Error reference: for a complex64 state of at most 30 qubits whose
// complex128 copy fits in free device memory, the circuit run gate by gate
// in complex128 (FP64 truth); otherwise the first candidate's result.
// Mixed precision per block: when the BF16x3 plan misses the bound and the
// FP32 one meets it, their measured errors give a per-pass error for each
// precision (error of the whole plan / its passes); the fewest passes that
// must run in FP32 for the predicted error (sum over passes) to stay within
// the bound run in FP32, the others in BF16x3, and that plan is measured as
// one more candidate.
static int autotune_impl(const qsim_circuit *c, qsim_state *s, int reps, double max_err, qsim_plan **out,
                         qsim_tune_entry *table, int table_cap, int *table_len) {
    if (!c || !s || !out) return set_error(QSIM_EINVAL, "NULL argument");
    if (c->n != s->n) return set_error(QSIM_EINVAL, "circuit has %d qubits, state %d", c->n, s->n);
    if (table_cap > 0 && !table) return set_error(QSIM_EINVAL, "table is NULL");
    *out = nullptr;
    if (table_len) *table_len = 0;
    if (reps < 1) reps = 1;
    struct Cand {
        int mode, kmax;
        int fp32;  // tensor-core plans: -1 every pass at the window's split, -2 every pass in FP32, k >= 0: k passes in FP32
    };
    std::vector<Cand> cands = {{QSIM_FUSE_STAGED, 3, -1}, {QSIM_FUSE_STAGED, 4, -1}};
    if (c->n >= SPECIALIZE_MIN_QUBITS) {
        // stage kernels compiled for the plan: worth their compile time on
        // large states only
        cands.push_back({QSIM_FUSE_STAGED | QSIM_PLAN_SPECIALIZE, 3, -1});
        cands.push_back({QSIM_FUSE_STAGED | QSIM_PLAN_SPECIALIZE, 4, -1});
    }
    if (s->dtype == QSIM_C64) {
        cands.push_back({QSIM_FUSE_TC, 6, -1});
        cands.push_back({QSIM_FUSE_TC, 5, -1});
        if (max_err > 0 || table_cap > 0) cands.push_back({QSIM_FUSE_TC, 6, -2});  // only an accuracy option
    } else {
        cands.push_back({QSIM_FUSE_GREEDY2, 1, -1});
    }
    const bool measure = max_err > 0 || table_cap > 0;
    const size_t bytes = s->size() * s->amp_bytes();
    // FP64 reference: the gate-by-gate complex128 run
    qsim_state *ref64 = nullptr;
    struct R64Guard {
        qsim_state *&p;
        ~R64Guard() {
            if (p) qsim_state_destroy(p);
        }
    } r64g{ref64};
    if (measure && s->dtype == QSIM_C64 && s->n <= 30) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && fr > 2 * s->size() * 16 + (size_t(1) << 30) &&
            qsim_state_create(s->n, QSIM_C128, nullptr, s->stream, &ref64) == QSIM_OK) {
            if (qsim_state_init(ref64, QSIM_INIT_ZERO, 0, nullptr) != QSIM_OK || qsim_run(ref64, c) != QSIM_OK) {
                qsim_state_destroy(ref64);
                ref64 = nullptr;
            }
        }
        cudaGetLastError();
    }
    void *ref = nullptr;
    bool have_ref = false;
    if (measure && !ref64 && dev_alloc(&ref, bytes) != cudaSuccess) {
        cudaGetLastError();  // not enough memory for the reference copy: errors are not measured
        ref = nullptr;
    }
    struct RefGuard {
        void *p;
        ~RefGuard() {
            if (p) cudaFree(p);
        }
    } rg{ref};
    const size_t np = reduce_partials_needed(s->n);
    cudaEvent_t e0, e1;
    QSIM_CUDA_TRY(cudaEventCreate(&e0), "event");
    QSIM_CUDA_TRY(cudaEventCreate(&e1), "event");
    qsim_plan *best = nullptr;
    float best_ms = 1e30f;
    int nt = 0;
    double err_bf = -1, err_fp = -1;  // whole-plan errors of the BF16x3 and FP32 6-qubit plans
    int passes_bf = 0;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        const Cand cd_ = cands[ci];
        qsim_tune_entry ent{cd_.mode, cd_.kmax, -1.0, -1.0, -1.0, ref64 ? 1 : 0, 0, 0};
        qsim_plan *p = nullptr;
        bool ok = qsim_plan_build(c, cd_.kmax, cd_.mode, &p) == QSIM_OK;  // e.g. too narrow for a tile
        if (ok && cd_.mode == QSIM_FUSE_TC && p->tc) {
            const int m = tc_nsweeps(*p);
            std::vector<int> prec(size_t(m), -1);
            for (int i = 0; i < m; ++i) prec[size_t(i)] = tc_pass_precision(*p, i);
            int nfp = 0;
            for (int i = 0; i < m; ++i)
                if (cd_.fp32 == -2 || (cd_.fp32 >= 0 && nfp < cd_.fp32)) {
                    prec[size_t(i)] = QSIM_PREC_FP32;
                    ++nfp;
                }
            ok = tc_set_precisions(*p, prec) == QSIM_OK;
            ent.npasses = m;
            ent.nfp32 = nfp;
        }
        ok = ok && qsim_state_init(s, QSIM_INIT_ZERO, 0, nullptr) == QSIM_OK && qsim_apply_fused(s, p) == QSIM_OK;
        if (ok && (ref64 || ref)) {
            if (!ref64 && !have_ref) {
                ok = cudaMemcpyAsync(ref, s->amps, bytes, cudaMemcpyDeviceToDevice, s->stream) == cudaSuccess;
                have_ref = ok;
                ent.err = ent.max_abs = 0.0;
            } else if (s->ensure_scratch((2 * np + 2) * sizeof(double)) == QSIM_OK) {
                double *part = static_cast<double *>(s->scratch);
                double host[2] = {0, 0};
                const int rc = ref64 ? launch_diff_norm2_c64_c128(s->amps, ref64->amps, s->n, part, part + 2 * np,
                                                                  s->stream)
                                     : launch_diff_norm2(s->amps, ref, s->n, s->dtype, part, part + 2 * np, s->stream);
                ok = rc == QSIM_OK &&
                     cudaMemcpyAsync(host, part + 2 * np, sizeof host, cudaMemcpyDeviceToHost, s->stream) ==
                         cudaSuccess &&
                     cudaStreamSynchronize(s->stream) == cudaSuccess;
                ent.err = std::sqrt(host[0]);
                ent.max_abs = std::sqrt(host[1]);
            }
        }
        if (ok) {
            cudaEventRecord(e0, s->stream);
            int rc = QSIM_OK;
            for (int r = 0; r < reps && rc == QSIM_OK; ++r) rc = qsim_apply_fused(s, p);
            cudaEventRecord(e1, s->stream);
            ok = rc == QSIM_OK && cudaEventSynchronize(e1) == cudaSuccess;
        }
        float ms = 0;
        if (ok) {
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            ent.ms = ms;
        }
        if (nt < table_cap) table[nt] = ent;
        ++nt;
        if (ok && cd_.mode == QSIM_FUSE_TC && cd_.kmax == 6 && cd_.fp32 == -1) {
            err_bf = ent.err;
            passes_bf = ent.npasses;
        }
        if (ok && cd_.mode == QSIM_FUSE_TC && cd_.fp32 == -2) {
            err_fp = ent.err;
            // per-block precision: how many passes must run in FP32
            if (max_err > 0 && err_bf > max_err && err_fp >= 0 && err_fp < max_err && passes_bf > 0) {
                const double x = double(passes_bf) * (err_bf - max_err) / (err_bf - err_fp);
                const int nfp = std::min(passes_bf, int(std::ceil(x)));
                if (nfp > 0 && nfp < passes_bf) cands.push_back({QSIM_FUSE_TC, 6, nfp});
            }
        }
        // within the bound: the error was measured and is small enough, or no bound
        const bool accurate = max_err <= 0 || (ent.err >= 0 && ent.err <= max_err);
        if (ok && accurate && ms < best_ms) {
            if (best) qsim_plan_destroy(best);
            best = p;
            best_ms = ms;
        } else if (p) {
            qsim_plan_destroy(p);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (table_len) *table_len = std::min(nt, table_cap);
    if (!best) return set_error(QSIM_EUNSUPPORTED, "no fusion plan could run this circuit within the bound");
    best->tuned_ms = best_ms;
    *out = best;
    return QSIM_OK;
}

int qsim_plan_autotune(const qsim_circuit *c, qsim_state *s, int reps, qsim_plan **out, int *mode_out,
                       int *kmax_out, double *ms_out) {
    QSIM_TRY(autotune_impl(c, s, reps, 0.0, out, nullptr, 0, nullptr));
    if (mode_out) *mode_out = (*out)->mode;
    if (kmax_out) *kmax_out = (*out)->kmax;
    if (ms_out) *ms_out = (*out)->tuned_ms;
    return QSIM_OK;
}

int qsim_plan_autotune_ex(const qsim_circuit *c, qsim_state *s, int reps, double max_err, qsim_plan **out,
                          qsim_tune_entry *table, int table_cap, int *table_len) {
    return autotune_impl(c, s, reps, max_err, out, table, table_cap, table_len);
}

int qsim_apply_fused(qsim_state *s, const qsim_plan *pc) {
    if (!s || !pc) return set_error(QSIM_EINVAL, "NULL argument");
    qsim_plan *p = const_cast<qsim_plan *>(pc);
    if (p->n != s->n) return set_error(QSIM_EINVAL, "plan has %d qubits, state %d", p->n, s->n);
    switch (p->mode) {
        case QSIM_FUSE_GREEDY2: return run_block_plan(s, *p);
        case QSIM_FUSE_STAGED: return run_staged(s, *p);
        case QSIM_FUSE_TC: return run_tc(s, *p);
    }
    return set_error(QSIM_EINVAL, "bad plan mode");
}

}  // extern "C"

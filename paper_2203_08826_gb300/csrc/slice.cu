// Sliced states (Sec. 3.1, the multi-GPU scheme and its figure): the state is
// split by its top g "global" qubits into 2^g slices of L = n - g "local"
// qubits.  Gates whose targets are all local act on every slice on its own;
// a control or a diagonal target on a global qubit only selects, per slice,
// which gate (or which part of a diagonal) applies there.  A dense or
// permutation gate on a global qubit first exchanges that qubit with a local
// one: slice pairs that differ in the global bit swap the halves in which the
// local bit differs from the global bit.
//
// The planner below turns a circuit into SWAP steps and local SEGMENTS (one
// fusion plan per distinct pattern of the global bits a segment reads).  The
// executors run the steps on slices that live in device memory (one GPU, or a
// caller that owns the slices of several ranks) or in host memory, streamed
// through the GPU in groups — the paper's scheme, where slices larger in total
// than device memory are copied to the GPU, updated and copied back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <set>
#include <vector>

#include "internal.h"
#include "plan.h"

namespace qsim {
namespace {

constexpr int SLICE_THREADS = 256;

int sm_count_s() { return device_sm_count(); }

__device__ __forceinline__ uint64_t insert_bit(uint64_t g, int l, uint64_t bit) {
    const uint64_t low = g & ((uint64_t(1) << l) - 1);
    return ((g >> l) << (l + 1)) | (bit << l) | low;
}

// a[x with bit l = 1] <-> b[x with bit l = 0]: the exchange of a global qubit
// (0 in a, 1 in b) with local qubit l.
template <typename C>
__global__ void k_exchange(C *__restrict__ a, C *__restrict__ b, uint64_t half, int l) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < half; g += stride) {
        const uint64_t i0 = insert_bit(g, l, 0);
        const uint64_t i1 = i0 | (uint64_t(1) << l);
        const C va = a[i1], vb = b[i0];
        a[i1] = vb;
        b[i0] = va;
    }
}

// complex64 with l >= 1: two neighbouring amplitudes (bit 0 differs, bit l
// equal) move as one 16-byte access; u indexes those pairs.
__global__ void k_exchange_c64x2(float4 *__restrict__ a, float4 *__restrict__ b, uint64_t pairs, int l) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t u = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < pairs; u += stride) {
        const uint64_t i0 = insert_bit(2 * u, l, 0) >> 1;  // float4 index of the bit-l = 0 pair
        const uint64_t i1 = i0 | (uint64_t(1) << (l - 1));
        const float4 va = a[i1], vb = b[i0];
        a[i1] = vb;
        b[i0] = va;
    }
}

// out[g] = slice[x_g] (pack) or slice[x_g] = in[g] (unpack), x_g = g with
// `bit` inserted at position l.
template <typename C, bool PACK>
__global__ void k_pack(C *__restrict__ slice, C *__restrict__ buf, uint64_t half, int l, uint64_t bit) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < half; g += stride) {
        const uint64_t x = insert_bit(g, l, bit);
        if (PACK)
            buf[g] = slice[x];
        else
            slice[x] = buf[g];
    }
}

unsigned grid_for(uint64_t work) {
    const uint64_t cap = uint64_t(sm_count_s()) * 8;
    const uint64_t want = (work + SLICE_THREADS - 1) / SLICE_THREADS;
    return unsigned(std::max<uint64_t>(1, std::min(cap, want)));
}

int launch_exchange(void *a, void *b, int L, int dtype, int l, cudaStream_t st) {
    const uint64_t half = uint64_t(1) << (L - 1);
    const size_t S = dtype == QSIM_C64 ? 8 : 16;
    LaunchScope ls(K_SLICE_EXCHANGE, st, 4.0 * double(half) * double(S));
    const bool al16 = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
    if (dtype == QSIM_C64 && l >= 1 && L >= 2 && al16)
        k_exchange_c64x2<<<grid_for(half / 2), SLICE_THREADS, 0, st>>>(static_cast<float4 *>(a),
                                                                        static_cast<float4 *>(b), half / 2, l);
    else if (dtype == QSIM_C64)
        k_exchange<float2><<<grid_for(half), SLICE_THREADS, 0, st>>>(static_cast<float2 *>(a), static_cast<float2 *>(b),
                                                                     half, l);
    else
        k_exchange<double2><<<grid_for(half), SLICE_THREADS, 0, st>>>(static_cast<double2 *>(a),
                                                                      static_cast<double2 *>(b), half, l);
    QSIM_CUDA_TRY(cudaGetLastError(), "slice exchange launch");
    return QSIM_OK;
}

int launch_pack(void *slice, void *buf, int L, int dtype, int l, int bit, bool pack, cudaStream_t st) {
    const uint64_t half = uint64_t(1) << (L - 1);
    const size_t S = dtype == QSIM_C64 ? 8 : 16;
    LaunchScope ls(K_SLICE_PACK, st, 2.0 * double(half) * double(S));
    const unsigned grid = grid_for(half);
    if (dtype == QSIM_C64) {
        auto *s = static_cast<float2 *>(slice);
        auto *b = static_cast<float2 *>(buf);
        if (pack)
            k_pack<float2, true><<<grid, SLICE_THREADS, 0, st>>>(s, b, half, l, uint64_t(bit));
        else
            k_pack<float2, false><<<grid, SLICE_THREADS, 0, st>>>(s, b, half, l, uint64_t(bit));
    } else {
        auto *s = static_cast<double2 *>(slice);
        auto *b = static_cast<double2 *>(buf);
        if (pack)
            k_pack<double2, true><<<grid, SLICE_THREADS, 0, st>>>(s, b, half, l, uint64_t(bit));
        else
            k_pack<double2, false><<<grid, SLICE_THREADS, 0, st>>>(s, b, half, l, uint64_t(bit));
    }
    QSIM_CUDA_TRY(cudaGetLastError(), "slice pack launch");
    return QSIM_OK;
}

// A gate of a segment in physical positions (classified form).
struct SegGate {
    Op op;
};

}  // namespace
}  // namespace qsim

// ------------------------------------------------------------------ plan
struct qsim_slice_plan {
    struct Step {
        int type = QSIM_SLICE_SEGMENT;
        int gbit = 0, lpos = 0;                // SWAP
        uint32_t keymask = 0;                  // SEGMENT: global bits the variants depend on
        int ngates = 0;                        // SEGMENT: gates of the source circuit in it
        std::map<uint32_t, qsim_circuit *> circuits;  // variant key -> local circuit (may be empty)
        std::map<uint32_t, qsim_plan *> plans;        // variant key -> plan (NULL: nothing to do)
    };
    int n = 0, g = 0, L = 0, kmax = 1, mode = 0;
    std::vector<Step> steps;
    std::vector<int> pos;  // logical qubit -> physical position after the last step
    ~qsim_slice_plan() {
        for (Step &s : steps) {
            for (auto &kv : s.circuits) qsim_circuit_destroy(kv.second);
            for (auto &kv : s.plans) qsim_plan_destroy(kv.second);
        }
    }
};

namespace qsim {
namespace {

// The local circuit of one segment for the slices whose global bits (masked
// by keymask) equal key: global controls decide whether a gate is present,
// global diagonal targets pick the sub-diagonal.
int segment_variant(const std::vector<SegGate> &gates, int L, uint32_t key, qsim_circuit **out) {
    QSIM_TRY(qsim_circuit_create(L, out));
    qsim_circuit *c = *out;
    auto gbit_of = [&](int p) { return int((key >> (p - L)) & 1u); };
    for (const SegGate &sg : gates) {
        const Op &op = sg.op;
        bool present = true;
        std::vector<int> lc;
        for (int i = 0; i < op.c; ++i) {
            const int p = op.controls[i];
            if (p >= L) {
                if (!gbit_of(p)) present = false;
            } else {
                lc.push_back(p);
            }
        }
        if (!present) continue;
        std::vector<int> lt;
        std::vector<cd> m;
        if (op.type == Op::DIAG) {
            // matrix index: targets[0] = MSB; fix the global target bits
            const int k = op.k;
            int gfix = 0;
            std::vector<int> lidx;  // matrix bit (from the MSB side) of each local target
            for (int t = 0; t < k; ++t) {
                const int p = op.targets[t];
                const int mb = k - 1 - t;
                if (p >= L) {
                    gfix |= gbit_of(p) << mb;
                } else {
                    lt.push_back(p);
                    lidx.push_back(mb);
                }
            }
            const int kl = int(lt.size());
            const size_t dl = size_t(1) << kl;
            std::vector<cd> d(dl);
            for (size_t j = 0; j < dl; ++j) {
                int full = gfix;
                for (int t = 0; t < kl; ++t)
                    if ((j >> (kl - 1 - t)) & 1) full |= 1 << lidx[t];
                d[j] = op.m[size_t(full)];
            }
            if (kl == 0) {
                // a phase z on this slice's control subspace: diag(1, z) on
                // one local control (the form a CZ classifies to), or, with
                // no local control, z on the whole slice
                if (d[0] == cd(1.0)) continue;
                if (!lc.empty()) {
                    lt.push_back(lc.back());
                    lc.pop_back();
                    d = {cd(1.0), d[0]};
                } else {
                    lt.push_back(0);
                    d = {d[0], d[0]};
                }
            }
            const size_t dd = size_t(1) << lt.size();
            m.assign(dd * dd, cd(0.0));
            for (size_t j = 0; j < dd; ++j) m[j * dd + j] = d[j];
        } else {
            for (int t = 0; t < op.k; ++t) {
                if (op.targets[t] >= L) return set_error(QSIM_EUNSUPPORTED, "slice: planner left a global target");
                lt.push_back(op.targets[t]);
            }
            const size_t d = size_t(1) << op.k;
            if (op.type == Op::DENSE) {
                m = op.m;
            } else {  // MONO
                m.assign(d * d, cd(0.0));
                for (size_t r = 0; r < d; ++r) m[r * d + size_t(op.perm[r])] = op.phase[r];
            }
        }
        std::vector<double> md(2 * m.size());
        for (size_t i = 0; i < m.size(); ++i) {
            md[2 * i] = m[i].real();
            md[2 * i + 1] = m[i].imag();
        }
        QSIM_TRY(qsim_circuit_add(c, QSIM_GATE_MATRIX, lt.data(), int(lt.size()), lc.data(), int(lc.size()), nullptr,
                                  -1, md.data()));
    }
    return QSIM_OK;
}

int close_segment(qsim_slice_plan &P, std::vector<SegGate> &gates, int ngates) {
    if (gates.empty()) return QSIM_OK;
    // the step joins the plan first, so that the plan owns whatever is built
    // for it even when a later variant fails
    P.steps.emplace_back();
    qsim_slice_plan::Step &st = P.steps.back();
    st.type = QSIM_SLICE_SEGMENT;
    st.ngates = ngates;
    for (const SegGate &sg : gates) {
        for (int i = 0; i < sg.op.c; ++i)
            if (sg.op.controls[i] >= P.L) st.keymask |= 1u << (sg.op.controls[i] - P.L);
        if (sg.op.type == Op::DIAG)
            for (int t = 0; t < sg.op.k; ++t)
                if (sg.op.targets[t] >= P.L) st.keymask |= 1u << (sg.op.targets[t] - P.L);
    }
    // every sub-mask of keymask is a variant, in increasing order
    uint32_t key = 0;
    while (true) {
        qsim_circuit *c = nullptr;
        int rc = segment_variant(gates, P.L, key, &c);
        if (c) st.circuits[key] = c;
        if (rc != QSIM_OK) return rc;
        qsim_plan *p = nullptr;
        if (!c->gates.empty()) QSIM_TRY(qsim_plan_build(c, P.kmax, P.mode, &p));
        st.plans[key] = p;
        if (key == st.keymask) break;
        key = (key - st.keymask) & st.keymask;
    }
    gates.clear();
    return QSIM_OK;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" {

int qsim_slice_plan_build(const qsim_circuit *c, int n_global, int kmax, int mode, int restore_layout,
                          qsim_slice_plan **out) {
    if (!c || !out) return set_error(QSIM_EINVAL, "NULL argument");
    *out = nullptr;
    const int n = c->n;
    if (n_global < 0 || n_global > QSIM_SLICE_MAX_GLOBAL || n_global >= n)
        return set_error(QSIM_EINVAL, "n_global=%d outside 0..min(%d, n-1)", n_global, QSIM_SLICE_MAX_GLOBAL);
    const int L = n - n_global;
    if (L > 34) return set_error(QSIM_EINVAL, "slices of %d qubits exceed the 34-qubit state limit", L);
    if (kmax < 1 || kmax > QSIM_MAX_TARGETS) return set_error(QSIM_EINVAL, "kmax=%d outside 1..6", kmax);
    if (mode != QSIM_FUSE_GREEDY2 && mode != QSIM_FUSE_STAGED && mode != QSIM_FUSE_TC &&
        mode != (QSIM_FUSE_STAGED | QSIM_PLAN_SPECIALIZE))
        return set_error(QSIM_EINVAL, "unknown fusion mode %d", mode);
    std::unique_ptr<qsim_slice_plan> P(new qsim_slice_plan());
    P->n = n;
    P->g = n_global;
    P->L = L;
    P->kmax = kmax;
    P->mode = mode;
    // classify every gate in logical qubits; collect the qubits that must be
    // local when it runs (targets of dense and permutation gates)
    const size_t G = c->gates.size();
    std::vector<Op> ops(G);
    std::vector<std::vector<int>> need(G);
    for (size_t i = 0; i < G; ++i) {
        const GateRec &g = c->gates[i];
        QSIM_TRY(classify(g.m, g.targets, g.k, g.controls, g.nc, ops[i]));
        if (ops[i].type == Op::DENSE || ops[i].type == Op::MONO)
            need[i].assign(ops[i].targets, ops[i].targets + ops[i].k);
        if (ops[i].type != Op::IDENTITY && ops[i].type != Op::DIAG && ops[i].k > L)
            return set_error(QSIM_EUNSUPPORTED, "gate %zu has more targets than a slice has qubits", i);
    }
    // Gates are scheduled over their dependency graph (a gate follows the
    // previous gate on each of its qubits; gates on disjoint qubits commute):
    // every ready gate whose must-be-local targets are local runs at once;
    // when all ready gates are blocked, the global qubits they need are
    // exchanged together, each with the local qubit whose next must-be-local
    // use is furthest away (Belady's rule).
    std::vector<std::vector<size_t>> uses(n), succ(G);
    std::vector<int> indeg(G, 0);
    {
        std::vector<long> last(n, -1);
        for (size_t i = 0; i < G; ++i) {
            for (int q : need[i]) uses[q].push_back(i);
            std::vector<int> qs(ops[i].targets, ops[i].targets + ops[i].k);
            qs.insert(qs.end(), ops[i].controls, ops[i].controls + ops[i].c);
            std::vector<long> preds;
            for (int q : qs) {
                if (last[q] >= 0 && std::find(preds.begin(), preds.end(), last[q]) == preds.end())
                    preds.push_back(last[q]);
                last[q] = long(i);
            }
            for (long pr : preds) succ[size_t(pr)].push_back(i);
            indeg[i] = int(preds.size());
        }
    }
    std::vector<char> done(G, 0);
    std::vector<size_t> cursor(n, 0);
    // gates on one qubit run in order, so the done uses of q form a prefix
    auto next_use = [&](int q) -> size_t {
        size_t &k = cursor[q];
        while (k < uses[q].size() && done[uses[q][k]]) ++k;
        return k < uses[q].size() ? uses[q][k] : size_t(-1);
    };
    std::vector<int> pos(n), inv(n);
    for (int q = 0; q < n; ++q) pos[q] = inv[q] = q;
    std::vector<SegGate> seg;
    int seg_gates = 0;
    auto swap_step = [&](int gpos, int lpos) -> int {
        QSIM_TRY(close_segment(*P, seg, seg_gates));
        seg_gates = 0;
        qsim_slice_plan::Step st;
        st.type = QSIM_SLICE_SWAP;
        st.gbit = gpos - L;
        st.lpos = lpos;
        P->steps.push_back(std::move(st));
        const int qa = inv[gpos], qb = inv[lpos];
        inv[gpos] = qb;
        inv[lpos] = qa;
        pos[qa] = lpos;
        pos[qb] = gpos;
        return QSIM_OK;
    };
    std::set<size_t> ready;
    for (size_t i = 0; i < G; ++i)
        if (indeg[i] == 0) ready.insert(i);
    size_t ndone = 0;
    while (ndone < G) {
        bool progress = true;
        while (progress) {
            progress = false;
            for (auto it = ready.begin(); it != ready.end(); ++it) {
                const size_t i = *it;
                bool local = true;
                for (int q : need[i]) local = local && pos[q] < L;
                if (!local) continue;
                if (ops[i].type != Op::IDENTITY) {
                    SegGate sg;
                    sg.op = ops[i];
                    for (int t = 0; t < sg.op.k; ++t) sg.op.targets[t] = pos[ops[i].targets[t]];
                    for (int t = 0; t < sg.op.c; ++t) sg.op.controls[t] = pos[ops[i].controls[t]];
                    seg.push_back(std::move(sg));
                }
                ++seg_gates;
                done[i] = 1;
                ++ndone;
                ready.erase(it);
                for (size_t s2 : succ[i])
                    if (--indeg[s2] == 0) ready.insert(s2);
                progress = true;
                break;  // rescan from the earliest ready gate
            }
        }
        if (ndone == G) break;
        // every ready gate is blocked: exchange the global qubits they need
        std::vector<int> want, keep;
        for (size_t i : ready)
            for (int q : need[i]) {
                if (pos[q] >= L) {
                    if (std::find(want.begin(), want.end(), q) == want.end()) want.push_back(q);
                } else if (std::find(keep.begin(), keep.end(), q) == keep.end()) {
                    keep.push_back(q);
                }
            }
        int swapped = 0;
        for (int q : want) {
            int best = -1;
            size_t best_use = 0;
            for (int p = L - 1; p >= 0; --p) {
                const int qq = inv[p];
                if (std::find(keep.begin(), keep.end(), qq) != keep.end()) continue;
                const size_t u = next_use(qq);
                if (best < 0 || u > best_use) {
                    best = p;
                    best_use = u;
                }
                if (u == size_t(-1)) break;
            }
            if (best < 0) break;
            keep.push_back(q);  // q stays local from now on
            QSIM_TRY(swap_step(pos[q], best));
            ++swapped;
        }
        if (!swapped) return set_error(QSIM_EUNSUPPORTED, "slice planner: no local qubit to exchange");
    }
    if (restore_layout) {
        // global positions first: bring logical qubit p to position p
        for (int gp = L; gp < n; ++gp) {
            if (inv[gp] == gp) continue;
            if (pos[gp] >= L) {  // it sits at another global position: route it through a local one
                QSIM_TRY(swap_step(pos[gp], 0));
            }
            QSIM_TRY(swap_step(gp, pos[gp]));
        }
        // then the local permutation, as SWAP gates on every slice
        for (int p = 0; p < L; ++p) {
            if (inv[p] == p) continue;
            const int r = pos[p];
            SegGate sg;
            sg.op.type = Op::MONO;
            sg.op.k = 2;
            sg.op.targets[0] = p;
            sg.op.targets[1] = r;
            sg.op.perm = {0, 2, 1, 3};
            sg.op.phase = {cd(1.0), cd(1.0), cd(1.0), cd(1.0)};
            seg.push_back(std::move(sg));
            const int qa = inv[p], qb = inv[r];
            inv[p] = qb;
            inv[r] = qa;
            pos[qa] = r;
            pos[qb] = p;
        }
    }
    QSIM_TRY(close_segment(*P, seg, seg_gates));
    P->pos = pos;
    *out = P.release();
    return QSIM_OK;
}

int qsim_slice_plan_destroy(qsim_slice_plan *p) {
    delete p;
    return QSIM_OK;
}

int qsim_slice_plan_info(const qsim_slice_plan *p, int *n_global, int *n_local, int *nsteps, int *nswaps,
                         int *nvariants) {
    if (!p) return set_error(QSIM_EINVAL, "plan is NULL");
    int sw = 0, nv = 0;
    for (const auto &s : p->steps) {
        if (s.type == QSIM_SLICE_SWAP) ++sw;
        nv += int(s.plans.size());
    }
    if (n_global) *n_global = p->g;
    if (n_local) *n_local = p->L;
    if (nsteps) *nsteps = int(p->steps.size());
    if (nswaps) *nswaps = sw;
    if (nvariants) *nvariants = nv;
    return QSIM_OK;
}

int qsim_slice_plan_step(const qsim_slice_plan *p, int i, int *type, int *global_bit, int *local_pos,
                         uint32_t *keymask, int *ngates) {
    if (!p) return set_error(QSIM_EINVAL, "plan is NULL");
    if (i < 0 || i >= int(p->steps.size())) return set_error(QSIM_EINVAL, "step %d outside the plan", i);
    const auto &s = p->steps[size_t(i)];
    if (type) *type = s.type;
    if (global_bit) *global_bit = s.gbit;
    if (local_pos) *local_pos = s.lpos;
    if (keymask) *keymask = s.keymask;
    if (ngates) *ngates = s.ngates;
    return QSIM_OK;
}

int qsim_slice_plan_layout(const qsim_slice_plan *p, int *pos) {
    if (!p || !pos) return set_error(QSIM_EINVAL, "NULL argument");
    for (int q = 0; q < p->n; ++q) pos[q] = p->pos[size_t(q)];
    return QSIM_OK;
}

static int segment_of(const qsim_slice_plan *p, int step, uint32_t slice, const qsim_slice_plan::Step **out) {
    if (!p) return set_error(QSIM_EINVAL, "plan is NULL");
    if (step < 0 || step >= int(p->steps.size())) return set_error(QSIM_EINVAL, "step %d outside the plan", step);
    const auto &s = p->steps[size_t(step)];
    if (s.type != QSIM_SLICE_SEGMENT) return set_error(QSIM_EINVAL, "step %d is not a segment", step);
    if (p->g < 32 && (slice >> p->g) != 0) return set_error(QSIM_EINVAL, "slice %u outside 0..2^%d", slice, p->g);
    *out = &s;
    return QSIM_OK;
}

int qsim_slice_segment_circuit(const qsim_slice_plan *p, int step, uint32_t slice, qsim_circuit **out) {
    if (!out) return set_error(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    const qsim_slice_plan::Step *s = nullptr;
    QSIM_TRY(segment_of(p, step, slice, &s));
    const qsim_circuit *src = s->circuits.at(slice & s->keymask);
    *out = new qsim_circuit(*src);
    return QSIM_OK;
}

int qsim_slice_apply_segment(const qsim_slice_plan *p, int step, uint32_t slice, qsim_state *state) {
    if (!state) return set_error(QSIM_EINVAL, "state is NULL");
    const qsim_slice_plan::Step *s = nullptr;
    QSIM_TRY(segment_of(p, step, slice, &s));
    if (state->n != p->L) return set_error(QSIM_EINVAL, "state has %d qubits, slices %d", state->n, p->L);
    const qsim_plan *pl = s->plans.at(slice & s->keymask);
    return pl ? qsim_apply_fused(state, pl) : QSIM_OK;
}

int qsim_slice_exchange(void *a, void *b, int n_local, int dtype, int local_pos, void *stream) {
    if (!a || !b) return set_error(QSIM_EINVAL, "NULL slice");
    if (a == b) return set_error(QSIM_EINVAL, "a slice cannot exchange with itself");
    if (n_local < 1 || n_local > 34) return set_error(QSIM_EINVAL, "n_local=%d outside 1..34", n_local);
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return set_error(QSIM_EINVAL, "bad dtype %d", dtype);
    if (local_pos < 0 || local_pos >= n_local) return set_error(QSIM_EINVAL, "local_pos=%d outside the slice", local_pos);
    return launch_exchange(a, b, n_local, dtype, local_pos, static_cast<cudaStream_t>(stream));
}

static int pack_common(void *slice, void *buf, int n_local, int dtype, int local_pos, int bit, bool pack,
                       void *stream) {
    if (!slice || !buf) return set_error(QSIM_EINVAL, "NULL buffer");
    if (n_local < 1 || n_local > 34) return set_error(QSIM_EINVAL, "n_local=%d outside 1..34", n_local);
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return set_error(QSIM_EINVAL, "bad dtype %d", dtype);
    if (local_pos < 0 || local_pos >= n_local) return set_error(QSIM_EINVAL, "local_pos=%d outside the slice", local_pos);
    if (bit != 0 && bit != 1) return set_error(QSIM_EINVAL, "bit must be 0 or 1");
    return launch_pack(slice, buf, n_local, dtype, local_pos, bit, pack, static_cast<cudaStream_t>(stream));
}

int qsim_slice_pack(const void *slice, int n_local, int dtype, int local_pos, int bit, void *out, void *stream) {
    return pack_common(const_cast<void *>(slice), out, n_local, dtype, local_pos, bit, true, stream);
}

int qsim_slice_unpack(void *slice, int n_local, int dtype, int local_pos, int bit, const void *in, void *stream) {
    return pack_common(slice, const_cast<void *>(in), n_local, dtype, local_pos, bit, false, stream);
}

}  // extern "C"

// ------------------------------------------------------------------ executors
namespace qsim {
namespace {

struct StateSet {
    std::vector<qsim_state *> s;
    ~StateSet() {
        for (qsim_state *x : s) qsim_state_destroy(x);
    }
};

int run_device(const qsim_slice_plan &P, int dtype, void *const *slices, cudaStream_t st) {
    const uint32_t ns = 1u << P.g;
    StateSet states;
    for (uint32_t i = 0; i < ns; ++i) {
        qsim_state *s = nullptr;
        QSIM_TRY(qsim_state_create(P.L, dtype, slices[i], st, &s));
        states.s.push_back(s);
    }
    for (size_t k = 0; k < P.steps.size(); ++k) {
        const auto &step = P.steps[k];
        if (step.type == QSIM_SLICE_SWAP) {
            for (uint32_t i = 0; i < ns; ++i)
                if (!((i >> step.gbit) & 1u))
                    QSIM_TRY(launch_exchange(slices[i], slices[i | (1u << step.gbit)], P.L, dtype, step.lpos, st));
        } else {
            for (uint32_t i = 0; i < ns; ++i)
                QSIM_TRY(qsim_slice_apply_segment(&P, int(k), i, states.s[i]));
        }
    }
    return QSIM_OK;
}

// One pass of the host executor: a run of SWAP steps (their global bits span
// `gmask`) followed by at most one segment.  Slices are processed in groups
// that share every global bit outside gmask.
struct Pass {
    std::vector<int> swaps;  // step indices
    int segment = -1;        // step index or -1
    uint32_t gmask = 0;
};

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

struct Streams {
    cudaStream_t up = nullptr, comp = nullptr, down = nullptr;
    std::vector<cudaEvent_t> ev;
    cudaEvent_t make() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ev.push_back(e);
        return e;
    }
    ~Streams() {
        for (cudaStream_t x : {up, comp, down})
            if (x) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// Slices stream through 2 x (largest group) staging slots on three streams:
// uploads, compute (exchanges and segments) and downloads.  Events order
// them per slot and per slice, so the upload of one slice overlaps the work
// on another and the download of a third; a slice is uploaded again only
// after its previous download, and a slot is reused only after it has been
// downloaded.
int run_host(const qsim_slice_plan &P, int dtype, void *const *slices, cudaStream_t user) {
    const uint32_t ns = 1u << P.g;
    const size_t S = dtype == QSIM_C64 ? 8 : 16;
    const size_t slice_bytes = (size_t(1) << P.L) * S;
    // a pass stages 2^m slices (m = global bits its exchanges touch) in each
    // of two slot sets, and tensor-core plans add a ping-pong copy of each
    size_t free_b = 0, total_b = 0;
    QSIM_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b), "device memory query");
    const size_t per_slice = slice_bytes * (P.mode == QSIM_FUSE_TC ? 2 : 1) * 2;
    const size_t reserve = size_t(1) << 30;
    int mcap = 0;
    while (mcap < P.g && (per_slice << (mcap + 1)) + reserve <= free_b) ++mcap;
    if (P.g > 0 && mcap < 1)
        return set_error(QSIM_ENOMEM, "host slices: two %zu MiB slices per staging set do not fit (%zu MiB free)",
                         slice_bytes >> 20, free_b >> 20);
    if (P.g == 0 && per_slice + reserve > free_b)
        return set_error(QSIM_ENOMEM, "host slices: staging of %zu MiB does not fit (%zu MiB free)", per_slice >> 20,
                         free_b >> 20);
    std::vector<Pass> passes;
    {
        Pass cur;
        for (size_t k = 0; k < P.steps.size(); ++k) {
            const auto &step = P.steps[k];
            if (step.type == QSIM_SLICE_SWAP) {
                if (__builtin_popcount(cur.gmask | (1u << step.gbit)) > mcap) {
                    passes.push_back(cur);
                    cur = Pass();
                }
                cur.swaps.push_back(int(k));
                cur.gmask |= 1u << step.gbit;
            } else {
                cur.segment = int(k);
                passes.push_back(cur);
                cur = Pass();
            }
        }
        if (!cur.swaps.empty() || cur.segment >= 0) passes.push_back(cur);
    }
    int maxm = 0;
    for (const Pass &ps : passes) maxm = std::max(maxm, __builtin_popcount(ps.gmask));
    const size_t nslots = size_t(2) << maxm;
    DevBuf buf;
    QSIM_CUDA_TRY(dev_alloc(&buf.p, nslots * slice_bytes), "slice staging");
    char *stage = static_cast<char *>(buf.p);
    Streams ss;
    for (cudaStream_t *x : {&ss.up, &ss.comp, &ss.down})
        QSIM_CUDA_TRY(cudaStreamCreateWithFlags(x, cudaStreamNonBlocking), "slice stream");
    std::vector<cudaEvent_t> up_done(nslots), comp_done(nslots), slot_free(nslots), written(ns);
    std::vector<char> slot_used(nslots, 0), slice_written(ns, 0);
    for (size_t k = 0; k < nslots; ++k) {
        up_done[k] = ss.make();
        comp_done[k] = ss.make();
        slot_free[k] = ss.make();
        if (!up_done[k] || !comp_done[k] || !slot_free[k]) return set_error(QSIM_ECUDA, "slice events");
    }
    for (uint32_t i = 0; i < ns; ++i)
        if (!(written[i] = ss.make())) return set_error(QSIM_ECUDA, "slice events");
    // work queued on the caller's stream before this call comes first
    cudaEvent_t start = ss.make();
    if (!start) return set_error(QSIM_ECUDA, "slice events");
    cudaEventRecord(start, user);
    for (cudaStream_t x : {ss.up, ss.comp, ss.down}) cudaStreamWaitEvent(x, start, 0);
    StateSet states;
    for (size_t k = 0; k < nslots; ++k) {
        qsim_state *st = nullptr;
        QSIM_TRY(qsim_state_create(P.L, dtype, stage + k * slice_bytes, ss.comp, &st));
        states.s.push_back(st);
    }
    size_t ring = 0;
    for (const Pass &ps : passes) {
        const int m = __builtin_popcount(ps.gmask);
        std::vector<int> gbits;
        for (int b = 0; b < P.g; ++b)
            if ((ps.gmask >> b) & 1u) gbits.push_back(b);
        const uint32_t gs = 1u << m;
        for (uint32_t lead = 0; lead < ns; ++lead) {
            if (lead & ps.gmask) continue;
            // member j of the group: the gmask bits of the slice index taken from j
            auto member = [&](uint32_t j) {
                uint32_t s = lead;
                for (int t = 0; t < m; ++t)
                    if ((j >> t) & 1u) s |= 1u << gbits[size_t(t)];
                return s;
            };
            std::vector<size_t> slot(gs);
            for (uint32_t j = 0; j < gs; ++j) {
                slot[j] = ring;
                ring = (ring + 1) % nslots;
            }
            for (uint32_t j = 0; j < gs; ++j) {
                const size_t k = slot[j];
                const uint32_t sl = member(j);
                if (slot_used[k]) cudaStreamWaitEvent(ss.up, slot_free[k], 0);
                if (slice_written[sl]) cudaStreamWaitEvent(ss.up, written[sl], 0);
                {
                    LaunchScope ls(K_H2D, ss.up, double(slice_bytes));
                    QSIM_CUDA_TRY(cudaMemcpyAsync(stage + k * slice_bytes, slices[sl], slice_bytes,
                                                  cudaMemcpyHostToDevice, ss.up),
                                  "slice upload");
                }
                cudaEventRecord(up_done[k], ss.up);
            }
            if (!ps.swaps.empty()) {
                for (uint32_t j = 0; j < gs; ++j) cudaStreamWaitEvent(ss.comp, up_done[slot[j]], 0);
                for (int kk : ps.swaps) {
                    const auto &step = P.steps[size_t(kk)];
                    int t = 0;
                    while (gbits[size_t(t)] != step.gbit) ++t;
                    for (uint32_t j = 0; j < gs; ++j)
                        if (!((j >> t) & 1u))
                            QSIM_TRY(launch_exchange(stage + slot[j] * slice_bytes,
                                                     stage + slot[j | (1u << t)] * slice_bytes, P.L, dtype,
                                                     step.lpos, ss.comp));
                }
            }
            for (uint32_t j = 0; j < gs; ++j) {
                const size_t k = slot[j];
                if (ps.swaps.empty()) cudaStreamWaitEvent(ss.comp, up_done[k], 0);
                if (ps.segment >= 0) QSIM_TRY(qsim_slice_apply_segment(&P, ps.segment, member(j), states.s[k]));
                cudaEventRecord(comp_done[k], ss.comp);
                cudaStreamWaitEvent(ss.down, comp_done[k], 0);
                {
                    LaunchScope ls(K_D2H, ss.down, double(slice_bytes));
                    QSIM_CUDA_TRY(cudaMemcpyAsync(slices[member(j)], stage + k * slice_bytes, slice_bytes,
                                                  cudaMemcpyDeviceToHost, ss.down),
                                  "slice download");
                }
                cudaEventRecord(slot_free[k], ss.down);
                cudaEventRecord(written[member(j)], ss.down);
                slot_used[k] = 1;
                slice_written[member(j)] = 1;
            }
        }
    }
    cudaEvent_t fin[3] = {ss.make(), ss.make(), ss.make()};
    cudaStream_t sts[3] = {ss.up, ss.comp, ss.down};
    for (int i = 0; i < 3; ++i) {
        if (!fin[i]) return set_error(QSIM_ECUDA, "slice events");
        cudaEventRecord(fin[i], sts[i]);
        cudaStreamWaitEvent(user, fin[i], 0);
    }
    QSIM_CUDA_TRY(cudaStreamSynchronize(user), "slice sync");
    QSIM_CUDA_TRY(cudaGetLastError(), "slice run");
    return QSIM_OK;
}

}  // namespace
}  // namespace qsim

extern "C" int qsim_slice_run(const qsim_slice_plan *p, int dtype, void *const *slices, int location, void *stream) {
    if (!p || !slices) return set_error(QSIM_EINVAL, "NULL argument");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return set_error(QSIM_EINVAL, "bad dtype %d", dtype);
    const uint32_t ns = 1u << p->g;
    for (uint32_t i = 0; i < ns; ++i) {
        if (!slices[i]) return set_error(QSIM_EINVAL, "slice %u is NULL", i);
        if (reinterpret_cast<uintptr_t>(slices[i]) & 255) return set_error(QSIM_EINVAL, "slice %u is not 256-byte aligned", i);
        for (uint32_t j = 0; j < i; ++j)
            if (slices[j] == slices[i]) return set_error(QSIM_EINVAL, "slices %u and %u share memory", j, i);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (location == QSIM_SLICES_DEVICE) return run_device(*p, dtype, slices, st);
    if (location == QSIM_SLICES_HOST) return run_host(*p, dtype, slices, st);
    return set_error(QSIM_EINVAL, "bad slice location %d", location);
}

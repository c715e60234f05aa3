// C ABI of libqsim: state objects, gate construction and classification,
// plain circuit execution, measurement entry points, error and launch
// accounting.  Kernels live in the other translation units.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "plan.h"

namespace qsim {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

// ------------------------------------------------------------------ allocation
// Injected allocation failures (test support): after `g_alloc_skip` more
// successful device allocations, the next `g_alloc_fail` ones fail as if the
// device were out of memory.
static std::mutex g_alloc_mu;
static int g_alloc_skip = 0, g_alloc_fail = 0;

cudaError_t dev_alloc(void **p, size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        if (g_alloc_fail > 0) {
            if (g_alloc_skip > 0) {
                --g_alloc_skip;
            } else {
                --g_alloc_fail;
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
        }
    }
    return cudaMalloc(p, bytes);
}

int cuda_error(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return set_error(QSIM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(QSIM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ profiling
static const char *k_names[K_NUM_KINDS] = {
    "init",          "sweep_dense1",  "sweep_densek", "sweep_diag",   "sweep_monomial",
    "probabilities", "marginal",      "reduce",       "expect_pauli", "sample_chunk",
    "sample_scan",   "sample_draw",   "stage",        "tc_block",     "batch",
    "adjoint_step",  "hamiltonian_apply", "copy",  "slice_exchange", "slice_pack",
    "copy_h2d",      "copy_d2h",     "pauli_phase"};

const char *kernel_name(int kind) { return (kind >= 0 && kind < K_NUM_KINDS) ? k_names[kind] : "?"; }

int device_sm_count() {
    constexpr int MAX_DEV = 64;
    static std::atomic<int> cache[MAX_DEV];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < MAX_DEV) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 148;
    }
    if (dev >= 0 && dev < MAX_DEV) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

namespace {
struct ProfSlot {
    int kind;
    cudaEvent_t a, b;
    double bytes, flops;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfSlot> g_slots;
size_t g_used = 0;
std::atomic<uint64_t> g_launches{0};
uint64_t g_kind_launches[K_NUM_KINDS];
double g_kind_ms[K_NUM_KINDS];
double g_kind_bytes[K_NUM_KINDS];
double g_kind_flops[K_NUM_KINDS];

int prof_collect() {
    // caller holds g_prof_mu
    for (size_t i = 0; i < g_used; ++i) {
        ProfSlot &s = g_slots[i];
        QSIM_CUDA_TRY(cudaEventSynchronize(s.b), "profile event sync");
        float ms = 0.f;
        QSIM_CUDA_TRY(cudaEventElapsedTime(&ms, s.a, s.b), "profile elapsed");
        g_kind_launches[s.kind] += 1;
        g_kind_ms[s.kind] += ms;
        g_kind_bytes[s.kind] += s.bytes;
        g_kind_flops[s.kind] += s.flops;
    }
    g_used = 0;
    return QSIM_OK;
}
}  // namespace

LaunchScope::LaunchScope(int kind_, cudaStream_t stream_, double bytes, double flops)
    : kind(kind_), stream(stream_), slot(-1) {
    if (kind_ != K_COPY && kind_ != K_H2D && kind_ != K_D2H) g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_used == g_slots.size()) {
        ProfSlot s{};
        if (cudaEventCreate(&s.a) != cudaSuccess || cudaEventCreate(&s.b) != cudaSuccess) return;
        g_slots.push_back(s);
    }
    slot = int(g_used++);
    g_slots[slot].kind = kind;
    g_slots[slot].bytes = bytes;
    g_slots[slot].flops = flops;
    cudaEventRecord(g_slots[slot].a, stream);
}

LaunchScope::~LaunchScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_slots[slot].b, stream);
}

// ------------------------------------------------------------------ qubits
int validate_qubits(int n, const int *targets, int k, const int *controls, int c) {
    if (k < 0 || k > QSIM_MAX_TARGETS) return set_error(QSIM_EINVAL, "k=%d outside 0..%d", k, QSIM_MAX_TARGETS);
    if (c < 0 || c > QSIM_MAX_CONTROLS) return set_error(QSIM_EINVAL, "c=%d outside 0..%d", c, QSIM_MAX_CONTROLS);
    if ((k > 0 && !targets) || (c > 0 && !controls)) return set_error(QSIM_EINVAL, "NULL qubit list");
    uint64_t seen = 0;
    for (int i = 0; i < k + c; ++i) {
        int q = i < k ? targets[i] : controls[i - k];
        if (q < 0 || q >= n) return set_error(QSIM_EINVAL, "qubit %d outside 0..%d", q, n - 1);
        if (seen >> q & 1) return set_error(QSIM_EINVAL, "qubit %d listed twice", q);
        seen |= uint64_t(1) << q;
    }
    return QSIM_OK;
}

IndexMap make_index_map(const int *zero_bits, int nz, const int *one_bits, int no) {
    IndexMap m{};
    int all[MAX_INS];
    int na = 0;
    m.set = 0;
    for (int i = 0; i < nz; ++i) all[na++] = zero_bits[i];
    for (int i = 0; i < no; ++i) {
        all[na++] = one_bits[i];
        m.set |= uint64_t(1) << one_bits[i];
    }
    // insertion sort ascending: inserting in ascending order keeps every
    // later position valid in the expanded index
    for (int i = 1; i < na; ++i)
        for (int j = i; j > 0 && all[j - 1] > all[j]; --j) std::swap(all[j - 1], all[j]);
    m.nins = na;
    for (int i = 0; i < na; ++i) m.ins[i] = all[i];
    return m;
}

// ------------------------------------------------------------------ gates
int gate_matrix(int kind, int k, const double *p, const double *matrix, std::vector<cd> &out) {
    const cd I(0, 1);
    auto need = [&](int kk, int np) -> int {
        if (k != kk) return set_error(QSIM_EINVAL, "gate kind %d takes %d targets, got %d", kind, kk, k);
        if (np > 0 && !p) return set_error(QSIM_EINVAL, "gate kind %d needs %d params", kind, np);
        return QSIM_OK;
    };
    switch (kind) {
        case QSIM_GATE_MATRIX: {
            if (k < 1 || k > QSIM_MAX_TARGETS || !matrix) return set_error(QSIM_EINVAL, "MATRIX gate needs 1..6 targets and a matrix");
            size_t d = size_t(1) << k;
            out.resize(d * d);
            for (size_t i = 0; i < d * d; ++i) out[i] = cd(matrix[2 * i], matrix[2 * i + 1]);
            return QSIM_OK;
        }
        case QSIM_GATE_H: {
            QSIM_TRY(need(1, 0));
            const double r = 1.0 / std::sqrt(2.0);
            out = {r, r, r, -r};
            return QSIM_OK;
        }
        case QSIM_GATE_X: QSIM_TRY(need(1, 0)); out = {0.0, 1.0, 1.0, 0.0}; return QSIM_OK;
        case QSIM_GATE_Y: QSIM_TRY(need(1, 0)); out = {0.0, -I, I, 0.0}; return QSIM_OK;
        case QSIM_GATE_Z: QSIM_TRY(need(1, 0)); out = {1.0, 0.0, 0.0, -1.0}; return QSIM_OK;
        case QSIM_GATE_S: QSIM_TRY(need(1, 0)); out = {1.0, 0.0, 0.0, I}; return QSIM_OK;
        case QSIM_GATE_T:
            QSIM_TRY(need(1, 0));
            out = {1.0, 0.0, 0.0, std::polar(1.0, M_PI / 4)};
            return QSIM_OK;
        case QSIM_GATE_RX: {
            QSIM_TRY(need(1, 1));
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            out = {c, -I * s, -I * s, c};
            return QSIM_OK;
        }
        case QSIM_GATE_RY: {
            QSIM_TRY(need(1, 1));
            double c = std::cos(p[0] / 2), s = std::sin(p[0] / 2);
            out = {c, -s, s, c};
            return QSIM_OK;
        }
        case QSIM_GATE_RZ:
            QSIM_TRY(need(1, 1));
            out = {std::polar(1.0, -p[0] / 2), 0.0, 0.0, std::polar(1.0, p[0] / 2)};
            return QSIM_OK;
        case QSIM_GATE_PHASE:
            QSIM_TRY(need(1, 1));
            out = {1.0, 0.0, 0.0, std::polar(1.0, p[0])};
            return QSIM_OK;
        case QSIM_GATE_RZZ: {  // exp(-i theta Z Z / 2): phase -theta/2 on even parity, +theta/2 on odd
            QSIM_TRY(need(2, 1));
            const cd e = std::polar(1.0, -p[0] / 2), o = std::polar(1.0, p[0] / 2);
            out.assign(16, 0.0);
            out[0] = e;
            out[5] = o;
            out[10] = o;
            out[15] = e;
            return QSIM_OK;
        }
        case QSIM_GATE_CZ:
            QSIM_TRY(need(2, 0));
            out.assign(16, 0.0);
            out[0] = out[5] = out[10] = 1.0;
            out[15] = -1.0;
            return QSIM_OK;
        case QSIM_GATE_SWAP:
            QSIM_TRY(need(2, 0));
            out.assign(16, 0.0);
            out[0] = out[6] = out[9] = out[15] = 1.0;
            return QSIM_OK;
        case QSIM_GATE_SU2: {
            QSIM_TRY(need(1, 4));
            out = {cd(p[0], p[1]), cd(p[2], p[3]), cd(-p[2], p[3]), cd(p[0], -p[1])};
            return QSIM_OK;
        }
        default:
            return set_error(QSIM_EINVAL, "unknown gate kind %d", kind);
    }
}

int classify(const std::vector<cd> &m_in, const int *targets, int k, const int *controls, int c,
             Op &op) {
    std::vector<cd> m = m_in;
    std::vector<int> t(targets, targets + k);
    std::vector<int> ctl(controls, controls + c);
    // A target whose bit is never flipped by G and on whose 0-half G is the
    // identity acts as a control: drop it from the targets (Sec. 2: only the
    // amplitudes a gate changes need to be touched).
    for (bool changed = true; changed && !t.empty();) {
        changed = false;
        const int kk = int(t.size());
        const size_t d = size_t(1) << kk;
        for (int i = 0; i < kk && !changed; ++i) {
            const size_t bit = size_t(1) << (kk - 1 - i);
            bool ok = true;
            for (size_t r = 0; r < d && ok; ++r)
                for (size_t col = 0; col < d && ok; ++col) {
                    const cd v = m[r * d + col];
                    if ((r & bit) != (col & bit)) {
                        if (v != cd(0.0)) ok = false;
                    } else if (!(r & bit)) {
                        if (v != (r == col ? cd(1.0) : cd(0.0))) ok = false;
                    }
                }
            if (!ok) continue;
            const size_t d2 = d / 2;
            std::vector<cd> sub(d2 * d2);
            auto expand = [&](size_t j) {  // index in the sub-block -> index with bit set
                const size_t low = j & (bit - 1);
                return ((j ^ low) << 1) | bit | low;
            };
            for (size_t r = 0; r < d2; ++r)
                for (size_t col = 0; col < d2; ++col) sub[r * d2 + col] = m[expand(r) * d + expand(col)];
            m.swap(sub);
            ctl.push_back(t[i]);
            t.erase(t.begin() + i);
            changed = true;
        }
    }
    op = Op{};
    op.k = int(t.size());
    op.c = int(ctl.size());
    for (int i = 0; i < op.k; ++i) op.targets[i] = t[i];
    for (int i = 0; i < op.c; ++i) op.controls[i] = ctl[i];
    const size_t d = size_t(1) << op.k;
    bool ident = true, diag = true, mono = true;
    for (size_t r = 0; r < d; ++r) {
        int nz = 0;
        for (size_t col = 0; col < d; ++col) {
            const cd v = m[r * d + col];
            if (v != (r == col ? cd(1.0) : cd(0.0))) ident = false;
            if (r != col && v != cd(0.0)) diag = false;
            if (v != cd(0.0)) ++nz;
        }
        if (nz != 1) mono = false;
    }
    if (mono) {  // every column must be hit once as well
        std::vector<int> hits(d, 0);
        for (size_t r = 0; r < d; ++r)
            for (size_t col = 0; col < d; ++col)
                if (m[r * d + col] != cd(0.0)) hits[col]++;
        for (size_t col = 0; col < d; ++col)
            if (hits[col] != 1) mono = false;
    }
    if (ident) {
        op.type = Op::IDENTITY;
    } else if (diag) {
        op.type = Op::DIAG;
        op.m.resize(d);
        for (size_t r = 0; r < d; ++r) op.m[r] = m[r * d + r];
    } else if (mono && op.k <= 3) {
        op.type = Op::MONO;
        op.perm.resize(d);
        op.phase.resize(d);
        for (size_t r = 0; r < d; ++r)
            for (size_t col = 0; col < d; ++col)
                if (m[r * d + col] != cd(0.0)) {
                    op.perm[r] = int(col);
                    op.phase[r] = m[r * d + col];
                }
    } else {
        op.type = Op::DENSE;
        op.m = m;
    }
    return QSIM_OK;
}

}  // namespace qsim

using namespace qsim;

// ------------------------------------------------------------------ state
int qsim_state::ensure_scratch(size_t bytes) {
    if (bytes <= scratch_bytes) return QSIM_OK;
    if (scratch) {
        cudaStreamSynchronize(stream);
        cudaFree(scratch);
        scratch = nullptr;
        scratch_bytes = 0;
    }
    const size_t want = std::max<size_t>(bytes, 1 << 20);
    QSIM_CUDA_TRY(dev_alloc(&scratch, want), "scratch allocation");
    scratch_bytes = want;
    return QSIM_OK;
}

extern "C" {

const char *qsim_last_error(void) { return g_last_error.c_str(); }
const char *qsim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }

int qsim_state_create(int n, int dtype, void *dev_ptr, void *cuda_stream, qsim_state **out) {
    if (!out) return set_error(QSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 34) return set_error(QSIM_EINVAL, "n=%d outside 1..34", n);
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return set_error(QSIM_EINVAL, "bad dtype %d", dtype);
    if (dev_ptr && (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
        return set_error(QSIM_EINVAL, "dev_ptr must be 256-byte aligned");
    qsim_state *s = new qsim_state();
    s->n = n;
    s->dtype = dtype;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&s->device);
    if (dev_ptr) {
        s->amps = dev_ptr;
        s->owned = false;
    } else {
        cudaError_t e = dev_alloc(&s->amps, s->size() * s->amp_bytes());
        if (e != cudaSuccess) {
            delete s;
            return cuda_error(e, "state allocation");
        }
        s->owned = true;
    }
    *out = s;
    return QSIM_OK;
}

int qsim_state_destroy(qsim_state *s) {
    if (!s) return QSIM_OK;
    cudaStreamSynchronize(s->stream);
    if (s->owned && s->amps) cudaFree(s->amps);
    if (s->scratch) cudaFree(s->scratch);
    delete s;
    return QSIM_OK;
}

int qsim_state_set_stream(qsim_state *s, void *cuda_stream) {
    if (!s) return set_error(QSIM_EINVAL, "state is NULL");
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    return QSIM_OK;
}

int qsim_state_info(const qsim_state *s, int *n, int *dtype, void **dev_ptr) {
    if (!s) return set_error(QSIM_EINVAL, "state is NULL");
    if (n) *n = s->n;
    if (dtype) *dtype = s->dtype;
    if (dev_ptr) *dev_ptr = s->amps;
    return QSIM_OK;
}

int qsim_state_init(qsim_state *s, int kind, uint64_t basis, const void *src) {
    if (!s) return set_error(QSIM_EINVAL, "state is NULL");
    const size_t bytes = s->size() * s->amp_bytes();
    switch (kind) {
        case QSIM_INIT_ZERO:
            return launch_init(s->amps, s->n, s->dtype, 0, s->stream);
        case QSIM_INIT_BASIS:
            if (basis >= s->size()) return set_error(QSIM_EINVAL, "basis index outside the state");
            return launch_init(s->amps, s->n, s->dtype, basis, s->stream);
        case QSIM_INIT_NULL:  // no index equals the marker: every amplitude is written 0
            return launch_init(s->amps, s->n, s->dtype, ~uint64_t(0), s->stream);
        case QSIM_INIT_HOST:
        case QSIM_INIT_DEVICE: {
            if (!src) return set_error(QSIM_EINVAL, "src is NULL");
            LaunchScope ls(K_COPY, s->stream, 2.0 * bytes);
            QSIM_CUDA_TRY(cudaMemcpyAsync(s->amps, src, bytes,
                                          kind == QSIM_INIT_HOST ? cudaMemcpyHostToDevice
                                                                 : cudaMemcpyDeviceToDevice,
                                          s->stream),
                          "state init copy");
            return QSIM_OK;
        }
        default:
            return set_error(QSIM_EINVAL, "bad init kind %d", kind);
    }
}

int qsim_state_copy_to_host(qsim_state *s, void *dst) {
    if (!s || !dst) return set_error(QSIM_EINVAL, "NULL argument");
    QSIM_CUDA_TRY(cudaMemcpyAsync(dst, s->amps, s->size() * s->amp_bytes(), cudaMemcpyDeviceToHost,
                                  s->stream),
                  "state copy to host");
    QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "state copy sync");
    return QSIM_OK;
}

int qsim_synchronize(qsim_state *s) {
    if (!s) return set_error(QSIM_EINVAL, "state is NULL");
    QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "synchronize");
#ifdef QSIM_DEBUG
    if (sweep_debug_oob(false) + staged_debug_oob(false))
        return set_error(QSIM_EINVAL, "debug build: a kernel index fell outside its state (access skipped)");
#endif
    return QSIM_OK;
}

long long qsim_debug_checks(int clear) {
#ifdef QSIM_DEBUG
    return (long long)(sweep_debug_oob(clear != 0) + staged_debug_oob(clear != 0));
#else
    (void)clear;
    return -1;
#endif
}

// ------------------------------------------------------------------ gates
static int apply_matrix(qsim_state *s, const std::vector<cd> &m, const int *targets, int k,
                        const int *controls, int c) {
    QSIM_TRY(validate_qubits(s->n, targets, k, controls, c));
    Op op;
    QSIM_TRY(classify(m, targets, k, controls, c, op));
    if (op.type == Op::IDENTITY) return QSIM_OK;
    void *mat_dev = nullptr;
    if (op.type == Op::DENSE && op.k >= 4) {
        // dense matrices of 4+ targets travel through the state's scratch
        // (smaller ones are kernel parameters)
        const size_t d = size_t(1) << op.k;
        const size_t eb = s->amp_bytes();
        QSIM_TRY(s->ensure_scratch(d * d * eb));
        mat_dev = s->scratch;
        std::vector<unsigned char> buf(d * d * eb);
        for (size_t i = 0; i < d * d; ++i) {
            if (s->dtype == QSIM_C64) {
                float v[2] = {float(op.m[i].real()), float(op.m[i].imag())};
                memcpy(&buf[i * eb], v, 8);
            } else {
                double v[2] = {op.m[i].real(), op.m[i].imag()};
                memcpy(&buf[i * eb], v, 16);
            }
        }
        QSIM_CUDA_TRY(cudaMemcpyAsync(mat_dev, buf.data(), buf.size(), cudaMemcpyHostToDevice, s->stream),
                      "gate matrix upload");
    }
    return launch_op(s->amps, s->n, s->dtype, op, s->stream, mat_dev);
}

int qsim_apply_gate(qsim_state *s, const double *matrix, const int *targets, int k,
                    const int *controls, int c) {
    if (!s || !matrix) return set_error(QSIM_EINVAL, "NULL argument");
    if (k < 1) return set_error(QSIM_EINVAL, "k=%d must be >= 1", k);
    std::vector<cd> m;
    QSIM_TRY(gate_matrix(QSIM_GATE_MATRIX, k, nullptr, matrix, m));
    return apply_matrix(s, m, targets, k, controls, c);
}

int qsim_apply_named(qsim_state *s, int kind, const int *targets, int k, const int *controls, int c,
                     const double *params) {
    if (!s) return set_error(QSIM_EINVAL, "state is NULL");
    if (kind == QSIM_GATE_MATRIX) return set_error(QSIM_EINVAL, "use qsim_apply_gate for matrices");
    std::vector<cd> m;
    QSIM_TRY(gate_matrix(kind, k, params, nullptr, m));
    return apply_matrix(s, m, targets, k, controls, c);
}

// ------------------------------------------------------------------ circuits
int qsim_circuit_create(int n, qsim_circuit **out) {
    if (!out) return set_error(QSIM_EINVAL, "out is NULL");
    if (n < 1 || n > QSIM_CIRCUIT_MAX_QUBITS)
        return set_error(QSIM_EINVAL, "n=%d outside 1..%d", n, QSIM_CIRCUIT_MAX_QUBITS);
    *out = new qsim_circuit();
    (*out)->n = n;
    return QSIM_OK;
}

int qsim_circuit_destroy(qsim_circuit *c) {
    delete c;
    return QSIM_OK;
}

int qsim_circuit_add(qsim_circuit *c, int kind, const int *targets, int k, const int *controls,
                     int nc, const double *params, int param_index, const double *matrix) {
    if (!c) return set_error(QSIM_EINVAL, "circuit is NULL");
    QSIM_TRY(validate_qubits(c->n, targets, k, controls, nc));
    GateRec g;
    g.kind = kind;
    g.k = k;
    g.nc = nc;
    for (int i = 0; i < k; ++i) g.targets[i] = targets[i];
    for (int i = 0; i < nc; ++i) g.controls[i] = controls[i];
    const int np = kind == QSIM_GATE_SU2 ? 4
                   : (kind == QSIM_GATE_RX || kind == QSIM_GATE_RY || kind == QSIM_GATE_RZ ||
                      kind == QSIM_GATE_PHASE || kind == QSIM_GATE_RZZ)
                       ? 1
                       : 0;
    for (int i = 0; i < np; ++i) g.params[i] = params ? params[i] : 0.0;
    if (param_index >= 0 && !(kind == QSIM_GATE_RX || kind == QSIM_GATE_RY || kind == QSIM_GATE_RZ))
        return set_error(QSIM_EINVAL, "only RX/RY/RZ angles can be trainable");
    g.pindex = param_index;
    // validates the kind/arity and keeps the matrix (also for named gates)
    QSIM_TRY(gate_matrix(kind, k, g.params, matrix, g.m));
    c->gates.push_back(std::move(g));
    if (param_index >= c->nparams) c->nparams = param_index + 1;
    return QSIM_OK;
}

int qsim_circuit_gate(const qsim_circuit *c, int i, int *kind, int *k, int *targets, int *nc, int *controls,
                      double *matrix) {
    if (!c) return set_error(QSIM_EINVAL, "circuit is NULL");
    if (i < 0 || i >= int(c->gates.size())) return set_error(QSIM_EINVAL, "gate %d outside the circuit", i);
    const GateRec &g = c->gates[size_t(i)];
    if (kind) *kind = g.kind;
    if (k) *k = g.k;
    if (nc) *nc = g.nc;
    if (targets)
        for (int t = 0; t < g.k; ++t) targets[t] = g.targets[t];
    if (controls)
        for (int t = 0; t < g.nc; ++t) controls[t] = g.controls[t];
    if (matrix)
        for (size_t e = 0; e < g.m.size(); ++e) {
            matrix[2 * e] = g.m[e].real();
            matrix[2 * e + 1] = g.m[e].imag();
        }
    return QSIM_OK;
}

int qsim_circuit_info(const qsim_circuit *c, int *n, int *ngates, int *nparams) {
    if (!c) return set_error(QSIM_EINVAL, "circuit is NULL");
    if (n) *n = c->n;
    if (ngates) *ngates = int(c->gates.size());
    if (nparams) *nparams = c->nparams;
    return QSIM_OK;
}

int qsim_run(qsim_state *s, const qsim_circuit *c) {
    if (!s || !c) return set_error(QSIM_EINVAL, "NULL argument");
    if (c->n != s->n) return set_error(QSIM_EINVAL, "circuit has %d qubits, state %d", c->n, s->n);
    for (const GateRec &g : c->gates) QSIM_TRY(apply_matrix(s, g.m, g.targets, g.k, g.controls, g.nc));
    return QSIM_OK;
}

// ------------------------------------------------------------------ measurement
int qsim_probabilities(qsim_state *s, const int *qubits, int m, double *out, int out_on_device) {
    if (!s || !out) return set_error(QSIM_EINVAL, "NULL argument");
    if (m < 0 || m > s->n) return set_error(QSIM_EINVAL, "m=%d outside 0..n", m);
    if (m > 0 && !qubits) return set_error(QSIM_EINVAL, "qubits is NULL");
    uint64_t seen = 0;
    for (int i = 0; i < m; ++i) {
        if (qubits[i] < 0 || qubits[i] >= s->n || (seen >> qubits[i] & 1))
            return set_error(QSIM_EINVAL, "bad or repeated qubit %d", qubits[i]);
        seen |= uint64_t(1) << qubits[i];
    }
    const int mm = m == 0 ? s->n : m;
    const size_t nout = size_t(1) << mm;
    double *dst = out;
    size_t off = 0;
    if (!out_on_device) {
        off = (nout * sizeof(double) + 255) & ~size_t(255);
    }
    const size_t scratch_d = m == 0 ? 0 : marginal_scratch_doubles(s->n, m);
    QSIM_TRY(s->ensure_scratch(off + scratch_d * sizeof(double) + 256));
    if (!out_on_device) dst = static_cast<double *>(s->scratch);
    double *scr = reinterpret_cast<double *>(static_cast<char *>(s->scratch) + off);
    if (m == 0)
        QSIM_TRY(launch_probs(s->amps, s->n, s->dtype, dst, s->stream));
    else
        QSIM_TRY(launch_marginal(s->amps, s->n, s->dtype, qubits, m, dst, scr, scratch_d, s->stream));
    if (!out_on_device) {
        QSIM_CUDA_TRY(cudaMemcpyAsync(out, dst, nout * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                      "probabilities copy");
        QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "probabilities sync");
    }
    return QSIM_OK;
}

int qsim_norm2(qsim_state *s, double *out) {
    if (!s || !out) return set_error(QSIM_EINVAL, "NULL argument");
    const size_t np = reduce_partials_needed(s->n);
    QSIM_TRY(s->ensure_scratch((np + 8) * sizeof(double)));
    double *part = static_cast<double *>(s->scratch);
    double *res = part + np;
    QSIM_TRY(launch_norm2(s->amps, s->n, s->dtype, part, res, s->stream));
    QSIM_CUDA_TRY(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream), "norm copy");
    QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "norm sync");
    return QSIM_OK;
}

int qsim_expectation_pauli(qsim_state *s, int nterms, const uint64_t *xmask, const uint64_t *zmask,
                           const double *coeff, double *out) {
    if (!s || !out) return set_error(QSIM_EINVAL, "NULL argument");
    if (nterms < 0 || (nterms > 0 && (!xmask || !zmask || !coeff)))
        return set_error(QSIM_EINVAL, "bad term arrays");
    const uint64_t full = s->n >= 64 ? ~uint64_t(0) : ((uint64_t(1) << s->n) - 1);
    for (int t = 0; t < nterms; ++t)
        if ((xmask[t] | zmask[t]) & ~full) return set_error(QSIM_EINVAL, "term %d acts outside the state", t);
    const size_t np = reduce_partials_needed(s->n);
    QSIM_TRY(s->ensure_scratch((np + 8) * sizeof(double)));
    double *part = static_cast<double *>(s->scratch);
    double *res = part + np;
    QSIM_TRY(launch_expect(s->amps, s->n, s->dtype, nterms, xmask, zmask, coeff, part, np, res, s->stream));
    QSIM_CUDA_TRY(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream),
                  "expectation copy");
    QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "expectation sync");
    return QSIM_OK;
}

static int sample_common(const void *src, int src_kind, uint64_t N, uint64_t nshots, uint64_t seed,
                         uint64_t counter0, uint64_t *out, int out_on_device, cudaStream_t st,
                         uint64_t *scratch) {
    // scratch layout: [chunk sums / prefix (sample_scratch_u64)] [scan offsets] [psum double] [shots if host]
    const size_t nsc = sample_scratch_u64(N), nof = sample_offsets_u64(N);
    uint64_t *offs = scratch + nsc;
    double *psum = reinterpret_cast<double *>(scratch + nsc + nof);
    uint64_t *dst = out_on_device ? out : scratch + nsc + nof + 8;
    QSIM_TRY(launch_sample(src, src_kind, N, nshots, seed, counter0, dst, scratch, offs, psum, st));
    double hp = 0.0;
    uint64_t total = 0;
    QSIM_CUDA_TRY(cudaMemcpyAsync(&hp, psum, sizeof(double), cudaMemcpyDeviceToHost, st), "psum copy");
    QSIM_CUDA_TRY(cudaMemcpyAsync(&total, scratch + nsc - 1, sizeof(uint64_t), cudaMemcpyDeviceToHost, st),
                  "total copy");
    if (!out_on_device && nshots)
        QSIM_CUDA_TRY(cudaMemcpyAsync(out, dst, nshots * sizeof(uint64_t), cudaMemcpyDeviceToHost, st),
                      "shots copy");
    QSIM_CUDA_TRY(cudaStreamSynchronize(st), "sample sync");
    if (!(hp <= 1.5) || total == 0)
        return set_error(QSIM_EINVAL, "probabilities must sum to a value in (0, 1.5] (got %g)", hp);
    return QSIM_OK;
}

int qsim_sample(qsim_state *s, uint64_t nshots, uint64_t seed, uint64_t counter0, uint64_t *out,
                int out_on_device) {
    if (!s || (!out && nshots)) return set_error(QSIM_EINVAL, "NULL argument");
    const size_t nsc = sample_scratch_u64(s->size()) + sample_offsets_u64(s->size());
    QSIM_TRY(s->ensure_scratch((nsc + 8 + (out_on_device ? 0 : nshots)) * sizeof(uint64_t)));
    return sample_common(s->amps, s->dtype == QSIM_C64 ? SRC_C64 : SRC_C128, s->size(), nshots, seed,
                         counter0, out, out_on_device, s->stream, static_cast<uint64_t *>(s->scratch));
}

int qsim_sample_probs(const double *p_dev, uint64_t N, uint64_t nshots, uint64_t seed, uint64_t counter0,
                      uint64_t *out, int out_on_device, void *cuda_stream) {
    if (!p_dev || N == 0 || (!out && nshots)) return set_error(QSIM_EINVAL, "bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t nsc = sample_scratch_u64(N) + sample_offsets_u64(N);
    uint64_t *scratch = nullptr;
    QSIM_CUDA_TRY(dev_alloc(&scratch, (nsc + 8 + (out_on_device ? 0 : nshots)) * sizeof(uint64_t)),
                  "sampler scratch");
    int rc = sample_common(p_dev, SRC_PROBS, N, nshots, seed, counter0, out, out_on_device, st, scratch);
    cudaStreamSynchronize(st);
    cudaFree(scratch);
    return rc;
}

// ------------------------------------------------------------------ profiling
int qsim_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return QSIM_OK;
}

int qsim_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    QSIM_TRY(prof_collect());
    for (int i = 0; i < K_NUM_KINDS; ++i) {
        g_kind_launches[i] = 0;
        g_kind_ms[i] = 0;
        g_kind_bytes[i] = 0;
        g_kind_flops[i] = 0;
    }
    return QSIM_OK;
}

int qsim_profile_count(int *nkinds) {
    if (!nkinds) return set_error(QSIM_EINVAL, "NULL argument");
    *nkinds = K_NUM_KINDS;
    return QSIM_OK;
}

int qsim_profile_get(int i, const char **name, uint64_t *launches, double *total_ms, double *total_bytes,
                     double *total_flops) {
    if (i < 0 || i >= K_NUM_KINDS) return set_error(QSIM_EINVAL, "kind index %d", i);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    QSIM_TRY(prof_collect());
    if (name) *name = k_names[i];
    if (launches) *launches = g_kind_launches[i];
    if (total_ms) *total_ms = g_kind_ms[i];
    if (total_bytes) *total_bytes = g_kind_bytes[i];
    if (total_flops) *total_flops = g_kind_flops[i];
    return QSIM_OK;
}

uint64_t qsim_launch_count(void) { return g_launches.load(); }

}  // extern "C"

extern "C" QSIM_API int qsim_debug_fail_alloc(int skip, int count) {
    if (skip < 0 || count < 0) return qsim::set_error(QSIM_EINVAL, "skip and count must be >= 0");
    std::lock_guard<std::mutex> lk(qsim::g_alloc_mu);
    qsim::g_alloc_skip = skip;
    qsim::g_alloc_fail = count;
    return QSIM_OK;
}

// Internal declarations shared by the translation units of libqsim.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qsim {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
#define QSIM_CUDA_TRY(call, what)                                   \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::qsim::cuda_error(e_, what);  \
    } while (0)
// QSIM_DEBUG builds check, before every global access of the plain sweeps and
// the staged tiles, that the index lies inside the state; an index outside is
// counted (per translation unit) and the access skipped.  These return the
// count since load (and clear it when asked); release builds have no checks.
unsigned long long sweep_debug_oob(bool clear);
unsigned long long staged_debug_oob(bool clear);

// Every device allocation of the library goes through here, so that a test can
// make chosen allocations fail (qsim_debug_fail_alloc) without a GPU fault.
cudaError_t dev_alloc(void **p, size_t bytes);
template <typename T> inline cudaError_t dev_alloc(T **p, size_t bytes) {
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}
#define QSIM_TRY(call)                 \
    do {                               \
        int rc_ = (call);              \
        if (rc_ != QSIM_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------------ profiling
// Kernel families; names are what profiling reports.
enum KernelKind {
    K_INIT = 0,
    K_DENSE1,
    K_DENSEK,
    K_DIAG,
    K_MONO,
    K_PROBS,
    K_MARGINAL,
    K_REDUCE,
    K_EXPECT,
    K_SAMPLE_CHUNK,
    K_SAMPLE_SCAN,
    K_SAMPLE_DRAW,
    K_STAGE,
    K_TC_BLOCK,
    K_BATCH,
    K_ADJ_STEP,
    K_HAPPLY,
    K_COPY,          // device-to-device copy (not a kernel)
    K_SLICE_EXCHANGE,
    K_SLICE_PACK,
    K_H2D,           // host-to-device copy (not a kernel)
    K_D2H,           // device-to-host copy (not a kernel)
    K_PAULI_PHASE,
    K_NUM_KINDS
};
const char *kernel_name(int kind);

// SM count of the current device, queried once per device (thread-safe).
int device_sm_count();

// RAII bracket around one launch: counts it (copies are not counted as
// kernel launches) and, when profiling is on, records CUDA events on `stream`
// before and after.
struct LaunchScope {
    // bytes: algorithmic HBM bytes of the launch; flops: useful arithmetic
    LaunchScope(int kind, cudaStream_t stream, double bytes, double flops = 0.0);
    ~LaunchScope();
    int kind;
    cudaStream_t stream;
    int slot;
};

// ------------------------------------------------------------------ index maps
// Expansion of a compact group index g into an amplitude index: a zero bit is
// inserted at every listed position (ascending), then `set` is ORed in.
constexpr int MAX_INS = QSIM_MAX_TARGETS + QSIM_MAX_CONTROLS;
struct IndexMap {
    int nins;
    int ins[MAX_INS];
    uint64_t set;
    uint64_t limit;  // 2^n of the state it indexes (0: unknown); checked in QSIM_DEBUG builds
};
IndexMap make_index_map(const int *zero_bits, int nz, const int *one_bits, int no);
// Offsets of the 2^k amplitudes of a group (matrix index j, targets[0] = MSB).
struct Offsets {
    uint64_t o[1 << QSIM_MAX_TARGETS];
};

// ------------------------------------------------------------------ gate ops
// One launchable sweep after classification of a gate.
struct Op {
    enum Type { IDENTITY, DENSE, DIAG, MONO } type = IDENTITY;
    int k = 0;                       // targets (matrix MSB first)
    int targets[QSIM_MAX_TARGETS] = {};
    int c = 0;                       // controls (all must be 1)
    int controls[QSIM_MAX_CONTROLS + QSIM_MAX_TARGETS] = {};
    std::vector<cd> m;               // DENSE: 2^k x 2^k; DIAG: 2^k entries
    std::vector<int> perm;           // MONO: row r takes column perm[r]
    std::vector<cd> phase;           // MONO: coefficient of row r
};

// Build a named gate's matrix (the library's own definitions).
int gate_matrix(int kind, int k, const double *params, const double *matrix, std::vector<cd> &out);
// Classify (dense / diagonal / monomial) and turn block-identity targets into controls.
int classify(const std::vector<cd> &m, const int *targets, int k, const int *controls, int c,
             Op &op);
int validate_qubits(int n, const int *targets, int k, const int *controls, int c);

// ------------------------------------------------------------------ launchers
// All launchers are asynchronous on `st` and return QSIM_OK or an error code.
int launch_op(void *psi, int n, int dtype, const Op &op, cudaStream_t st, void *mat_dev);
int launch_init(void *psi, int n, int dtype, uint64_t basis, cudaStream_t st);
int launch_probs(const void *psi, int n, int dtype, double *out, cudaStream_t st);
int launch_marginal(const void *psi, int n, int dtype, const int *qubits, int m, double *out,
                    double *scratch, size_t scratch_doubles, cudaStream_t st);
size_t marginal_scratch_doubles(int n, int m);
int launch_norm2(const void *psi, int n, int dtype, double *partials, double *result,
                 cudaStream_t st);
size_t reduce_partials_needed(int n);
// a complex64, b complex128 (a result against its FP64 reference); otherwise as below
int launch_diff_norm2_c64_c128(const void *a, const void *b, int n, double *partials, double *result,
                               cudaStream_t st);
// result[0] = sum |a - b|^2, result[1] = max |a - b|^2 (partials: 2 x reduce_partials_needed)
int launch_diff_norm2(const void *a, const void *b, int n, int dtype, double *partials, double *result,
                      cudaStream_t st);
int launch_expect(const void *psi, int n, int dtype, int nterms, const uint64_t *xmask,
                  const uint64_t *zmask, const double *coeff, double *partials,
                  size_t npartials, double *result, cudaStream_t st);
size_t sample_scratch_u64(uint64_t N);
// scratch: sample_scratch_u64(N) words (chunk prefix + total); offs:
// sample_offsets_u64(N) words for the scan
int launch_sample(const void *src, int src_kind, uint64_t N, uint64_t nshots, uint64_t seed,
                  uint64_t counter0, uint64_t *out_dev, uint64_t *scratch, uint64_t *offs, double *psum_dev,
                  cudaStream_t st);
size_t sample_offsets_u64(uint64_t N);
enum { SRC_C64 = 0, SRC_C128 = 1, SRC_PROBS = 2 };

}  // namespace qsim

// ------------------------------------------------------------------ state
struct qsim_state {
    int n = 0;
    int dtype = QSIM_C64;
    void *amps = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    // grow-only scratch owned by the state (reductions, sampler, matrices)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int ensure_scratch(size_t bytes);
    size_t amp_bytes() const { return dtype == QSIM_C64 ? 8 : 16; }
    uint64_t size() const { return uint64_t(1) << n; }
};

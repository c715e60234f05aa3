/*
 * qsim.h -- C ABI of libqsim, a GB300 (sm_103a) state-vector simulator.
 *
 * The library applies quantum gates to a 2^n-amplitude state vector by the
 * contraction of Eq. (1) of arXiv 2203.08826 (Sec. 1):
 *
 *     psi'(s_1..tau..s_n) = sum_{tau'} G(tau, tau') psi(s_1..tau'..s_n)
 *
 * in place (Sec. 2: custom operators update the state without a copy), and
 * measures the result (probabilities, shots, Pauli expectation values).
 *
 * Conventions used by every entry point
 *   - Amplitudes are interleaved (re, im).  QSIM_C64 stores two floats per
 *     amplitude (8 bytes), QSIM_C128 two doubles (16 bytes).  Amplitude x is at
 *     element x; qubit q is bit q of x (qubit 0 = least significant bit), as in
 *     the single-qubit kernel of Sec. 2 which pairs x with x + 2^target.
 *   - A k-qubit gate matrix is row-major complex128 (2^k * 2^k pairs of
 *     doubles, re then im), and targets[0] is the MOST significant bit of its
 *     row/column index: G(tau_1..tau_k, tau_1'..tau_k') of Eq. (1) takes tau_1
 *     from targets[0].
 *   - Controls (the controlled-gate operators of Sec. 2) act when all control
 *     bits are 1.
 *   - Host arrays passed in are read during the call and may be reused when it
 *     returns.  Device work runs asynchronously on the state's CUDA stream;
 *     calls that return host values synchronise that stream.
 *   - QSIM_C128 arithmetic: dense 1-qubit and diagonal sweeps compute each
 *     amplitude either in FP64 or in double-float arithmetic (a double held as
 *     the sum of two floats, about 48 significant bits, on the FP32 pipes, with
 *     FP64 for values outside [2^-74, 2^77) and subnormals read as 0); other
 *     complex128 kernels use FP64.  The per-gate error stays near 1e-14
 *     relative.
 *   - One process drives one device (the multi-GPU paths run one rank per
 *     GPU): the kernels' shared-memory limits are raised once per process,
 *     on the device current at the first launch.
 *
 * Errors: every int-returning call returns QSIM_OK (0) or a negative code;
 * qsim_last_error() returns a thread-local message for the last failure.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(QSIM_BUILD) && defined(__GNUC__)
#define QSIM_API __attribute__((visibility("default")))
#else
#define QSIM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define QSIM_OK 0
#define QSIM_EINVAL (-1)       /* bad argument: qubit >= n, duplicate qubit, k too large, NULL */
#define QSIM_ENOMEM (-2)       /* a device or host allocation failed */
#define QSIM_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define QSIM_ETIMEOUT (-4)     /* a bounded device-side wait expired */
#define QSIM_EUNSUPPORTED (-5) /* valid request that this build cannot run */

#define QSIM_C64 0
#define QSIM_C128 1

#define QSIM_MAX_TARGETS 6     /* largest dense gate / fused block */
#define QSIM_MAX_CONTROLS 16

/* ---------------------------------------------------------------- gates */
/* Named gates; the library builds their matrices itself.
 *   H X Y Z S T        fixed single-qubit gates
 *   RX RY RZ (theta)   exp(-i theta P / 2), P the Pauli matrix
 *   PHASE (phi)        diag(1, e^{i phi})   (with a control: the QFT's R_k)
 *   CZ                 diag(1, 1, 1, -1) on two targets
 *   SWAP               exchange of two targets
 *   SU2 (a, b, c, d)   [[a + ib, c + id], [-c + id, a - ib]] (unit quaternion)
 *   RZZ (theta)        exp(-i theta Z Z / 2) on two targets: the two-qubit
 *                      factor of a Trotter step of the TFIM (Sec. 3.3)
 *   MATRIX             explicit matrix given by the caller                     */
enum {
    QSIM_GATE_MATRIX = 0,
    QSIM_GATE_H = 1,
    QSIM_GATE_X = 2,
    QSIM_GATE_Y = 3,
    QSIM_GATE_Z = 4,
    QSIM_GATE_S = 5,
    QSIM_GATE_T = 6,
    QSIM_GATE_RX = 7,
    QSIM_GATE_RY = 8,
    QSIM_GATE_RZ = 9,
    QSIM_GATE_PHASE = 10,
    QSIM_GATE_CZ = 11,
    QSIM_GATE_SWAP = 12,
    QSIM_GATE_SU2 = 13,
    QSIM_GATE_RZZ = 14
};

QSIM_API const char *qsim_last_error(void);
QSIM_API const char *qsim_version(void);

/* ---------------------------------------------------------------- state */
typedef struct qsim_state qsim_state;

/* Create a state of n qubits (1 <= n <= 34) in precision dtype (QSIM_C64 or
 * QSIM_C128) whose work runs on `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  If dev_ptr is non-NULL it must point to 2^n amplitudes of
 * device memory, 256-byte aligned, that the caller owns and keeps alive until
 * qsim_state_destroy (the library borrows it); otherwise the library
 * allocates the amplitudes and destroy frees them.  The contents are
 * undefined until qsim_state_init.  Citation: the state vector of 2^n
 * amplitudes, Sec. 1; in-place updates, Sec. 2. */
QSIM_API int qsim_state_create(int n, int dtype, void *dev_ptr, void *cuda_stream, qsim_state **out);
QSIM_API int qsim_state_destroy(qsim_state *s);
QSIM_API int qsim_state_set_stream(qsim_state *s, void *cuda_stream);
/* n, dtype and the device pointer of the amplitudes (any may be NULL). */
QSIM_API int qsim_state_info(const qsim_state *s, int *n, int *dtype, void **dev_ptr);

#define QSIM_INIT_ZERO 0   /* |0...0>                                      */
#define QSIM_INIT_BASIS 1  /* |basis>                                      */
#define QSIM_INIT_HOST 2   /* copy 2^n amplitudes (state precision) from host `src` */
#define QSIM_INIT_DEVICE 3 /* copy 2^n amplitudes (state precision) from device `src` */
#define QSIM_INIT_NULL 4   /* every amplitude 0 (a slice of a larger state that
                              holds none of its weight, Sec. 3.1 slices)   */
QSIM_API int qsim_state_init(qsim_state *s, int kind, uint64_t basis, const void *src);
/* Copy all 2^n amplitudes (state precision) to host memory `dst`; synchronous. */
QSIM_API int qsim_state_copy_to_host(qsim_state *s, void *dst);
/* Block until all work queued on the state's stream has finished; returns
 * QSIM_ECUDA if a kernel failed and QSIM_ETIMEOUT if a bounded wait expired. */
QSIM_API int qsim_synchronize(qsim_state *s);

/* ---------------------------------------------------------------- Eq. (1) */
/* Apply one gate in place.  matrix: 2^k x 2^k row-major complex128 host array
 * (targets[0] = most significant matrix bit); targets: k distinct qubits,
 * 1 <= k <= QSIM_MAX_TARGETS; controls: c distinct qubits not among the
 * targets (may be NULL when c == 0).  The library classifies the matrix
 * (Sec. 2: dense, diagonal, permutation-with-phases; a block that leaves a
 * target untouched when it is 0 becomes a control) and launches one sweep.
 * Citation: Eq. (1), Sec. 1; single-qubit kernel listing and the
 * multi-target / controlled / Pauli / SWAP operators, Sec. 2. */
QSIM_API int qsim_apply_gate(qsim_state *s, const double *matrix, const int *targets, int k,
                    const int *controls, int c);
/* Apply a named gate (QSIM_GATE_*; params as listed above, may be NULL). */
QSIM_API int qsim_apply_named(qsim_state *s, int kind, const int *targets, int k, const int *controls,
                     int c, const double *params);

/* ---------------------------------------------------------------- circuits */
typedef struct qsim_circuit qsim_circuit;

/* Circuits may name up to QSIM_CIRCUIT_MAX_QUBITS qubits; states, plans and
 * the adjoint method take at most 34, wider circuits run on sliced states. */
#define QSIM_CIRCUIT_MAX_QUBITS 48
QSIM_API int qsim_circuit_create(int n, qsim_circuit **out);
QSIM_API int qsim_circuit_destroy(qsim_circuit *c);
/* Append a gate.  params: up to 4 doubles (angle, or the SU2 quaternion);
 * param_index >= 0 marks an RX/RY/RZ angle as trainable parameter number
 * param_index (used by qsim_adjoint_grad, which substitutes its own values);
 * matrix: for QSIM_GATE_MATRIX only, 2^k x 2^k row-major complex128. */
QSIM_API int qsim_circuit_add(qsim_circuit *c, int kind, const int *targets, int k, const int *controls,
                     int nc, const double *params, int param_index, const double *matrix);
QSIM_API int qsim_circuit_info(const qsim_circuit *c, int *n, int *ngates, int *nparams);
/* Gate i as stored: kind, k targets, nc controls and its 2^k x 2^k matrix
 * (row-major, interleaved re/im: 2 * 4^k doubles).  Any output may be NULL;
 * targets/controls need room for k / nc entries. */
QSIM_API int qsim_circuit_gate(const qsim_circuit *c, int i, int *kind, int *k, int *targets, int *nc,
                               int *controls, double *matrix);
/* Plain execution: one sweep per gate, in order (the unfused baseline). */
QSIM_API int qsim_run(qsim_state *s, const qsim_circuit *c);

/* ---------------------------------------------------------------- fusion */
typedef struct qsim_plan qsim_plan;

/* Fusion modes.
 *   QSIM_FUSE_GREEDY2  the paper's fusion (Sec. 3.2): one pass over the gates
 *                      multiplies each 1- or 2-qubit gate into the fused
 *                      gate on its qubits while their union stays within
 *                      kmax qubits; one sweep per fused gate (kmax = 1 merges
 *                      only 1-qubit gates on the same qubit).
 *   QSIM_FUSE_STAGED   cache-blocked stages: each stage loads tiles of 2^m
 *                      amplitudes spanning a chosen qubit set into registers
 *                      (qubits 0..4 across the lanes of a warp, 4 qubits per
 *                      thread, min(kmax, 4) qubits across warps, with shared
 *                      memory to re-assign them), applies every gate of the
 *                      stage there (gates on qubits outside the set only if
 *                      diagonal, or through their controls), and writes the
 *                      tile back: one HBM pass per stage.  Needs n >= 9;
 *                      smaller circuits get a QSIM_FUSE_GREEDY2 plan.
 *   QSIM_FUSE_TC       dense blocks on windows of 6 consecutive qubits
 *                      (kmax >= 6, BF16x3 split) or 5 (kmax <= 5, 3xTF32
 *                      split) applied on the tensor cores as real GEMMs
 *                      (complex64 states only; n >= window + 7), with the
 *                      qubit order rotated by each pass so every block's
 *                      targets are the low bits; diagonal gates that straddle
 *                      a window are applied in the pass's epilogue.
 * kmax (1..6): for QSIM_FUSE_GREEDY2 the most qubits a fused gate may act on;
 * for QSIM_FUSE_STAGED the tile's warp qubits (at most 4); for QSIM_FUSE_TC
 * the window width as above.  The plan copies what it needs from the circuit;
 * it does not depend on the circuit afterwards.
 * QSIM_PLAN_SPECIALIZE may be ORed into QSIM_FUSE_STAGED: the same stages,
 * but each tile stage runs as a kernel written out for its own op list (every
 * position, mask and coefficient offset a constant) and compiled with NVRTC
 * for sm_103a when the plan first runs on a dtype; the coefficients are
 * kernel parameters, so circuits of the same structure with other angles
 * reuse the compiled code (an in-process cache keyed by the stages'
 * structure).  Complex64 register ops run in paired FP32 (fma.rn.f32x2 on
 * (re, im) pairs), with the scalar kernels' products in the same order.  The
 * first run pays the compile (about a second per few stages, in parallel
 * threads); QSIM_ECUDA with the compiler's log if it fails.  qsim_plan_info
 * reports the flag in *mode.
 * Citation: Sec. 3.2 (gate fusion; fusing up to about five qubits may help);
 * the paper compiles its own kernels at run time as well (Sec. 2). */
#define QSIM_FUSE_GREEDY2 0
#define QSIM_FUSE_STAGED 1
#define QSIM_FUSE_TC 2
#define QSIM_PLAN_SPECIALIZE 0x100
QSIM_API int qsim_plan_build(const qsim_circuit *c, int kmax, int mode, qsim_plan **out);
/* Arithmetic of a staged plan per amplitude of the state: the flops its
 * stages execute (a complex multiply-add is 8 flops; a fused 4x4 on a pair
 * costs 32, a 1-qubit gate 16) and those of the circuit's gates applied one
 * sweep each (what the plan replaces).  Host-only; QSIM_EINVAL for other
 * plans.  The library profiler counts the executed flops. */
QSIM_API int qsim_plan_flops(const qsim_plan *p, double *executed, double *circuit);
/* Specialised stage kernels compiled since the library was loaded: seconds
 * spent in the compiler, programs compiled, programs found in the cache. */
QSIM_API int qsim_spec_stats(double *compile_s, uint64_t *compiles, uint64_t *cache_hits);
/* CUDA source of the specialised kernels of a staged plan's tile stages
 * (one kernel per stage, `qsim_spec_stage_<i>`) for dtype, NUL-terminated
 * and truncated to len bytes; *needed (may be NULL) receives the full length
 * + 1, and buf may be NULL with len 0 to ask for it.  Host-only (works on any
 * staged plan, specialised or not); QSIM_EINVAL for a plan that is not
 * staged or a dtype other than QSIM_C64 / QSIM_C128. */
QSIM_API int qsim_plan_source(const qsim_plan *p, int dtype, char *buf, size_t len, size_t *needed);
QSIM_API int qsim_plan_destroy(qsim_plan *p);
/* Number of sweeps (HBM passes) and of source gates the plan covers. */
QSIM_API int qsim_plan_info(const qsim_plan *p, int *nsweeps, int *ngates, int *mode);
/* Fused matrix of block i of a QSIM_FUSE_GREEDY2 plan (0 <= i < nsweeps):
 * writes k and the targets (targets[0] = MSB) and, if matrix_out is non-NULL,
 * the 2^k x 2^k row-major complex128 matrix.  Staged and tensor-core plans
 * keep their work in other forms (stage op lists; window blocks with
 * diagonal epilogues) and return QSIM_EINVAL here.  Host-only; no GPU
 * needed. */
QSIM_API int qsim_plan_block(const qsim_plan *p, int i, int *k, int *targets, double *matrix_out);
/* Human-readable summary of a plan (stages, tile qubits, op counts),
 * NUL-terminated and truncated to len bytes.  Host-only. */
QSIM_API int qsim_plan_describe(const qsim_plan *p, char *buf, size_t len);
/* Pass i of a QSIM_FUSE_TC plan (0 <= i < nsweeps) as the gates it applies,
 * on the circuit's own qubits (host-only; for checking the planner against
 * the gate-by-gate product of Eq. (1)).  *plain = 1: a gate no window holds,
 * applied by a plain sweep: its k targets (targets[0] = MSB), nc controls and
 * 2^k x 2^k row-major complex128 matrix (controls needs room for
 * QSIM_MAX_CONTROLS + QSIM_MAX_TARGETS entries).  *plain = 0: the fused block
 * on the window's k qubits (targets[0] = MSB), nc = 0, followed by *nepi
 * diagonal gates (qsim_plan_tc_epilogue) that the pass applies after it.
 * Outputs may be NULL; QSIM_EINVAL for other plans or i out of range. */
QSIM_API int qsim_plan_tc_pass(const qsim_plan *p, int i, int *plain, int *k, int *targets, int *nc, int *controls,
                               double *matrix, int *nepi);
/* Epilogue gate e of pass i: k targets (targets[0] = MSB), nc controls and
 * its 2^k diagonal entries (complex128, interleaved).  Host-only. */
QSIM_API int qsim_plan_tc_epilogue(const qsim_plan *p, int i, int e, int *k, int *targets, int *nc, int *controls,
                                   double *diag);
/* Arithmetic of each pass of a QSIM_FUSE_TC plan (mixed-precision refinement
 * of the fused blocks): BF16x3 or 3xTF32 split products on the tensor cores,
 * or the same contraction in FP32 on the CUDA cores (slower, no split error).
 * A plan starts with every pass at its window width's split (BF16x3 for
 * kmax >= 6, 3xTF32 for kmax 5); 3xTF32 needs a 5-qubit window.  set takes
 * one value per pass (npasses = the plan's sweeps; plain passes ignore
 * theirs) and QSIM_EINVAL for a bad value; host-only, the next run rebuilds
 * the device images.  Citation: Sec. 3.2 (fusion into blocks of a few qubits);
 * the precision choice itself has no counterpart in the paper. */
#define QSIM_PREC_BF16X3 0
#define QSIM_PREC_TF32X3 1
#define QSIM_PREC_FP32 2
QSIM_API int qsim_plan_tc_precision(const qsim_plan *p, int i, int *prec);
QSIM_API int qsim_plan_tc_set_precision(qsim_plan *p, int npasses, const int *prec);
/* Stage i of a QSIM_FUSE_STAGED plan (0 <= i < nsweeps; host-only, for
 * checking the planner): *plain = 1 for a gate applied by a plain sweep;
 * otherwise the tile's qubits beyond the lanes (nslots of them, in slot
 * order; the lanes hold qubits 0..4).  gates receives the indices of the
 * circuit's gates the stage applies (ngates of them, room for the circuit's
 * gate count), in schedule order: the planner's order before the stage's op
 * list is lowered, where commuting gates may still be merged (a 1-qubit
 * diagonal into a neighbouring 1-qubit gate) or batched (runs of 1-qubit
 * gates on distinct qubits).  QSIM_EINVAL for other plans (a staged request
 * on fewer than 9 qubits builds a greedy plan). */
QSIM_API int qsim_plan_stage(const qsim_plan *p, int i, int *plain, int *ngates, int *gates, int *nslots, int *slots);
/* Stage i of a QSIM_FUSE_STAGED plan as text: the op list its kernels run
 * (positions, masks, coefficient offsets), the phases (register, warp and
 * shared-memory assignments of the tile qubits) and the coefficient pool in
 * full precision; one item per line, the format documented at the
 * definition.  NUL-terminated and truncated to len bytes; *needed receives
 * the full length + 1.  Host-only (for checking the op lists against the
 * gate-by-gate result without a GPU); QSIM_EINVAL for other plans or i out
 * of range. */
QSIM_API int qsim_plan_stage_dump(const qsim_plan *p, int i, char *buf, size_t len, size_t *needed);
/* Autotuner: builds the candidate plans (staged tiles of 2^12 and 2^13
 * amplitudes; for complex64 also tensor-core blocks of 5 and 6 qubits, for
 * complex128 one sweep per gate (greedy fusion with kmax = 1)), runs each on
 * the scratch state `s` (its contents are overwritten) once to warm up and
 * `reps` times under CUDA events on the state's stream, and returns the
 * fastest plan in *out (the caller destroys it) with its mode, kmax and time
 * per run.  Synchronous. */
QSIM_API int qsim_plan_autotune(const qsim_circuit *c, qsim_state *s, int reps, qsim_plan **out, int *mode_out,
                                int *kmax_out, double *ms_out);
/* Autotuner with a measured error/speed table (mixed-precision refinement of
 * the fused blocks).  Candidates for complex64: FP32 register stages (kmax 3
 * and 4), tensor-core plans with every pass in BF16x3 (6-qubit windows),
 * 3xTF32 (5-qubit windows) or FP32 on the CUDA cores (6-qubit windows), and a
 * mixed plan chosen per block: when the BF16x3 plan misses max_err and the
 * FP32 one meets it, the per-pass errors measured for the two (plan error /
 * passes) give the fewest passes that must run in FP32 for the predicted
 * error (summed over passes) to stay within max_err; that plan runs as one
 * more candidate.  complex128: stages against one sweep per gate.  Every
 * candidate runs from |0...0> once; its error is err = ||psi - psi_ref||_2
 * (relative to ||psi|| = 1) and max_abs = max_x |psi(x) - psi_ref(x)|, where
 * psi_ref is the circuit run gate by gate in complex128 (FP64 truth; ref = 1
 * in the table) for a complex64 state of at most 30 qubits whose complex128
 * copy fits in free device memory, else the first candidate's result
 * (ref = 0; its own error then reads 0).  The fastest candidate with
 * err <= max_err is kept (max_err <= 0: no bound, and errors are measured
 * only when table_cap > 0).  When no reference can be allocated errors read
 * -1, and with max_err > 0 no candidate qualifies (QSIM_EUNSUPPORTED).  table
 * (may be NULL when table_cap = 0) receives one entry per candidate, in
 * order; ms < 0 marks a candidate that could not run. */
typedef struct qsim_tune_entry {
    int mode;       /* QSIM_FUSE_* */
    int kmax;
    double ms;      /* time per circuit, CUDA events */
    double err;     /* 2-norm of the difference from the reference result */
    double max_abs; /* largest amplitude difference */
    int ref;        /* 1: reference = gate-by-gate complex128 run; 0: the first candidate */
    int npasses;    /* tensor-core plans: passes */
    int nfp32;      /* tensor-core plans: passes run in FP32 on the CUDA cores */
} qsim_tune_entry;
QSIM_API int qsim_plan_autotune_ex(const qsim_circuit *c, qsim_state *scratch, int reps, double max_err,
                                   qsim_plan **out, qsim_tune_entry *table, int table_cap, int *table_len);
/* Execute a plan on a state of the circuit's width and precision. */
QSIM_API int qsim_apply_fused(qsim_state *s, const qsim_plan *p);

/* ---------------------------------------------------------------- measurement */
/* Probabilities (Sec. 2, measurement operators).  m = 0 or qubits == NULL:
 * out[x] = |psi(x)|^2 for all 2^n x.  Otherwise the marginal over qubits[0..m-1]
 * (distinct, qubits[0] = most significant bit of the output index):
 * out[y] = sum over x whose listed bits spell y of |psi(x)|^2, 2^m doubles.
 * out is device memory if out_on_device, else host memory (then synchronous).
 * |psi|^2 is formed as re*re + im*im in double with no fused multiply-add. */
QSIM_API int qsim_probabilities(qsim_state *s, const int *qubits, int m, double *out, int out_on_device);
/* Squared norm sum_x |psi(x)|^2, accumulated in double; synchronous. */
QSIM_API int qsim_norm2(qsim_state *s, double *out);

/* Shot sampling by inverse CDF over integer weights (replaces the paper's
 * Metropolis sampler, Sec. 2, so that shots are reproducible bit for bit):
 *   w(x) = floor(p(x) 2^62), p(x) = |psi(x)|^2;  CDF(x) = w(0) + ... + w(x)
 *   shot s uses Philox4x32-10 (Salmon et al., SC'11) with counter
 *   (lo32(counter0 + s), hi32(counter0 + s), 0, 0) and key (lo32(seed),
 *   hi32(seed)); with outputs o0, o1: u = o1 * 2^32 + o0,
 *   r = floor(u * CDF(N-1) / 2^64), and the shot is the smallest x with
 *   CDF(x) > r.
 * out: nshots uint64 bitstrings, device memory if out_on_device, else host
 * (synchronous).  The library keeps a scratch array of N/2048 + 1 uint64 in
 * the state.  Returns QSIM_EINVAL if sum p > 1.5 or the weights sum to 0. */
QSIM_API int qsim_sample(qsim_state *s, uint64_t nshots, uint64_t seed, uint64_t counter0, uint64_t *out,
                int out_on_device);
/* The same sampler on caller-supplied probabilities: p_dev is device memory
 * holding N doubles (N >= 1).  Runs on `cuda_stream` and allocates its scratch
 * (N/2048 + 1 uint64) for the duration of the call. */
QSIM_API int qsim_sample_probs(const double *p_dev, uint64_t N, uint64_t nshots, uint64_t seed,
                      uint64_t counter0, uint64_t *out, int out_on_device, void *cuda_stream);

/* The sampler of qsim_sample_probs for callers that may not allocate device
 * memory (a framework whose allocator owns the device pool, a service with a
 * memory budget fixed at start-up, a loop that cannot take the device
 * synchronisation cudaMalloc/cudaFree can cause).  The paper has no
 * counterpart; this is a deployment variant.  It calls no allocator: its
 * scratch is a 512.25 KiB array in the library's device image that every GPU
 * loading the library holds until exit, so N is limited to 1 <= N <= 2^27
 * (larger N returns QSIM_EINVAL without launching).  p_dev: N doubles on the
 * device; out_dev: nshots uint64 on the device (required); the call runs on
 * `cuda_stream` and synchronises it before returning (it reads back the
 * total weight to validate the probabilities).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Under CUDA's
 * default lazy module loading the array is placed in device memory when the
 * library's measurement module is first used on a device, which can be this
 * first call: callers that must not see the driver allocate later make one
 * call (or any measurement call) at start-up, or run with
 * CUDA_MODULE_LOADING=EAGER.  The looked-up address is kept for the life of
 * the process, so a cudaDeviceReset while the library is in use is not
 * supported.  All calls share the one array: calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller. */
QSIM_API int qsim_sample_probs_static(const double *p_dev, uint64_t N, uint64_t nshots, uint64_t seed,
                                      uint64_t counter0, uint64_t *out_dev, void *cuda_stream);

/* Measurement collapse (Sec. 2: the operator that collapses and re-normalises
 * a state after a measurement): the outcome's m bits are read with
 * qubits[0] as the most significant; P = sum of |psi(x)|^2 over the x whose
 * listed bits spell the outcome (written to *prob_out if not NULL); those
 * amplitudes are divided by sqrt(P) and all others set to 0.  Synchronous
 * (reads P back); QSIM_EINVAL when P = 0 (the state is then left unchanged). */
QSIM_API int qsim_collapse(qsim_state *s, const int *qubits, int m, uint64_t outcome, double *prob_out);

/* Pauli expectation <psi| sum_t coeff[t] P_t |psi> with P_t given by bit masks
 * (bit q of xmask/zmask: X = (1,0), Y = (1,1), Z = (0,1) on qubit q):
 *   P|y> = i^{#Y} (-1)^{popcount(y & zmask)} |y ^ xmask>.
 * Terms sharing an xmask are evaluated in one pass; partial sums are
 * accumulated in double (for a complex64 state and a diagonal pass with one
 * real coefficient, |psi|^2 times the integer sign sum is formed in fp32 over
 * 16 amplitudes per thread first).  Host arrays of nterms entries; *out (host) receives
 * the real part; synchronous.  (TFIM-type Hamiltonians, Sec. 3.3.) */
QSIM_API int qsim_expectation_pauli(qsim_state *s, int nterms, const uint64_t *xmask,
                           const uint64_t *zmask, const double *coeff, double *out);

/* ---------------------------------------------------------------- gradients */
/* Adjoint-method gradient of E(theta) = <psi0|U(theta)^dag H U(theta)|psi0> for
 * every trainable parameter of circuit c (RX/RY/RZ gates with param_index >= 0),
 * for nsets parameter vectors: params is nsets x nparams (host, row-major).
 * psi0: the start state (a state of the circuit's width in precision dtype,
 * read only; its stream's pending work completes first), or NULL for
 * |0...0>.
 * Writes grads (nsets x nparams, host) and energies (nsets, host; may be NULL).
 * One forward sweep, then one reverse sweep that un-applies each gate to the
 * state and to lambda = H psi and accumulates 2 Re<lambda|dU psi> (for
 * U = exp(-i theta P / 2): Im<lambda|P psi>); complex64 from 12 qubits sums
 * in fp32 within a warp and in double beyond it, otherwise in double.
 * H: nterms Pauli strings as for qsim_expectation_pauli, at most 64 distinct
 * X masks and 128 terms (QSIM_EUNSUPPORTED beyond).  Trainable rotations must
 * be uncontrolled 1-qubit gates, and the complex64 path from 12 qubits takes
 * dense gates of at most 2 targets (QSIM_EUNSUPPORTED otherwise).  dtype: QSIM_C64 or
 * QSIM_C128.  Allocates psi, lambda and the per-rotation partial sums for the
 * duration of the call; synchronous.
 * (The paper obtains gradients only through TensorFlow autodiff, Sec. 2.) */
QSIM_API int qsim_adjoint_grad(const qsim_circuit *c, const qsim_state *psi0, int dtype, int nsets,
                               const double *params, int nterms, const uint64_t *xmask, const uint64_t *zmask,
                               const double *coeff, double *grads, double *energies, void *cuda_stream);
/* Whether qsim_adjoint_grad (complex64, n >= 12) runs its forward and
 * reverse stages through kernels compiled for the circuit's structure (as
 * QSIM_PLAN_SPECIALIZE does for staged plans; compiled once per structure,
 * reused for every parameter set and later call): 1 always, -1 never, 0
 * (default) from 20 qubits.  Process-wide; *previous (may be NULL) receives
 * the mode it replaces; QSIM_EINVAL for another value. */
QSIM_API int qsim_adjoint_specialize(int mode, int *previous);

/* ---------------------------------------------------------------- batches */
typedef struct qsim_batch qsim_batch;

/* A batch of many small circuits (9 <= n <= 20 qubits each, gates of at most
 * 2 targets, complex64 states) run by one persistent kernel: each CTA takes
 * the next circuit from a device work counter (largest first) and simulates
 * it with the staged register-tile interpreter.  A circuit as wide as the
 * tile (2^(tile_qubits) amplitudes) stays in the CTA's registers for its whole
 * run; a wider one lives in a per-CTA global slot (at most 8 MiB, mostly
 * L2-resident) that each stage streams through the registers tile by tile.
 * The CTA then writes <sum_i Z_i Z_{i+1}> of its final state.  The plan
 * (gate tables) is uploaded once at creation. */
QSIM_API int qsim_batch_create(int ncircuits, const qsim_circuit *const *circuits, qsim_batch **out);
QSIM_API int qsim_batch_destroy(qsim_batch *b);
/* Run every circuit from |0...0> on `cuda_stream`; out_dev: device array of
 * ncircuits doubles receiving <sum_{i=0}^{n-2} Z_i Z_{i+1}> per circuit.
 * Safe to capture in a CUDA graph (the work counter is reset by a memset
 * node inside the captured sequence). */
QSIM_API int qsim_batch_run(qsim_batch *b, double *out_dev, void *cuda_stream);
/* Tuning knobs: CTAs per SM (1..8) and tile width in qubits (9..12, at most
 * the smallest circuit's width; threads per CTA = 2^(tile_qubits - 4));
 * 0 = automatic. */
QSIM_API int qsim_batch_set_config(qsim_batch *b, int ctas_per_sm, int tile_qubits);
/* Autotuner: runs the batch (reps timed runs per candidate, CUDA events on
 * `cuda_stream`) for every tile width / CTAs-per-SM candidate, keeps the
 * fastest as the batch's configuration and reports it (outputs may be NULL). */
QSIM_API int qsim_batch_autotune(qsim_batch *b, void *cuda_stream, int reps, int *best_tile_qubits,
                                 int *best_ctas_per_sm, double *best_ms);

/* ---------------------------------------------------------------- evolution
 * psi <- exp(-i theta D) psi for the diagonal Pauli sum
 * D = sum_t coeff[t] Z(zmask[t]) (Z on every qubit set in zmask[t]): the
 * diagonal factor of a Trotter step of time evolution (Sec. 3.3, the
 * adiabatic evolution benchmark, whose Trotter decomposition turns the
 * evolution into a circuit; for the TFIM the Z_i Z_{i+1} terms form this
 * factor).  One sweep over the state; 0 <= nterms <= 128; asynchronous on the
 * state's stream. */
QSIM_API int qsim_apply_pauli_phase(qsim_state *s, int nterms, const uint64_t *zmask, const double *coeff,
                                    double theta);

/* ---------------------------------------------------------------- sliced states
 * The multi-GPU scheme of Sec. 3.1 (its figure: one or several devices, the
 * full state in host memory, slices copied to the GPU and processed in turn).
 * An n-qubit state is split by its top g ("global") qubits into 2^g slices of
 * L = n - g ("local") qubits; slice i holds the amplitudes whose top g bits
 * equal i, in the usual order.  A gate whose targets are local acts on each
 * slice alone; a control, or a diagonal target, on a global qubit only
 * decides per slice what applies.  Every other gate on a global qubit is
 * preceded by an exchange of that qubit with a local one (SWAP step): for
 * global bit b and local position l, every slice pair (i, i | 1<<b) with bit b
 * of i clear swaps the amplitudes of slice i whose bit l is 1 with those of
 * slice i | 1<<b whose bit l is 0.  Afterwards the two qubits have traded
 * positions; the plan keeps the map.
 *
 * qsim_slice_plan_build: n_global = g (0..QSIM_SLICE_MAX_GLOBAL, < n; L <= 34);
 * each local segment gets a fusion plan (kmax, mode as qsim_plan_build) per
 * distinct value of the global bits it reads.  restore_layout != 0 appends
 * exchanges and local SWAP gates that return every qubit to its own position,
 * so the slices end in the plain order; otherwise qsim_slice_plan_layout gives
 * the final position of each qubit.  Host-side only (no device work). */
typedef struct qsim_slice_plan qsim_slice_plan;
#define QSIM_SLICE_MAX_GLOBAL 16
#define QSIM_SLICE_SEGMENT 0
#define QSIM_SLICE_SWAP 1
#define QSIM_SLICES_DEVICE 0 /* slices[i] are device pointers              */
#define QSIM_SLICES_HOST 1   /* slices[i] are page-locked host pointers    */
QSIM_API int qsim_slice_plan_build(const qsim_circuit *c, int n_global, int kmax, int mode, int restore_layout,
                                   qsim_slice_plan **out);
QSIM_API int qsim_slice_plan_destroy(qsim_slice_plan *p);
/* Counts (outputs may be NULL): global and local qubits, steps, SWAP steps,
 * segment variants (fusion plans) in total. */
QSIM_API int qsim_slice_plan_info(const qsim_slice_plan *p, int *n_global, int *n_local, int *nsteps, int *nswaps,
                                  int *nvariants);
/* Step i: type (QSIM_SLICE_SEGMENT / QSIM_SLICE_SWAP); for a SWAP the global
 * bit b and local position l; for a SEGMENT the mask of global bits whose
 * value selects the variant and the number of source gates it covers. */
QSIM_API int qsim_slice_plan_step(const qsim_slice_plan *p, int i, int *type, int *global_bit, int *local_pos,
                                  uint32_t *keymask, int *ngates);
/* Final physical position of every logical qubit (n ints). */
QSIM_API int qsim_slice_plan_layout(const qsim_slice_plan *p, int *pos);
/* The local circuit that segment `step` applies to slice `slice` (a new
 * circuit of L qubits, owned by the caller). */
QSIM_API int qsim_slice_segment_circuit(const qsim_slice_plan *p, int step, uint32_t slice, qsim_circuit **out);
/* Apply segment `step` to one slice held in `state` (an L-qubit state, e.g.
 * borrowing the slice's device memory); asynchronous on the state's stream. */
QSIM_API int qsim_slice_apply_segment(const qsim_slice_plan *p, int step, uint32_t slice, qsim_state *state);
/* The SWAP step's data movement between two slices in device memory of this
 * process: a = the slice with the global bit 0, b = its partner; both 2^n_local
 * amplitudes of dtype; asynchronous on `stream`. */
QSIM_API int qsim_slice_exchange(void *a, void *b, int n_local, int dtype, int local_pos, void *stream);
/* For an exchange between processes: gather the 2^(n_local-1) amplitudes of a
 * device slice whose bit local_pos equals `bit` into the contiguous device
 * buffer `out` (pack), or scatter them back from `in` (unpack). */
QSIM_API int qsim_slice_pack(const void *slice, int n_local, int dtype, int local_pos, int bit, void *out,
                             void *stream);
QSIM_API int qsim_slice_unpack(void *slice, int n_local, int dtype, int local_pos, int bit, const void *in,
                               void *stream);
/* Run every step on 2^g slices (each 2^L amplitudes of dtype, 256-byte
 * aligned, distinct).  QSIM_SLICES_DEVICE: in place in device memory, on
 * `stream`.  QSIM_SLICES_HOST: slices stay in page-locked host memory; each
 * pass (a run of SWAP steps and the segment after it) streams groups of
 * slices through two sets of device staging slots on three internal streams
 * (uploads, compute, downloads), so the upload of one slice overlaps the work
 * on another and the download of a third; the call returns after the last
 * download.  QSIM_ENOMEM when two staging slots per set do not fit. */
QSIM_API int qsim_slice_run(const qsim_slice_plan *p, int dtype, void *const *slices, int location, void *stream);

/* ---------------------------------------------------------------- test support
 * The sampler's integer weight of a complex64 amplitude, evaluated on the
 * host by the same source the device runs: floor(p * 2^62) for
 * p = re^2 + im^2 rounded once to double (the inverse-CDF weights
 * qsim_sample draws complex64 shots from), 2^62 for p >= 1 or an infinite
 * part, 0 for a NaN.  Pure function, no device work. */
QSIM_API uint64_t qsim_sampler_weight_c64(float re, float im);
/* The complex64 probability re^2 + im^2 rounded once to double, by the
 * integer rule qsim_probabilities uses for complex64 states (host). */
QSIM_API double qsim_prob_c64(float re, float im);
/* Failure injection on the host (test support; the paper has no counterpart):
 * after `skip` more successful device allocations by the library, the next
 * `count` fail as if the device were out of memory, so every entry point's
 * QSIM_ENOMEM path (and its release of what it had allocated) can be
 * exercised without exhausting a GPU.  (0, 0) turns injection off.  Affects
 * all threads; QSIM_EINVAL for negative arguments. */
QSIM_API int qsim_debug_fail_alloc(int skip, int count);
/* Polls a tensor-core pipeline wait (QSIM_FUSE_TC passes) makes before it
 * gives up (test support; 0 restores the default of 2^26).  A wait that gives
 * up stops every role of its CTA; the CTA still waits, with the default
 * bound, for the tensor-core work it has committed before it frees its tensor
 * memory, and qsim_apply_fused returns QSIM_ETIMEOUT with the state's
 * contents undefined.  A limit of a few polls makes the first waits expire,
 * which tests the timeout path without a fault or a hang. */
QSIM_API int qsim_debug_set_wait_limit(unsigned long long polls);
/* Index bound checks (test support; the paper has no counterpart).  A build
 * compiled with QSIM_DEBUG checks, before every global access of the plain
 * sweeps and of the staged register tiles, that the index lies inside the
 * state; an index outside is counted and its access skipped, and
 * qsim_synchronize then returns QSIM_EINVAL.  Returns the count since the
 * library was loaded (cleared when clear != 0), or -1 in a release build,
 * which has no checks. */
QSIM_API long long qsim_debug_checks(int clear);

/* ---------------------------------------------------------------- profiling */
/* Launch accounting for every kernel the library starts.  When enabled, each
 * launch is bracketed by CUDA events on its own stream; qsim_profile_get
 * synchronises those events and reports, per kernel name, the launches, the
 * summed device time, the summed algorithmic HBM bytes and the summed useful
 * floating-point operations (a complex multiply-add counts 8; tensor-core
 * passes count the complex flops of the gate they apply, not the split). */
QSIM_API int qsim_profile_enable(int on);
QSIM_API int qsim_profile_reset(void);
QSIM_API int qsim_profile_count(int *nkinds);
QSIM_API int qsim_profile_get(int i, const char **name, uint64_t *launches, double *total_ms,
                     double *total_bytes, double *total_flops);
/* Total kernel launches issued by the library since load (always counted;
 * host/device copies are not kernel launches and are not counted). */
QSIM_API uint64_t qsim_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* QSIM_H */

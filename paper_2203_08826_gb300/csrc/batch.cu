// Batched persistent execution of many small circuits (qsim_batch_*).
//
// One launch runs a whole batch.  Every CTA repeatedly takes the next circuit
// from a device work counter (circuits are ordered by cost, largest first, so
// the tail of the launch is made of small ones) and simulates it from |0...0>
// with the register-tile interpreter of the staged fusion (stage_common.cuh):
//   - a circuit whose width equals the tile (2^(9+W) amplitudes) lives in the
//     registers of the CTA for its whole run -- no global memory traffic at
//     all; consecutive stages hand the state over through shared memory;
//   - a wider circuit lives in a per-CTA slot of global memory (at most
//     8 MiB at 20 qubits, mostly L2-resident) that each stage streams through
//     the registers tile by tile, with a CTA barrier between stages.
// Finally the CTA reduces <sum_i Z_i Z_{i+1}> of its state: fp32 sums of at
// most 16 terms per thread (fp64 runs at 1/64 of the fp32 rate), then
// double.  No CTA waits on another, so the launch cannot deadlock; the
// counter is reset by a memset on the same stream, which keeps the pair
// capturable in a CUDA graph.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "internal.h"
#include "plan.h"
#include "stage_common.cuh"

namespace qsim {
namespace {
using namespace stage;

struct BCirc {
    int n, stage0, nstages, pad;
};
struct BStage {
    IndexMap outer;  // zeros at the tile qubits (tile id -> base index)
    int op0, nops, phase_base, phase0, pool0, aux0;
};

struct BatchParams {
    const BCirc *circ;
    const BStage *stages;
    const StageOp *ops;
    const Phase *phases;
    const float2 *pool;
    const uint64_t *aux;
    const int *order;
    int ncirc;
    int *counter;
    float2 *slots;
    uint64_t slot_amps;
    double *out;
};

struct GSrc {
    const StageOp *ops;
    const Phase *phases;
    const float2 *pl;
    const uint64_t *ax;
    __device__ const StageOp &op(int o) const { return ops[o]; }
    __device__ const Phase &phase(int i) const { return phases[i]; }
    __device__ float2 pool(int i) const { return pl[i]; }
    __device__ uint64_t aux(int i) const { return ax[i]; }
};

// sum_i Z_i Z_{i+1} at basis state x (open chain), exact as a float
__device__ __forceinline__ float zz_chain(uint64_t x, int n) {
    const uint64_t m = (uint64_t(1) << (n - 1)) - 1;
    return float(n - 1 - 2 * __popcll((x ^ (x >> 1)) & m));
}

// Index bits of the register qubits of phase P, read once: the phases live
// in global memory, which the stage's own stores may alias, so offsets
// computed from P directly would reload it for every amplitude.
struct RegMasks {
    uint64_t m[REG_BITS];
    __device__ __forceinline__ explicit RegMasks(const Phase &P) {
#pragma unroll
        for (int b = 0; b < REG_BITS; ++b) m[b] = uint64_t(1) << P.rq[b];
    }
    __device__ __forceinline__ uint64_t operator()(int j) const {
        uint64_t o = 0;
#pragma unroll
        for (int b = 0; b < REG_BITS; ++b)
            if ((j >> b) & 1) o |= m[b];
        return o;
    }
};

template <int W>
__global__ void __launch_bounds__(32 << W, W <= 3 ? 3 : 1) k_batch(const BatchParams bp) {
    using C = float2;
    constexpr int NR = 1 << REG_BITS;
    constexpr int TB = LANE_BITS + REG_BITS + W;  // tile qubits
    extern __shared__ unsigned char smem_raw[];
    C *tile = reinterpret_cast<C *>(smem_raw);
    __shared__ int s_ci;
    __shared__ double s_red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C *slot = bp.slots + uint64_t(blockIdx.x) * bp.slot_amps;

    for (;;) {
        if (threadIdx.x == 0) s_ci = atomicAdd(bp.counter, 1);
        __syncthreads();
        const int idx = s_ci;
        __syncthreads();
        if (idx >= bp.ncirc) break;
        const int ci = bp.order[idx];
        const BCirc bc = bp.circ[ci];
        const int n = bc.n;
        double acc = 0.0;
        if (n == TB) {
            // the whole state is one tile, held in registers
            C v[NR];
            int ph = 0;
            uint64_t base = 0;
            for (int s = 0; s < bc.nstages; ++s) {
                const BStage &S = bp.stages[bc.stage0 + s];
                const GSrc src{bp.ops + S.op0, bp.phases + S.phase_base, bp.pool + S.pool0, bp.aux + S.aux0};
                ph = S.phase0;
                base = thread_base<W>(src.phase(ph), 0, lane, warp);
                {
                    const RegMasks rm(src.phase(ph));
#pragma unroll
                    for (int j = 0; j < NR; ++j) {
                        const uint64_t x = base | rm(j);
                        if (s == 0) v[j] = make_float2(x == 0 ? 1.f : 0.f, 0.f);
                        else v[j] = tile[x];
                    }
                }
                if (s > 0) __syncthreads();  // hand-over reads before any exchange writes
                stage_exec<C, W>(src, S.nops, v, ph, base, 0, tile, lane, warp);
                const RegMasks rm(src.phase(ph));
                if (s + 1 < bc.nstages) {
                    // hand over through shared memory, indexed by the amplitude index
                    __syncthreads();
#pragma unroll
                    for (int j = 0; j < NR; ++j) tile[base | rm(j)] = v[j];
                    __syncthreads();
                } else {
                    float f = 0.f;
#pragma unroll
                    for (int j = 0; j < NR; ++j) {
                        const uint64_t x = base | rm(j);
                        f = fmaf(fmaf(v[j].x, v[j].x, v[j].y * v[j].y), zz_chain(x, n), f);
                    }
                    acc = double(f);
                }
            }
        } else {
            const uint64_t N = uint64_t(1) << n;
            for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) slot[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
            __syncthreads();
            const uint64_t ntiles = uint64_t(1) << (n - TB);
            for (int s = 0; s < bc.nstages; ++s) {
                const BStage &S = bp.stages[bc.stage0 + s];
                const GSrc src{bp.ops + S.op0, bp.phases + S.phase_base, bp.pool + S.pool0, bp.aux + S.aux0};
                for (uint64_t t = 0; t < ntiles; ++t) {
                    uint64_t tb = t;
                    for (int i = 0; i < S.outer.nins; ++i) {
                        const uint64_t low = tb & ((uint64_t(1) << S.outer.ins[i]) - 1);
                        tb = ((tb ^ low) << 1) | low;
                    }
                    int ph = S.phase0;
                    uint64_t base = thread_base<W>(src.phase(ph), tb, lane, warp);
                    C v[NR];
                    {
                        const RegMasks rm(src.phase(ph));
#pragma unroll
                        for (int j = 0; j < NR; ++j) v[j] = slot[base | rm(j)];
                    }
                    stage_exec<C, W>(src, S.nops, v, ph, base, tb, tile, lane, warp);
                    const RegMasks rm(src.phase(ph));
#pragma unroll
                    for (int j = 0; j < NR; ++j) slot[base | rm(j)] = v[j];
                }
                __syncthreads();  // the next stage reads what other threads wrote
            }
            // fp32 sums of 16 terms, added in double
            for (uint64_t i0 = threadIdx.x; i0 < N; i0 += uint64_t(blockDim.x) * 16) {
                float f = 0.f;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const uint64_t i = i0 + uint64_t(u) * blockDim.x;
                    if (i < N) {
                        const C a = slot[i];
                        f = fmaf(fmaf(a.x, a.x, a.y * a.y), zz_chain(i, n), f);
                    }
                }
                acc += double(f);
            }
        }
        // block reduction in double
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < int(blockDim.x >> 5); ++w) t += s_red[w];
            bp.out[ci] = t;
        }
        __syncthreads();
    }
}

struct Packed {
    bool ready = false;
    int W = 3;
    double flops = 0;  // useful flops of one run of the whole batch
    std::vector<BCirc> circ;
    std::vector<BStage> stages;
    std::vector<StageOp> ops;
    std::vector<Phase> phases;
    std::vector<float2> pool;
    std::vector<uint64_t> aux;
    // device copies
    BCirc *d_circ = nullptr;
    BStage *d_stages = nullptr;
    StageOp *d_ops = nullptr;
    Phase *d_phases = nullptr;
    float2 *d_pool = nullptr;
    uint64_t *d_aux = nullptr;
    void release() {
        cudaFree(d_circ);
        cudaFree(d_stages);
        cudaFree(d_ops);
        cudaFree(d_phases);
        cudaFree(d_pool);
        cudaFree(d_aux);
        d_aux = nullptr;
        d_circ = nullptr;
        d_stages = nullptr;
        d_ops = nullptr;
        d_phases = nullptr;
        d_pool = nullptr;
        ready = false;
    }
};

int sm_count_b() { return device_sm_count(); }

}  // namespace
}  // namespace qsim

using namespace qsim;

struct qsim_batch {
    std::vector<qsim_circuit> circuits;  // copies
    int nmin = 64, nmax = 0;
    int W = 0;            // 0 = automatic
    int ctas_per_sm = 0;  // 0 = automatic
    Packed packed[4];     // per W (0..3)
    std::vector<int> order;
    int *d_order = nullptr;
    int *d_counter = nullptr;
    float2 *d_slots = nullptr;
    size_t slot_ctas = 0;
    double *d_tune_out = nullptr;
    ~qsim_batch() {
        for (Packed &p : packed) p.release();
        cudaFree(d_order);
        cudaFree(d_counter);
        cudaFree(d_slots);
        cudaFree(d_tune_out);
    }
};

namespace {

int pack(qsim_batch &b, int W) {
    Packed &pk = b.packed[W];
    if (pk.ready) return QSIM_OK;
    pk.W = W;
    pk.circ.clear();
    pk.stages.clear();
    pk.ops.clear();
    pk.phases.clear();
    pk.pool.clear();
    pk.aux.clear();
    pk.flops = 0;
    for (const qsim_circuit &c : b.circuits) {
        std::vector<stage::Stage> st;
        QSIM_TRY(stage::plan_stage_list(c, W, false, st, false));
        BCirc bc{c.n, int(pk.stages.size()), int(st.size()), 0};
        for (const stage::Stage &s : st) {
            if (s.plain) return set_error(QSIM_EUNSUPPORTED, "batch circuits need gates of at most 2 targets");
            pk.flops += stage::stage_exec_flops_per_amp(s) * double(uint64_t(1) << c.n);
            BStage bs{};
            int tq[LANE_BITS + MAX_SLOTS];
            int nt = 0;
            for (int q = 0; q < LANE_BITS; ++q) tq[nt++] = q;
            for (int q : s.slots) tq[nt++] = q;
            bs.outer = make_index_map(tq, nt, nullptr, 0);
            bs.op0 = int(pk.ops.size());
            bs.nops = int(s.ops.size());
            bs.phase_base = int(pk.phases.size());
            bs.phase0 = s.phase0;
            bs.pool0 = int(pk.pool.size());
            bs.aux0 = int(pk.aux.size());
            pk.aux.insert(pk.aux.end(), s.aux.begin(), s.aux.end());
            pk.ops.insert(pk.ops.end(), s.ops.begin(), s.ops.end());
            pk.phases.insert(pk.phases.end(), s.phases.begin(), s.phases.end());
            for (const cd &z : s.pool) pk.pool.push_back(make_float2(float(z.real()), float(z.imag())));
            pk.stages.push_back(bs);
        }
        pk.circ.push_back(bc);
    }
    auto up = [](auto &vec, auto **dst, const char *what) -> int {
        using T = typename std::remove_reference<decltype(vec)>::type::value_type;
        const size_t bytes = std::max<size_t>(1, vec.size()) * sizeof(T);
        QSIM_CUDA_TRY(dev_alloc(reinterpret_cast<void **>(dst), bytes), what);
        if (!vec.empty()) QSIM_CUDA_TRY(cudaMemcpy(*dst, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice), what);
        return QSIM_OK;
    };
    QSIM_TRY(up(pk.circ, &pk.d_circ, "batch circuits"));
    QSIM_TRY(up(pk.stages, &pk.d_stages, "batch stages"));
    QSIM_TRY(up(pk.ops, &pk.d_ops, "batch ops"));
    QSIM_TRY(up(pk.phases, &pk.d_phases, "batch phases"));
    QSIM_TRY(up(pk.pool, &pk.d_pool, "batch pool"));
    QSIM_TRY(up(pk.aux, &pk.d_aux, "batch aux"));
    pk.ready = true;
    return QSIM_OK;
}

int choose_W(const qsim_batch &b) {
    if (b.W) return b.W;
    return std::max(0, std::min(3, b.nmin - LANE_BITS - REG_BITS));
}

template <int W>
int launch_batch(qsim_batch &b, double *out, cudaStream_t st, int ctas_per_sm) {
    Packed &pk = b.packed[W];
    const size_t smem = (size_t(1) << (LANE_BITS + REG_BITS + W)) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        QSIM_CUDA_TRY(cudaFuncSetAttribute(k_batch<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                      "batch smem attribute");
        attr = true;
    }
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        QSIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<W>, 32 << W, smem), "occupancy");
        per_sm = std::max(1, occ);
    }
    const size_t grid = std::min<size_t>(size_t(sm_count_b()) * per_sm, b.circuits.size());
    const uint64_t slot_amps = uint64_t(1) << b.nmax;
    if (b.nmax > LANE_BITS + REG_BITS + W && grid > b.slot_ctas) {
        // per-CTA state slots for circuits wider than one tile
        if (b.d_slots) {
            cudaStreamSynchronize(st);
            cudaFree(b.d_slots);
            b.d_slots = nullptr;
        }
        QSIM_CUDA_TRY(dev_alloc(&b.d_slots, grid * slot_amps * sizeof(float2)), "batch slots");
        b.slot_ctas = grid;
    }
    BatchParams bp{};
    bp.circ = pk.d_circ;
    bp.stages = pk.d_stages;
    bp.ops = pk.d_ops;
    bp.phases = pk.d_phases;
    bp.pool = pk.d_pool;
    bp.aux = pk.d_aux;
    bp.order = b.d_order;
    bp.ncirc = int(b.circuits.size());
    bp.counter = b.d_counter;
    bp.slots = b.d_slots;
    bp.slot_amps = slot_amps;
    bp.out = out;
    QSIM_CUDA_TRY(cudaMemsetAsync(b.d_counter, 0, sizeof(int), st), "batch counter reset");
    double bytes = 0;
    for (const qsim_circuit &c : b.circuits) bytes += double(uint64_t(1) << c.n) * 8.0;
    LaunchScope ls(K_BATCH, st, bytes, pk.flops);
    k_batch<W><<<unsigned(grid), 32 << W, smem, st>>>(bp);
    QSIM_CUDA_TRY(cudaGetLastError(), "batch launch");
    return QSIM_OK;
}

int run_batch(qsim_batch &b, double *out, cudaStream_t st, int W, int ctas) {
    QSIM_TRY(pack(b, W));
    switch (W) {
        case 0: return launch_batch<0>(b, out, st, ctas);
        case 1: return launch_batch<1>(b, out, st, ctas);
        case 2: return launch_batch<2>(b, out, st, ctas);
        default: return launch_batch<3>(b, out, st, ctas);
    }
}

}  // namespace

extern "C" {

int qsim_batch_create(int ncircuits, const qsim_circuit *const *circuits, qsim_batch **out) {
    if (!out || ncircuits < 1 || !circuits) return set_error(QSIM_EINVAL, "bad batch arguments");
    *out = nullptr;
    qsim_batch *b = new qsim_batch();
    for (int i = 0; i < ncircuits; ++i) {
        if (!circuits[i]) {
            delete b;
            return set_error(QSIM_EINVAL, "circuit %d is NULL", i);
        }
        const int n = circuits[i]->n;
        if (n < LANE_BITS + REG_BITS || n > 20) {
            delete b;
            return set_error(QSIM_EINVAL, "batch circuits need 9 <= n <= 20 qubits (circuit %d has %d)", i, n);
        }
        b->circuits.push_back(*circuits[i]);
        b->nmin = std::min(b->nmin, n);
        b->nmax = std::max(b->nmax, n);
    }
    // largest (2^n x gates) first
    b->order.resize(ncircuits);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const double cx = double(uint64_t(1) << b->circuits[x].n) * double(b->circuits[x].gates.size());
        const double cy = double(uint64_t(1) << b->circuits[y].n) * double(b->circuits[y].gates.size());
        return cx > cy;
    });
    cudaError_t e = dev_alloc(&b->d_order, sizeof(int) * ncircuits);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * ncircuits, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_alloc(&b->d_counter, sizeof(int));
    if (e != cudaSuccess) {
        delete b;
        return cuda_error(e, "batch setup");
    }
    // validate every circuit now (host planning) for the default tile
    const int rc = pack(*b, choose_W(*b));
    if (rc != QSIM_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return QSIM_OK;
}

int qsim_batch_destroy(qsim_batch *b) {
    delete b;
    return QSIM_OK;
}

int qsim_batch_set_config(qsim_batch *b, int ctas_per_sm, int tile_qubits) {
    if (!b) return set_error(QSIM_EINVAL, "batch is NULL");
    if (ctas_per_sm < 0 || ctas_per_sm > 8) return set_error(QSIM_EINVAL, "ctas_per_sm outside 0..8");
    if (tile_qubits) {
        const int W = tile_qubits - LANE_BITS - REG_BITS;
        if (W < 0 || W > 3 || tile_qubits > b->nmin)
            return set_error(QSIM_EINVAL, "tile_qubits must be in 9..min(12, smallest circuit width)");
        b->W = W;
        QSIM_TRY(pack(*b, W));
    } else {
        b->W = 0;
    }
    b->ctas_per_sm = ctas_per_sm;
    return QSIM_OK;
}

int qsim_batch_run(qsim_batch *b, double *out_dev, void *cuda_stream) {
    if (!b || !out_dev) return set_error(QSIM_EINVAL, "NULL argument");
    return run_batch(*b, out_dev, static_cast<cudaStream_t>(cuda_stream), choose_W(*b), b->ctas_per_sm);
}

int qsim_batch_autotune(qsim_batch *b, void *cuda_stream, int reps, int *best_tile_qubits, int *best_ctas_per_sm,
                        double *best_ms) {
    if (!b) return set_error(QSIM_EINVAL, "batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (reps < 1) reps = 2;
    if (!b->d_tune_out)
        QSIM_CUDA_TRY(dev_alloc(&b->d_tune_out, sizeof(double) * b->circuits.size()), "autotune buffer");
    cudaEvent_t e0, e1;
    QSIM_CUDA_TRY(cudaEventCreate(&e0), "event");
    QSIM_CUDA_TRY(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int bw = choose_W(*b), bc = 0;
    const int wmax = std::min(3, b->nmin - LANE_BITS - REG_BITS);
    for (int W = std::max(0, wmax - 1); W <= wmax; ++W)
        for (int ctas = 1; ctas <= 4; ++ctas) {
            int rc = run_batch(*b, b->d_tune_out, st, W, ctas);  // warm-up (and packing)
            if (rc != QSIM_OK) continue;
            cudaEventRecord(e0, st);
            for (int r = 0; r < reps && rc == QSIM_OK; ++r) rc = run_batch(*b, b->d_tune_out, st, W, ctas);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || rc != QSIM_OK) continue;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best) {
                best = ms;
                bw = W;
                bc = ctas;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->W = bw;
    b->ctas_per_sm = bc;
    if (best_tile_qubits) *best_tile_qubits = LANE_BITS + REG_BITS + bw;
    if (best_ctas_per_sm) *best_ctas_per_sm = bc;
    if (best_ms) *best_ms = best;
    return QSIM_OK;
}

}  // extern "C"

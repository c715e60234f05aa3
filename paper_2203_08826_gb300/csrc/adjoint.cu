// Adjoint-method gradients (qsim_adjoint_grad).
//
// For E(theta) = <psi_L| H |psi_L> with psi_l = U_l psi_{l-1}, psi_0 = |0>, and
// lambda_l = U_{l+1}^dag ... U_L^dag H psi_L, every parametrised rotation
// U_l = exp(-i theta P / 2) contributes
//     dE/dtheta = 2 Re <lambda_l| dU_l/dtheta psi_{l-1}> = Im <lambda_l| P |psi_l>
// (dU/dtheta = (-i/2) P U).  One forward sweep builds psi_L, one pass forms
// lambda = H psi_L, and one reverse sweep walks the gates from the last to the
// first: at a rotation it accumulates Im<lambda|P|psi> (double, per block) and
// un-applies U_l to both states in the same pass; any other gate is
// un-applied to both states with the plain sweeps.  The paper differentiates
// only through TensorFlow's automatic differentiation (Sec. 2); this is the
// GPU-native replacement.
#include <atomic>
#include <cstring>

#include "internal.h"
#include "plan.h"
#include "stage_common.cuh"

namespace qsim {
namespace {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

constexpr int ADJ_BLOCKS_PER_SM = 4;
constexpr int HAPPLY_GROUPS = 64;
constexpr int HAPPLY_TERMS = 128;

int sm_count_a() { return device_sm_count(); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v) {
    __shared__ double red[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = 0;
    if (w == 0) {
        v = lane < int(blockDim.x >> 5) ? red[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

template <typename C> struct M2 {
    C m00, m01, m10, m11;
};

template <typename C> __device__ __forceinline__ C mul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C add(C a, C b) {
    a.x += b.x;
    a.y += b.y;
    return a;
}

// One rotation of the reverse sweep: g += Im(<lambda|P|psi>) over the pairs
// of qubit q (partials per block), then psi <- U^dag psi, lambda <- U^dag lambda.
// P: 0 = X, 1 = Y, 2 = Z.
template <typename C>
__global__ void __launch_bounds__(256) k_adj_rot(C *__restrict__ psi, C *__restrict__ lam, uint64_t npairs, int q,
                                                 int P, M2<C> u, double *__restrict__ partial) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t bit = uint64_t(1) << q;
    double acc = 0;
    for (uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < npairs; g += stride) {
        const uint64_t low = g & (bit - 1);
        const uint64_t i0 = ((g ^ low) << 1) | low, i1 = i0 | bit;
        const C a0 = psi[i0], a1 = psi[i1], l0 = lam[i0], l1 = lam[i1];
        C p0, p1;
        if (P == 0) {
            p0 = a1;
            p1 = a0;
        } else if (P == 1) {  // Y|0> = i|1>, Y|1> = -i|0>:  (P psi)_0 = -i a1, (P psi)_1 = i a0
            p0.x = a1.y;
            p0.y = -a1.x;
            p1.x = -a0.y;
            p1.y = a0.x;
        } else {
            p0 = a0;
            p1.x = -a1.x;
            p1.y = -a1.y;
        }
        // Im(conj(l) p) = l.x p.y - l.y p.x
        acc += double(l0.x) * p0.y - double(l0.y) * p0.x + double(l1.x) * p1.y - double(l1.y) * p1.x;
        psi[i0] = add(mul(u.m00, a0), mul(u.m01, a1));
        psi[i1] = add(mul(u.m10, a0), mul(u.m11, a1));
        lam[i0] = add(mul(u.m00, l0), mul(u.m01, l1));
        lam[i1] = add(mul(u.m10, l0), mul(u.m11, l1));
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// lambda[y] = sum_groups f_g(y ^ X_g) psi[y ^ X_g],
// f_g(x) = sum_{t in g} c_t (-1)^{popcount(x & Z_t)},  c_t = coeff_t i^{#Y_t}
struct HParams {
    int ngroups;
    uint64_t X[HAPPLY_GROUPS];
    int t0[HAPPLY_GROUPS + 1];
    uint64_t Z[HAPPLY_TERMS];
    double cr[HAPPLY_TERMS], ci[HAPPLY_TERMS];
    float fr[HAPPLY_TERMS], fi[HAPPLY_TERMS];  // the same, rounded once for complex64
};

__device__ __forceinline__ void hcoef(const HParams &h, int t, float &r, float &i) {
    r = h.fr[t];
    i = h.fi[t];
}
__device__ __forceinline__ void hcoef(const HParams &h, int t, double &r, double &i) {
    r = h.cr[t];
    i = h.ci[t];
}

// Arithmetic in the state's own precision (fp32 for complex64: lambda is
// stored in complex64 anyway; the coefficients are rounded to fp32 on the
// host), so the fp64 units are not on this path.
template <typename C>
__global__ void __launch_bounds__(256) k_happly(const C *__restrict__ psi, C *__restrict__ lam, uint64_t N,
                                                const __grid_constant__ HParams h, int accumulate) {
    using R = decltype(C::x);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t y = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; y < N; y += stride) {
        R sr = 0, si = 0;
#pragma unroll 4
        for (int g = 0; g < h.ngroups; ++g) {
            const uint64_t x = y ^ h.X[g];
            const C a = psi[x];
            R fr = 0, fi = 0;
            for (int t = h.t0[g]; t < h.t0[g + 1]; ++t) {
                const bool odd = __popcll(x & h.Z[t]) & 1;
                R cr, ci;
                hcoef(h, t, cr, ci);
                fr += odd ? -cr : cr;
                fi += odd ? -ci : ci;
            }
            sr += fr * a.x - fi * a.y;
            si += fr * a.y + fi * a.x;
        }
        C o = accumulate ? lam[y] : C{};
        o.x += sr;
        o.y += si;
        lam[y] = o;
    }
}

// Tiled form for the groups whose X mask lies inside a tile: a CTA holds
// the 2^(5 + m) amplitudes whose index varies over bits 0..4 and the chunk
// [c0, c0 + m) (the other bits fixed by the tile id) in shared memory, so
// psi[y ^ X_g] is a shared-memory read; lambda is written by the first pass
// and accumulated by the others.  Bits 0..4 in every tile keep the global
// accesses 256-byte contiguous per warp.  Each thread holds PER amplitudes
// and walks the groups and terms once for all of them.  The diagonal group
// (X = 0, real coefficients, up to 64 Z strings) is evaluated from tables:
// the parity of every term is one XOR of per-byte masks of the index,
// P(y) = XOR_b ptab[b][byte b of y], and f(y) = sum_j stab[j][byte j of P]
// with stab[j][m] = sum over the 8 terms of byte j of c_t (-1)^(bit of m).
struct HTile {
    int c0, m, first, ng;
    int dg;                        // pass-local index of the table group, or -1
    int nbytes, nsum;              // its table sizes (index bytes, term bytes)
    int gidx[HAPPLY_GROUPS];       // groups of this pass (indices into HParams)
    uint32_t xl[HAPPLY_GROUPS];    // their X masks in tile coordinates
};
constexpr int HTAB_TERMS = 64;

template <typename C, int PER>
__global__ void __launch_bounds__(256) k_happly_tile(const C *__restrict__ psi, C *__restrict__ lam,
                                                     const __grid_constant__ HParams h,
                                                     const __grid_constant__ HTile tp,
                                                     const void *__restrict__ tabs) {
    using R = decltype(C::x);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t TN = 1u << (5 + tp.m);
    C *tile = reinterpret_cast<C *>(smem_raw);
    uint64_t *ptab = reinterpret_cast<uint64_t *>(tile + TN);
    R *stab = reinterpret_cast<R *>(ptab + tp.nbytes * 256);
    const uint64_t t = blockIdx.x;
    const uint64_t lowm = (uint64_t(1) << (tp.c0 - 5)) - 1;
    const uint64_t base = ((t & lowm) << 5) | ((t >> (tp.c0 - 5)) << (tp.c0 + tp.m));
    auto glob = [&](uint32_t l) { return base | uint64_t(l & 31u) | (uint64_t(l >> 5) << tp.c0); };
    for (uint32_t l = threadIdx.x; l < TN; l += blockDim.x) tile[l] = psi[glob(l)];
    if (tp.dg >= 0) {
        const uint64_t *gp = static_cast<const uint64_t *>(tabs);
        for (int i = threadIdx.x; i < tp.nbytes * 256; i += blockDim.x) ptab[i] = gp[i];
        const R *gs = reinterpret_cast<const R *>(gp + tp.nbytes * 256);
        for (int i = threadIdx.x; i < tp.nsum * 256; i += blockDim.x) stab[i] = gs[i];
    }
    __syncthreads();
    uint64_t y[PER];
    R sr[PER], si[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        y[u] = glob(threadIdx.x + uint32_t(u) * blockDim.x);
        sr[u] = 0;
        si[u] = 0;
    }
    for (int g = 0; g < tp.ng; ++g) {
        if (g == tp.dg) {
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                uint64_t P = 0;
                for (int b = 0; b < tp.nbytes; ++b) P ^= ptab[b * 256 + int((y[u] >> (8 * b)) & 255)];
                R f = 0;
                for (int j = 0; j < tp.nsum; ++j) f += stab[j * 256 + int((P >> (8 * j)) & 255)];
                const C a = tile[threadIdx.x + uint32_t(u) * blockDim.x];
                sr[u] += f * a.x;
                si[u] += f * a.y;
            }
            continue;
        }
        const int gi = tp.gidx[g];
        const uint64_t X = h.X[gi];
        const uint32_t xl = tp.xl[g];
        R fr[PER], fi[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) fr[u] = fi[u] = 0;
        for (int k = h.t0[gi]; k < h.t0[gi + 1]; ++k) {
            const uint64_t Z = h.Z[k];
            R cr, ci;
            hcoef(h, k, cr, ci);
            if (Z == 0) {  // pure X string: a constant factor
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    fr[u] += cr;
                    fi[u] += ci;
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const bool odd = __popcll((y[u] ^ X) & Z) & 1;
                fr[u] += odd ? -cr : cr;
                fi[u] += odd ? -ci : ci;
            }
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const C a = tile[(threadIdx.x + uint32_t(u) * blockDim.x) ^ xl];
            sr[u] += fr[u] * a.x - fi[u] * a.y;
            si[u] += fr[u] * a.y + fi[u] * a.x;
        }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        C o = tp.first ? C{} : lam[y[u]];
        o.x += sr[u];
        o.y += si[u];
        lam[y[u]] = o;
    }
}

// lambda = H psi: tiled passes for every group whose X mask fits a tile
// (bits 0..T-1, then bits 0..4 plus successive chunks of the high bits),
// one gather pass for the rest.  Built once per Hamiltonian and state size.
template <typename C>
struct HPlan {
    using R = decltype(C::x);
    int n = 0;
    std::vector<HTile> passes;
    HParams left;
    bool gather = false;  // the gather pass runs (groups fitting no tile)
    void *dtabs = nullptr;
    ~HPlan() {
        if (dtabs) cudaFree(dtabs);
    }

    int build(const HParams &hp, int n_, cudaStream_t st) {
        n = n_;
        const int TBMAX = sizeof(C) == 8 ? 12 : 11;  // 32 KiB tiles
        if (n >= TBMAX) {
            HTile t0{};
            t0.c0 = 5;
            t0.m = TBMAX - 5;
            t0.dg = -1;
            passes.push_back(t0);
            for (int c0 = TBMAX; c0 < n;) {
                HTile t{};
                t.c0 = c0;
                t.m = std::min(TBMAX - 5, n - c0);
                t.dg = -1;
                passes.push_back(t);
                c0 += t.m;
            }
        }
        memset(&left, 0, sizeof left);
        int nt = 0;
        for (int g = 0; g < hp.ngroups; ++g) {
            bool placed = false;
            for (HTile &t : passes) {
                const uint64_t B = 31u | (((uint64_t(1) << t.m) - 1) << t.c0);
                if (hp.X[g] & ~B) continue;
                const int nterm = hp.t0[g + 1] - hp.t0[g];
                if (hp.X[g] == 0 && t.dg < 0 && nterm > 4 && nterm <= HTAB_TERMS) {
                    // tables for the diagonal group
                    t.dg = t.ng;
                    t.nbytes = (n + 7) / 8;
                    t.nsum = (nterm + 7) / 8;
                    std::vector<uint64_t> pt(size_t(t.nbytes) * 256, 0);
                    std::vector<R> sm(size_t(t.nsum) * 256, R(0));
                    for (int b = 0; b < t.nbytes; ++b)
                        for (int v = 0; v < 256; ++v)
                            for (int k = 0; k < nterm; ++k)
                                if (__builtin_popcountll((hp.Z[hp.t0[g] + k] >> (8 * b)) & uint64_t(v)) & 1)
                                    pt[size_t(b) * 256 + size_t(v)] |= uint64_t(1) << k;
                    for (int j = 0; j < t.nsum; ++j)
                        for (int v = 0; v < 256; ++v) {
                            double f = 0;
                            for (int k = 8 * j; k < std::min(nterm, 8 * j + 8); ++k)
                                f += ((v >> (k - 8 * j)) & 1) ? -hp.cr[hp.t0[g] + k] : hp.cr[hp.t0[g] + k];
                            sm[size_t(j) * 256 + size_t(v)] = R(f);
                        }
                    const size_t pb = pt.size() * sizeof(uint64_t), sb = sm.size() * sizeof(R);
                    QSIM_CUDA_TRY(dev_alloc(&dtabs, pb + sb), "hamiltonian tables");
                    QSIM_CUDA_TRY(cudaMemcpyAsync(dtabs, pt.data(), pb, cudaMemcpyHostToDevice, st), "hamiltonian tables");
                    QSIM_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(dtabs) + pb, sm.data(), sb,
                                                  cudaMemcpyHostToDevice, st),
                                  "hamiltonian tables");
                    QSIM_CUDA_TRY(cudaStreamSynchronize(st), "hamiltonian tables");
                }
                t.gidx[t.ng] = g;
                t.xl[t.ng] = uint32_t((hp.X[g] & 31u) | ((hp.X[g] >> t.c0) << 5));
                ++t.ng;
                placed = true;
                break;
            }
            if (placed) continue;
            left.X[left.ngroups] = hp.X[g];
            left.t0[left.ngroups] = nt;
            for (int k = hp.t0[g]; k < hp.t0[g + 1]; ++k, ++nt) {
                left.Z[nt] = hp.Z[k];
                left.cr[nt] = hp.cr[k];
                left.ci[nt] = hp.ci[k];
                left.fr[nt] = hp.fr[k];
                left.fi[nt] = hp.fi[k];
            }
            ++left.ngroups;
            left.t0[left.ngroups] = nt;
        }
        bool first = true;
        for (HTile &t : passes) {
            if (t.ng == 0) continue;
            t.first = first ? 1 : 0;
            first = false;
        }
        gather = left.ngroups > 0;
        return QSIM_OK;
    }

    static size_t smem_of(const HTile &t) {
        return (size_t(1) << (5 + t.m)) * sizeof(C) +
               (t.dg >= 0 ? size_t(t.nbytes) * 256 * 8 + size_t(t.nsum) * 256 * sizeof(R) : 0);
    }

    template <int PER>
    int launch(const C *psi, C *lam, const HParams &hp, const HTile &t, unsigned threads, cudaStream_t st) {
        static bool attr = false;
        if (!attr) {
            QSIM_CUDA_TRY(cudaFuncSetAttribute(k_happly_tile<C, PER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               64 * 1024),
                          "hamiltonian apply smem");
            attr = true;
        }
        const uint64_t ntiles = (uint64_t(1) << n) >> (5 + t.m);
        k_happly_tile<C, PER><<<unsigned(ntiles), threads, smem_of(t), st>>>(psi, lam, hp, t, dtabs);
        QSIM_CUDA_TRY(cudaGetLastError(), "hamiltonian apply launch");
        return QSIM_OK;
    }

    int run(const C *psi, C *lam, const HParams &hp, cudaStream_t st) {
        const uint64_t N = uint64_t(1) << n;
        bool wrote = false;
        for (const HTile &t : passes) {
            if (t.ng == 0) continue;
            const uint32_t TN = 1u << (5 + t.m);
            const unsigned threads = std::min<uint32_t>(256, TN);
            LaunchScope ls(K_HAPPLY, st, double(N) * sizeof(C) * (t.first ? 2.0 : 3.0));
            switch (TN / threads) {
                case 16: QSIM_TRY(launch<16>(psi, lam, hp, t, threads, st)); break;
                case 8: QSIM_TRY(launch<8>(psi, lam, hp, t, threads, st)); break;
                case 4: QSIM_TRY(launch<4>(psi, lam, hp, t, threads, st)); break;
                case 2: QSIM_TRY(launch<2>(psi, lam, hp, t, threads, st)); break;
                default: QSIM_TRY(launch<1>(psi, lam, hp, t, threads, st)); break;
            }
            wrote = true;
        }
        if (gather) {
            const int blocks = sm_count_a() * ADJ_BLOCKS_PER_SM;
            LaunchScope ls(K_HAPPLY, st, double(N) * sizeof(C) * (left.ngroups + (wrote ? 2 : 1)));
            k_happly<C><<<blocks, 256, 0, st>>>(psi, lam, N, left, wrote ? 1 : 0);
            QSIM_CUDA_TRY(cudaGetLastError(), "hamiltonian apply launch");
        }
        return QSIM_OK;
    }
};

template <typename C>
__global__ void __launch_bounds__(256) k_dot_re(const C *__restrict__ a, const C *__restrict__ b, uint64_t N,
                                                double *__restrict__ partial) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    double acc = 0;
    if constexpr (sizeof(a[0].x) == 4) {
        // complex64: fp32 sums of 8 terms, added in double (fp64 runs at 1/64
        // of the fp32 rate)
        for (uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < N; i0 += 8 * stride) {
            float f = 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint64_t i = i0 + uint64_t(u) * stride;
                if (i < N) f = fmaf(a[i].x, b[i].x, fmaf(a[i].y, b[i].y, f));
            }
            acc += double(f);
        }
    } else {
        for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride)
            acc += double(a[i].x) * b[i].x + double(a[i].y) * b[i].y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out[r] = sum of row r of partial (rows of `cols` entries), fixed order
__global__ void k_rows(const double *__restrict__ partial, int rows, int cols, double *__restrict__ out) {
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        double acc = 0;
        for (int c = threadIdx.x; c < cols; c += blockDim.x) acc += partial[size_t(r) * cols + c];
        acc = block_sum(acc);
        if (threadIdx.x == 0) out[r] = acc;
    }
}

struct AdjGate {
    bool param = false;
    int P = 0;       // generator for rotations
    int q = 0;
    int pindex = -1;
    Op fwd, inv;     // forward and inverse sweeps (non-parametrised gates)
    std::vector<cd> mfwd;
};

int rotation_matrix(int kind, double th, std::vector<cd> &m) { return gate_matrix(kind, 1, &th, nullptr, m); }

template <typename R>
int adjoint_t(const qsim_circuit &c, const void *psi0, int nsets, const double *params, const HParams &hp, double *grads,
              double *energies, cudaStream_t st) {
    using C = typename CT<R>::T;
    const int n = c.n;
    const uint64_t N = uint64_t(1) << n;
    const int blocks = sm_count_a() * ADJ_BLOCKS_PER_SM;
    int nrot = 0;
    std::vector<int> rot_of_gate(c.gates.size(), -1);
    for (size_t i = 0; i < c.gates.size(); ++i) {
        const GateRec &g = c.gates[i];
        if (g.pindex < 0) continue;
        if (g.nc != 0 || g.k != 1) return set_error(QSIM_EUNSUPPORTED, "trainable rotations must be uncontrolled 1-qubit gates");
        rot_of_gate[i] = nrot++;
    }
    // device buffers: psi, lambda, one row of partials per rotation, reductions
    C *psi = nullptr, *lam = nullptr;
    double *partial = nullptr, *rows = nullptr;
    const size_t prow = size_t(blocks);
    cudaError_t e = dev_alloc(&psi, N * sizeof(C));
    if (e == cudaSuccess) e = dev_alloc(&lam, N * sizeof(C));
    if (e == cudaSuccess) e = dev_alloc(&partial, (size_t(nrot) + 1) * prow * sizeof(double));
    // result rows (gradient terms + energy), two as in the fused path
    const size_t nrow = size_t(nrot) + 1;
    if (e == cudaSuccess) e = dev_alloc(&rows, 2 * nrow * sizeof(double));
    struct Guard {
        void *p[4];
        ~Guard() {
            for (void *x : p)
                if (x) cudaFree(x);
        }
    } guard{{psi, lam, partial, rows}};
    if (e != cudaSuccess) return cuda_error(e, "adjoint buffers");
    // pinned host rows and one event per buffer
    struct HostRows {
        double *h = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~HostRows() {
            if (h) cudaFreeHost(h);
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
        }
    } hr;
    QSIM_CUDA_TRY(cudaMallocHost(&hr.h, 2 * nrow * sizeof(double)), "adjoint host rows");
    for (cudaEvent_t &x : hr.ev) QSIM_CUDA_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "adjoint event");
    auto finish = [&](int set) -> int {
        const int b = set & 1;
        QSIM_CUDA_TRY(cudaEventSynchronize(hr.ev[b]), "adjoint sync");
        const double *row = hr.h + size_t(b) * nrow;
        double *gset = grads + size_t(set) * size_t(c.nparams);
        for (int p = 0; p < c.nparams; ++p) gset[p] = 0.0;
        for (size_t i = 0; i < c.gates.size(); ++i)
            if (rot_of_gate[i] >= 0) gset[c.gates[i].pindex] += row[rot_of_gate[i]];
        if (energies) energies[set] = row[nrot];
        return QSIM_OK;
    };
    std::vector<void *> mats;  // dense k >= 2 matrices (uploaded per set)
    HPlan<C> hplan;
    QSIM_TRY(hplan.build(hp, n, st));
    for (int set = 0; set < nsets; ++set) {
        const double *th = params + size_t(set) * size_t(c.nparams);
        // forward and inverse ops with this set's angles
        std::vector<AdjGate> gs(c.gates.size());
        std::vector<unsigned char> matbuf;
        std::vector<size_t> moff_f(c.gates.size(), size_t(-1)), moff_i(c.gates.size(), size_t(-1));
        const size_t eb = sizeof(C);
        auto stash = [&](const Op &op) -> size_t {
            if (op.type != Op::DENSE || op.k < 2) return size_t(-1);
            const size_t d = size_t(1) << op.k, off = matbuf.size();
            matbuf.resize(off + d * d * eb);
            for (size_t i = 0; i < d * d; ++i) {
                R v[2] = {R(op.m[i].real()), R(op.m[i].imag())};
                memcpy(&matbuf[off + i * eb], v, eb);
            }
            return off;
        };
        for (size_t i = 0; i < c.gates.size(); ++i) {
            const GateRec &g = c.gates[i];
            AdjGate &a = gs[i];
            std::vector<cd> m = g.m;
            if (g.pindex >= 0) {
                QSIM_TRY(rotation_matrix(g.kind, th[g.pindex], m));
                a.param = true;
                a.P = g.kind == QSIM_GATE_RX ? 0 : g.kind == QSIM_GATE_RY ? 1 : 2;
                a.q = g.targets[0];
                a.pindex = g.pindex;
            }
            a.mfwd = m;
            QSIM_TRY(classify(m, g.targets, g.k, g.controls, g.nc, a.fwd));
            const size_t d = size_t(1) << g.k;
            std::vector<cd> mi(d * d);
            for (size_t r = 0; r < d; ++r)
                for (size_t col = 0; col < d; ++col) mi[col * d + r] = std::conj(m[r * d + col]);
            if (a.param) a.mfwd = mi;  // the reverse sweep needs U^dag
            QSIM_TRY(classify(mi, g.targets, g.k, g.controls, g.nc, a.inv));
            moff_f[i] = stash(a.fwd);
            moff_i[i] = stash(a.inv);
        }
        void *dmats = nullptr;
        if (!matbuf.empty()) {
            QSIM_CUDA_TRY(dev_alloc(&dmats, matbuf.size()), "adjoint matrices");
            QSIM_CUDA_TRY(cudaMemcpyAsync(dmats, matbuf.data(), matbuf.size(), cudaMemcpyHostToDevice, st),
                          "adjoint matrix upload");
            mats.push_back(dmats);
        }
        auto mptr = [&](size_t off) -> void * {
            return off == size_t(-1) ? nullptr : static_cast<char *>(dmats) + off;
        };
        // forward sweep from psi0 (|0> when none is given)
        if (psi0)
            QSIM_CUDA_TRY(cudaMemcpyAsync(psi, psi0, N * sizeof(C), cudaMemcpyDeviceToDevice, st), "adjoint psi0 copy");
        else
            QSIM_TRY(launch_init(psi, n, sizeof(R) == 4 ? QSIM_C64 : QSIM_C128, 0, st));
        const int dtype = sizeof(R) == 4 ? QSIM_C64 : QSIM_C128;
        for (size_t i = 0; i < gs.size(); ++i)
            QSIM_TRY(launch_op(psi, n, dtype, gs[i].fwd, st, mptr(moff_f[i])));
        // lambda = H psi, energy = Re <psi|lambda>
        {
            QSIM_TRY(hplan.run(psi, lam, hp, st));
        }
        double *prow_e = partial + size_t(nrot) * prow;
        {
            LaunchScope ls(K_REDUCE, st, 2.0 * double(N) * sizeof(C));
            k_dot_re<C><<<blocks, 256, 0, st>>>(psi, lam, N, prow_e);
            QSIM_CUDA_TRY(cudaGetLastError(), "energy launch");
        }
        // reverse sweep
        for (size_t ii = gs.size(); ii-- > 0;) {
            const AdjGate &a = gs[ii];
            if (a.param) {
                M2<C> u;
                auto tc = [](const cd &z) {
                    C r;
                    r.x = R(z.real());
                    r.y = R(z.imag());
                    return r;
                };
                u.m00 = tc(a.mfwd[0]);
                u.m01 = tc(a.mfwd[1]);
                u.m10 = tc(a.mfwd[2]);
                u.m11 = tc(a.mfwd[3]);
                LaunchScope ls(K_ADJ_STEP, st, 4.0 * double(N) * sizeof(C));
                k_adj_rot<C><<<blocks, 256, 0, st>>>(psi, lam, N / 2, a.q, a.P, u,
                                                     partial + size_t(rot_of_gate[ii]) * prow);
                QSIM_CUDA_TRY(cudaGetLastError(), "adjoint step launch");
            } else {
                QSIM_TRY(launch_op(psi, n, dtype, a.inv, st, mptr(moff_i[ii])));
                QSIM_TRY(launch_op(lam, n, dtype, a.inv, st, mptr(moff_i[ii])));
            }
        }
        {
            LaunchScope ls(K_REDUCE, st, double(nrot + 1) * prow * 8.0);
            k_rows<<<std::min(nrot + 1, 1024), 256, 0, st>>>(partial, nrot + 1, int(prow), rows);
            QSIM_CUDA_TRY(cudaGetLastError(), "adjoint reduce launch");
        }
        // this path uploads matrices per set and frees them after it: one set
        // at a time
        QSIM_CUDA_TRY(cudaMemcpyAsync(hr.h + size_t(set & 1) * nrow, rows, nrow * sizeof(double),
                                      cudaMemcpyDeviceToHost, st),
                      "adjoint result copy");
        QSIM_CUDA_TRY(cudaEventRecord(hr.ev[set & 1], st), "adjoint event record");
        QSIM_TRY(finish(set));
        for (void *m : mats) cudaFree(m);
        mats.clear();
    }
    return QSIM_OK;
}

// ------------------------------------------------------------------ fused reverse sweep
// complex64, n >= 12: the reverse sweep runs as register-tile stages over both
// states at once (tiles of 2^12 amplitudes, the forward sweep as a staged
// plan).  Each rotation's gradient is a SOP_GRAD op of the stage holding its
// qubit; each warp sums it in fp32 into its own shared-memory slot, the CTA
// adds its warps' sums in double and writes one partial per tile, reduced per
// rotation afterwards.
constexpr int DUAL_W = 3;
// stage kernels compiled for the circuit: 1 always, -1 never, 0 from
// SPECIALIZE_MIN_QUBITS qubits (qsim_adjoint_specialize)
std::atomic<int> g_adj_specialize{0};

struct DualParams {
    stage::StageParams<float2> sp;
    int ngrad, ngradops;
    int gslot[stage::MAX_GRAD];     // gradient term g: global slot,
    int gop[stage::MAX_GRAD];       // the SOP_GRAD op whose sums it combines,
    float gv[stage::MAX_GRAD][3];   // and its Pauli vector
    uint64_t ntiles;
};
static_assert(sizeof(DualParams) <= 32764, "two-state stage parameters exceed the kernel parameter limit");

struct DualSrc {
    const stage::StageParams<float2> &p;
    __device__ const stage::StageOp &op(int o) const { return p.ops[o]; }
    __device__ const stage::Phase &phase(int i) const { return p.phases[i]; }
    __device__ float2 pool(int i) const { return p.pool[i]; }
    __device__ uint64_t aux(int i) const { return p.aux[i]; }
};

template <int W>
__global__ void __launch_bounds__(32 << W) k_adj_stage(float2 *psi, float2 *lam, const __grid_constant__ DualParams dp,
                                                      double *__restrict__ partial) {
    using namespace stage;
    extern __shared__ unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    __shared__ float gw[(3 * MAX_GRAD) << W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int g = threadIdx.x; g < ((3 * dp.ngradops) << W); g += blockDim.x) gw[g] = 0.f;
    __syncthreads();
    const uint64_t tile_base = expand(blockIdx.x, dp.sp.outer);
    int ph = dp.sp.phase0;
    uint64_t base = thread_base<W>(dp.sp.phases[ph], tile_base, lane, warp);
    float2 v[1 << REG_BITS], w[1 << REG_BITS];
    tile_global<float2, W, false>(psi, v, dp.sp.phases[ph], base);
    tile_global<float2, W, false>(lam, w, dp.sp.phases[ph], base);
    const DualSrc src{dp.sp};
    stage_exec2<float2, W>(src, dp.sp.nops, v, w, ph, base, tile_base, tile, lane, warp, gw);
    tile_global<float2, W, true>(psi, v, dp.sp.phases[ph], base);
    tile_global<float2, W, true>(lam, w, dp.sp.phases[ph], base);
    __syncthreads();
    for (int g = threadIdx.x; g < dp.ngrad; g += blockDim.x) {
        const float *s = gw + ((3 * dp.gop[g]) << W);
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < (1 << W); ++i)
            t += double(dp.gv[g][0]) * s[i] + double(dp.gv[g][1]) * s[(1 << W) + i] + double(dp.gv[g][2]) * s[(2 << W) + i];
        partial[uint64_t(dp.gslot[g]) * dp.ntiles + blockIdx.x] = t;
    }
}

// A marker evaluated after a gate h of the reverse sweep, Im<h lam| P |h psi>,
// equals Im<lam| h^dag P h |psi> evaluated before it.  Each marker moves ahead
// of the uncontrolled 1-qubit gates on its qubit that precede it (past other
// markers and gates on other qubits), its operator conjugated by each, so
// that consecutive un-applied rotations on one qubit become adjacent and the
// stage planner merges them into one 2x2 matrix.  A multi-qubit or controlled
// gate on the qubit stops the marker.
void hoist_markers(std::vector<GateRec> &gates) {
    for (size_t i = 0; i < gates.size(); ++i) {
        if (gates[i].grad_slot < 0) continue;
        const int q = gates[i].targets[0];
        cd P[4] = {gates[i].grad_v[2], cd(gates[i].grad_v[0], -gates[i].grad_v[1]),
                   cd(gates[i].grad_v[0], gates[i].grad_v[1]), -gates[i].grad_v[2]};
        size_t dest = i;
        for (size_t j = i; j-- > 0;) {
            const GateRec &h = gates[j];
            if (h.grad_slot >= 0) continue;
            bool on_q = false;
            for (int t = 0; t < h.k; ++t) on_q |= h.targets[t] == q;
            for (int t = 0; t < h.nc; ++t) on_q |= h.controls[t] == q;
            if (!on_q) continue;
            if (h.k != 1 || h.nc != 0) break;
            // P <- h^dag P h
            cd T[4], R[4];
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) T[r * 2 + c] = P[r * 2] * h.m[c] + P[r * 2 + 1] * h.m[2 + c];
            for (int r = 0; r < 2; ++r)
                for (int c = 0; c < 2; ++c) R[r * 2 + c] = std::conj(h.m[r]) * T[c] + std::conj(h.m[2 + r]) * T[2 + c];
            std::copy(R, R + 4, P);
            dest = j;
        }
        if (dest == i) continue;
        GateRec mk = gates[i];
        // P = [[pz, px - i py], [px + i py, -pz]]
        mk.grad_v[0] = P[2].real();
        mk.grad_v[1] = P[2].imag();
        mk.grad_v[2] = P[0].real();
        gates.erase(gates.begin() + long(i));
        gates.insert(gates.begin() + long(dest), mk);
    }
}

int adjoint_fused_c64(const qsim_circuit &c, const void *psi0, int nsets, const double *params, const HParams &hp, double *grads,
                      double *energies, cudaStream_t st) {
    const int n = c.n;
    const uint64_t N = uint64_t(1) << n;
    const int blocks = sm_count_a() * ADJ_BLOCKS_PER_SM;
    const int TB = stage::LANE_BITS + stage::REG_BITS + DUAL_W;
    const uint64_t ntiles = uint64_t(1) << (n - TB);
    std::vector<int> rot_of_gate(c.gates.size(), -1);
    int nrot = 0;
    for (size_t i = 0; i < c.gates.size(); ++i) {
        const GateRec &g = c.gates[i];
        if (g.pindex < 0) continue;
        if (g.nc != 0 || g.k != 1) return set_error(QSIM_EUNSUPPORTED, "trainable rotations must be uncontrolled 1-qubit gates");
        rot_of_gate[i] = nrot++;
    }
    float2 *psi = nullptr, *lam = nullptr;
    double *partial = nullptr, *rows = nullptr, *epart = nullptr;
    cudaError_t e = dev_alloc(&psi, N * sizeof(float2));
    if (e == cudaSuccess) e = dev_alloc(&lam, N * sizeof(float2));
    if (e == cudaSuccess) e = dev_alloc(&partial, std::max<size_t>(1, size_t(nrot) * ntiles) * sizeof(double));
    // two result rows (gradient terms + energy): set k's are read back while
    // set k + 1 runs
    const size_t nrow = size_t(nrot) + 1;
    if (e == cudaSuccess) e = dev_alloc(&rows, 2 * nrow * sizeof(double));
    if (e == cudaSuccess) e = dev_alloc(&epart, size_t(blocks) * sizeof(double));
    struct Guard {
        void *p[5];
        ~Guard() {
            for (void *x : p)
                if (x) cudaFree(x);
        }
    } guard{{psi, lam, partial, rows, epart}};
    if (e != cudaSuccess) return cuda_error(e, "adjoint buffers");
    qsim_state *ps = nullptr;
    QSIM_TRY(qsim_state_create(n, QSIM_C64, psi, st, &ps));
    struct SGuard {
        qsim_state *s;
        ~SGuard() { qsim_state_destroy(s); }
    } sguard{ps};
    // pinned host rows and one event per buffer: the host plans set k + 1
    // while the GPU runs set k, and reads set k's rows when it is done
    struct HostRows {
        double *h = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~HostRows() {
            if (h) cudaFreeHost(h);
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
        }
    } hr;
    QSIM_CUDA_TRY(cudaMallocHost(&hr.h, 2 * nrow * sizeof(double)), "adjoint host rows");
    for (cudaEvent_t &x : hr.ev) QSIM_CUDA_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "adjoint event");
    auto finish = [&](int set) -> int {
        const int b = set & 1;
        QSIM_CUDA_TRY(cudaEventSynchronize(hr.ev[b]), "adjoint sync");
        const double *row = hr.h + size_t(b) * nrow;
        double *gset = grads + size_t(set) * size_t(c.nparams);
        for (int p = 0; p < c.nparams; ++p) gset[p] = 0.0;
        for (size_t i = 0; i < c.gates.size(); ++i)
            if (rot_of_gate[i] >= 0) gset[c.gates[i].pindex] += row[rot_of_gate[i]];
        if (energies) energies[set] = row[nrot];
        return QSIM_OK;
    };
    const size_t smem = (size_t(1) << TB) * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        QSIM_CUDA_TRY(cudaFuncSetAttribute(k_adj_stage<DUAL_W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                      "adjoint stage smem");
        attr = true;
    }
    HPlan<float2> hplan;
    QSIM_TRY(hplan.build(hp, n, st));
    for (int set = 0; set < nsets; ++set) {
        const double *th = params + size_t(set) * size_t(c.nparams);
        // forward circuit with this set's angles, and the reverse sweep:
        // gates un-applied last to first, a gradient marker before each rotation
        qsim_circuit fwd, bwd;
        fwd.n = bwd.n = n;
        fwd.gates = c.gates;
        for (size_t i = 0; i < fwd.gates.size(); ++i)
            if (fwd.gates[i].pindex >= 0) QSIM_TRY(rotation_matrix(fwd.gates[i].kind, th[fwd.gates[i].pindex], fwd.gates[i].m));
        for (size_t ii = fwd.gates.size(); ii-- > 0;) {
            const GateRec &g = fwd.gates[ii];
            if (rot_of_gate[ii] >= 0) {
                GateRec mk;
                mk.kind = QSIM_GATE_MATRIX;
                mk.k = 1;
                mk.targets[0] = g.targets[0];
                mk.m = {1.0, 0.0, 0.0, 1.0};
                mk.grad_slot = rot_of_gate[ii];
                mk.grad_v[g.kind == QSIM_GATE_RX ? 0 : g.kind == QSIM_GATE_RY ? 1 : 2] = 1.0;
                bwd.gates.push_back(mk);
            }
            GateRec inv = g;
            inv.kind = QSIM_GATE_MATRIX;
            inv.pindex = -1;
            const size_t d = size_t(1) << g.k;
            for (size_t r = 0; r < d; ++r)
                for (size_t col = 0; col < d; ++col) inv.m[col * d + r] = std::conj(g.m[r * d + col]);
            bwd.gates.push_back(inv);
        }
        hoist_markers(bwd.gates);
        // forward sweep (staged plan) from |0>
        qsim_plan *fp = nullptr;
        const bool spec = g_adj_specialize > 0 || (g_adj_specialize == 0 && n >= SPECIALIZE_MIN_QUBITS);
        QSIM_TRY(qsim_plan_build(&fwd, DUAL_W, QSIM_FUSE_STAGED | (spec ? QSIM_PLAN_SPECIALIZE : 0), &fp));
        struct PGuard {
            qsim_plan *p;
            ~PGuard() { qsim_plan_destroy(p); }
        } pguard{fp};
        if (psi0)
            QSIM_CUDA_TRY(cudaMemcpyAsync(psi, psi0, N * sizeof(float2), cudaMemcpyDeviceToDevice, st),
                          "adjoint psi0 copy");
        else
            QSIM_TRY(launch_init(psi, n, QSIM_C64, 0, st));
        QSIM_TRY(qsim_apply_fused(ps, fp));
        {
            QSIM_TRY(hplan.run(psi, lam, hp, st));
        }
        {
            LaunchScope ls(K_REDUCE, st, 2.0 * double(N) * sizeof(float2));
            k_dot_re<float2><<<blocks, 256, 0, st>>>(psi, lam, N, epart);
            QSIM_CUDA_TRY(cudaGetLastError(), "energy launch");
        }
        // reverse sweep as two-state stages
        std::vector<stage::Stage> stages;
        QSIM_TRY(stage::plan_stage_list(bwd, DUAL_W, true, stages));
        DualSpec dspec;
        if (spec) QSIM_TRY(spec_dual_prepare(stages, n, DUAL_W, dspec));
        for (size_t si = 0; si < stages.size(); ++si) {
            const stage::Stage &sg = stages[si];
            if (sg.plain) {
                if (sg.op.type == Op::DENSE && sg.op.k >= 2)
                    return set_error(QSIM_EUNSUPPORTED, "adjoint: gates of more than 2 targets");
                QSIM_TRY(launch_op(psi, n, QSIM_C64, sg.op, st, nullptr));
                QSIM_TRY(launch_op(lam, n, QSIM_C64, sg.op, st, nullptr));
                continue;
            }
            if (spec) {
                LaunchScope ls(K_ADJ_STEP, st, 4.0 * double(N) * sizeof(float2),
                               (2.0 * stage::stage_exec_flops_per_amp(sg) + 12.0 * sg.ngradops) * double(N));
                QSIM_TRY(spec_dual_launch(dspec, sg, si, psi, lam, partial, n, DUAL_W, st));
                continue;
            }
            DualParams dp;
            memset(&dp, 0, sizeof dp);
            stage::make_params<float2>(sg, dp.sp);
            dp.ngrad = int(sg.grads.size());
            dp.ngradops = sg.ngradops;
            for (int g = 0; g < dp.ngrad; ++g) {
                dp.gslot[g] = sg.grads[g].slot;
                dp.gop[g] = sg.grads[g].op;
                for (int c = 0; c < 3; ++c) dp.gv[g][c] = float(sg.grads[g].v[c]);
            }
            dp.ntiles = ntiles;
            // useful flops: the stage's gates on both states, 6 FMAs per
            // amplitude for each gradient op's three sums
            LaunchScope ls(K_ADJ_STEP, st, 4.0 * double(N) * sizeof(float2),
                           (2.0 * stage::stage_exec_flops_per_amp(sg) + 12.0 * sg.ngradops) * double(N));
            k_adj_stage<DUAL_W><<<unsigned(ntiles), 32 << DUAL_W, smem, st>>>(psi, lam, dp, partial);
            QSIM_CUDA_TRY(cudaGetLastError(), "adjoint stage launch");
        }
        {
            double *row = rows + size_t(set & 1) * nrow;
            LaunchScope ls(K_REDUCE, st, double(nrot) * ntiles * 8.0);
            if (nrot) k_rows<<<std::min(nrot, 1024), 256, 0, st>>>(partial, nrot, int(ntiles), row);
            k_rows<<<1, 256, 0, st>>>(epart, 1, blocks, row + nrot);
            QSIM_CUDA_TRY(cudaGetLastError(), "adjoint reduce launch");
            QSIM_CUDA_TRY(cudaMemcpyAsync(hr.h + size_t(set & 1) * nrow, row, nrow * sizeof(double),
                                          cudaMemcpyDeviceToHost, st),
                          "adjoint result copy");
            QSIM_CUDA_TRY(cudaEventRecord(hr.ev[set & 1], st), "adjoint event record");
        }
        if (set > 0) QSIM_TRY(finish(set - 1));
    }
    QSIM_TRY(finish(nsets - 1));
    return QSIM_OK;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" int qsim_adjoint_grad(const qsim_circuit *c, const qsim_state *psi0, int dtype, int nsets,
                                 const double *params, int nterms, const uint64_t *xmask, const uint64_t *zmask,
                                 const double *coeff, double *grads, double *energies, void *cuda_stream) {
    if (!c || !grads || nsets < 1 || (c->nparams > 0 && !params)) return set_error(QSIM_EINVAL, "bad arguments");
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return set_error(QSIM_EINVAL, "bad dtype");
    if (psi0 && (psi0->n != c->n || psi0->dtype != dtype || !psi0->amps))
        return set_error(QSIM_EINVAL, "psi0 must be a state of the circuit's width (%d) in the requested precision",
                         c->n);
    if (c->n > 34) return set_error(QSIM_EINVAL, "the adjoint method needs a state of at most 34 qubits");
    if (nterms < 1 || !xmask || !zmask || !coeff) return set_error(QSIM_EINVAL, "empty Hamiltonian");
    const uint64_t full = (uint64_t(1) << c->n) - 1;
    HParams hp;
    memset(&hp, 0, sizeof hp);
    std::vector<bool> done(nterms, false);
    int nt = 0;
    for (int t0 = 0; t0 < nterms; ++t0) {
        if (done[t0]) continue;
        if ((xmask[t0] | zmask[t0]) & ~full) return set_error(QSIM_EINVAL, "term %d acts outside the state", t0);
        if (hp.ngroups >= HAPPLY_GROUPS) return set_error(QSIM_EUNSUPPORTED, "more than %d distinct X masks", HAPPLY_GROUPS);
        hp.X[hp.ngroups] = xmask[t0];
        hp.t0[hp.ngroups] = nt;
        for (int t = t0; t < nterms; ++t) {
            if (done[t] || xmask[t] != xmask[t0]) continue;
            if (nt >= HAPPLY_TERMS) return set_error(QSIM_EUNSUPPORTED, "more than %d Pauli terms", HAPPLY_TERMS);
            done[t] = true;
            const int ny = __builtin_popcountll(xmask[t] & zmask[t]);
            const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
            hp.Z[nt] = zmask[t];
            hp.cr[nt] = coeff[t] * re[ny & 3];
            hp.ci[nt] = coeff[t] * im[ny & 3];
            hp.fr[nt] = float(hp.cr[nt]);
            hp.fi[nt] = float(hp.ci[nt]);
            ++nt;
        }
        ++hp.ngroups;
        hp.t0[hp.ngroups] = nt;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const void *a0 = psi0 ? psi0->amps : nullptr;
    if (psi0 && psi0->stream != st)  // the start state's pending work comes first
        QSIM_CUDA_TRY(cudaStreamSynchronize(psi0->stream), "psi0 stream sync");
    // complex64 from 12 qubits: register-tile stages over both states;
    // otherwise one sweep per gate
    if (dtype == QSIM_C64 && c->n >= stage::LANE_BITS + stage::REG_BITS + DUAL_W)
        return adjoint_fused_c64(*c, a0, nsets, params, hp, grads, energies, st);
    return dtype == QSIM_C64 ? adjoint_t<float>(*c, a0, nsets, params, hp, grads, energies, st)
                             : adjoint_t<double>(*c, a0, nsets, params, hp, grads, energies, st);
}

extern "C" QSIM_API int qsim_adjoint_specialize(int mode, int *previous) {
    if (mode < -1 || mode > 1) return set_error(QSIM_EINVAL, "mode must be -1, 0 or 1");
    const int old = qsim::g_adj_specialize.exchange(mode);
    if (previous) *previous = old;
    return QSIM_OK;
}

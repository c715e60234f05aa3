// Plain gate sweeps: one HBM pass per gate, in place (Eq. (1); Sec. 2).
//
// Every kernel enumerates a compact index g over the amplitudes it must touch
// and expands it to an amplitude index by inserting zero bits at the target
// positions and one bits at the control positions (the index arithmetic of
// the single-qubit listing of Sec. 2, generalised to several bits).
// Consecutive threads take consecutive g, so each of a thread's loads is
// coalesced across the warp for every target, high or low: the 2^k partner
// amplitudes of a group form 2^k separate contiguous streams.
#include <cuComplex.h>

#include "internal.h"

namespace qsim {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

__device__ __forceinline__ uint64_t expand_index(uint64_t g, const IndexMap &m) {
#pragma unroll 1
    for (int i = 0; i < m.nins; ++i) {
        const uint64_t low = g & ((uint64_t(1) << m.ins[i]) - 1);
        g = ((g ^ low) << 1) | low;
    }
    return g | m.set;
}

// ------------------------------------------------------------------ init
template <typename C>
__global__ void k_init(C *psi, uint64_t N, uint64_t basis) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        C v;
        v.x = (i == basis) ? 1 : 0;
        v.y = 0;
        psi[i] = v;
    }
}

static int sm_count() { return device_sm_count(); }

int launch_init(void *psi, int n, int dtype, uint64_t basis, cudaStream_t st) {
    const uint64_t N = uint64_t(1) << n;
    const double bytes = double(N) * (dtype == QSIM_C64 ? 8 : 16);
    const int threads = 512;
    const uint64_t want = (N + threads - 1) / threads;
    const int blocks = int(std::min<uint64_t>(want, uint64_t(sm_count()) * 8));
    LaunchScope ls(K_INIT, st, bytes);
    if (dtype == QSIM_C64)
        k_init<<<blocks, threads, 0, st>>>(static_cast<float2 *>(psi), N, basis);
    else
        k_init<<<blocks, threads, 0, st>>>(static_cast<double2 *>(psi), N, basis);
    QSIM_CUDA_TRY(cudaGetLastError(), "init launch");
    return QSIM_OK;
}

// ------------------------------------------------------------------ dense 1q
template <typename R> struct Mat2 {
    typename CT<R>::T m00, m01, m10, m11;
};

// Each thread updates PER pairs (i1, i1 + 2^t): the in-place 2x2 update of
// the single-qubit listing, Sec. 2, with controls folded into the index map.
template <typename R, int PER>
__global__ void __launch_bounds__(256) k_dense1(typename CT<R>::T *__restrict__ psi, uint64_t npairs,
                                                const __grid_constant__ IndexMap map, uint64_t stride, Mat2<R> m) {
    using C = typename CT<R>::T;
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    C a[PER], b[PER];
    uint64_t idx[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        idx[j] = g < npairs ? expand_index(g, map) : ~uint64_t(0);
        if (g < npairs) {
            a[j] = psi[idx[j]];
            b[j] = psi[idx[j] + stride];
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
        C o0 = cmul(m.m00, a[j]);
        o0 = cfma(m.m01, b[j], o0);
        C o1 = cmul(m.m10, a[j]);
        o1 = cfma(m.m11, b[j], o1);
        psi[idx[j]] = o0;
        psi[idx[j] + stride] = o1;
    }
}

// ------------------------------------------------------------------ dense k = 2, 3
// Register form for small blocks: each thread loads PER whole groups (2^K
// amplitudes each at the target offsets), multiplies by G held in kernel
// parameters and stores them back (Eq. (1) over the 2^K target values).
template <typename R, int K> struct SmallDense {
    typename CT<R>::T m[1 << (2 * K)];
    uint64_t off[1 << K];
};

template <typename R, int K, int PER>
__global__ void __launch_bounds__(256) k_dense_small(typename CT<R>::T *__restrict__ psi, uint64_t ngroups,
                                                     const __grid_constant__ IndexMap map, const __grid_constant__ SmallDense<R, K> G) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    C v[PER][D];
    uint64_t idx[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        idx[j] = g < ngroups ? expand_index(g, map) : ~uint64_t(0);
        if (g < ngroups) {
#pragma unroll
            for (int r = 0; r < D; ++r) v[j][r] = psi[idx[j] | G.off[r]];
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            C acc = cmul(G.m[r * D], v[j][0]);
#pragma unroll
            for (int c = 1; c < D; ++c) acc = cfma(G.m[r * D + c], v[j][c], acc);
            psi[idx[j] | G.off[r]] = acc;
        }
    }
}

// ------------------------------------------------------------------ dense k = 4..6
// Register form for wide blocks: the matrix is staged once per CTA in shared
// memory (every thread reads the same element: a broadcast); each thread
// loads a whole group of 2^K amplitudes into registers, then forms and stores
// the outputs one row at a time (two accumulators per row for ILP).
template <typename R, int K>
__global__ void __launch_bounds__(128) k_dense_big(typename CT<R>::T *__restrict__ psi, uint64_t ngroups,
                                                   const __grid_constant__ IndexMap map,
                                                   const typename CT<R>::T *__restrict__ mat,
                                                   const __grid_constant__ Offsets offs) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    extern __shared__ unsigned char dense_smem[];
    C *gm = reinterpret_cast<C *>(dense_smem);
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) gm[i] = mat[i];
    __syncthreads();
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        const uint64_t x = expand_index(g, map);
        C v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = psi[x | offs.o[c]];
#pragma unroll 1
        for (int r = 0; r < D; ++r) {
            const C *row = gm + r * D;
            C a0 = cmul(row[0], v[0]), a1 = cmul(row[1], v[1]);
#pragma unroll
            for (int c = 2; c < D; c += 2) {
                a0 = cfma(row[c], v[c], a0);
                a1 = cfma(row[c + 1], v[c + 1], a1);
            }
            a0.x += a1.x;
            a0.y += a1.y;
            psi[x | offs.o[r]] = a0;
        }
    }
}

// ------------------------------------------------------------------ dense k
// CTA stages GPB groups of 2^K amplitudes in shared memory (coalesced loads:
// consecutive threads take consecutive groups for the same matrix column),
// then each thread produces outputs (group, row) = sum_j G[row, j] v[group, j].
template <typename R, int K, int GPB>
__global__ void __launch_bounds__(256) k_densek(typename CT<R>::T *__restrict__ psi, uint64_t ngroups,
                                                const __grid_constant__ IndexMap map, const typename CT<R>::T *__restrict__ mat,
                                                Offsets offs) {
    using C = typename CT<R>::T;
    constexpr int D = 1 << K;
    __shared__ C v[GPB][D + 1];
    const uint64_t g0 = uint64_t(blockIdx.x) * GPB;
    for (int i = threadIdx.x; i < GPB * D; i += blockDim.x) {
        const int gl = i % GPB, j = i / GPB;
        const uint64_t g = g0 + gl;
        if (g < ngroups) v[gl][j] = psi[expand_index(g, map) | offs.o[j]];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < GPB * D; i += blockDim.x) {
        const int gl = i % GPB, r = i / GPB;
        const uint64_t g = g0 + gl;
        if (g >= ngroups) continue;
        C acc;
        acc.x = 0;
        acc.y = 0;
        const C *row = mat + r * D;
#pragma unroll 8
        for (int j = 0; j < D; ++j) acc = cfma(__ldg(&row[j]), v[gl][j], acc);
        psi[expand_index(g, map) | offs.o[r]] = acc;
    }
}

// ------------------------------------------------------------------ diagonal
// psi[x] *= d[j(x)] over the amplitudes whose control bits are 1; j(x) reads
// the target bits (targets[0] = MSB).  k = 0 is a phase on the control subspace.
template <typename R> struct DiagParams {
    int k;
    int tbits[QSIM_MAX_TARGETS];
    typename CT<R>::T d[1 << QSIM_MAX_TARGETS];
};

template <typename R, int PER>
__global__ void __launch_bounds__(256) k_diag(typename CT<R>::T *__restrict__ psi, uint64_t count,
                                              const __grid_constant__ IndexMap map, const __grid_constant__ DiagParams<R> p) {
    using C = typename CT<R>::T;
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    C a[PER];
    uint64_t idx[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        idx[j] = g < count ? expand_index(g, map) : ~uint64_t(0);
        if (g < count) a[j] = psi[idx[j]];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
        int sel = 0;
        for (int i = 0; i < p.k; ++i) sel = (sel << 1) | int((idx[j] >> p.tbits[i]) & 1);
        psi[idx[j]] = cmul(p.d[sel], a[j]);
    }
}

// ------------------------------------------------------------------ monomial
// Permutation with phases (X, Y, SWAP, ...): only the rows that change are
// loaded and stored: out[dst_a] = ph_a * in[src_a].
template <typename R> struct MonoParams {
    int na;
    uint64_t dst[8];
    uint64_t src[8];
    typename CT<R>::T ph[8];
};

// NA rows move per group; each thread takes PER groups (loads first, then
// stores) so that several loads per thread are in flight.
template <typename R, int NA, int PER>
__global__ void __launch_bounds__(256) k_mono(typename CT<R>::T *__restrict__ psi, uint64_t ngroups,
                                              const __grid_constant__ IndexMap map,
                                              const __grid_constant__ MonoParams<R> p) {
    using C = typename CT<R>::T;
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    C v[PER][NA];
    uint64_t x[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        x[j] = g < ngroups ? expand_index(g, map) : ~uint64_t(0);
        if (g < ngroups) {
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < p.na) v[j][a] = psi[x[j] | p.src[a]];
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (x[j] == ~uint64_t(0)) continue;
#pragma unroll
        for (int a = 0; a < NA; ++a)
            if (a < p.na) psi[x[j] | p.dst[a]] = cmul(p.ph[a], v[j][a]);
    }
}

// ------------------------------------------------------------------ dispatch
template <typename R> static typename CT<R>::T to_c(const cd &z) {
    typename CT<R>::T r;
    r.x = R(z.real());
    r.y = R(z.imag());
    return r;
}

static uint64_t target_offset(int j, const int *targets, int k) {
    uint64_t off = 0;
    for (int i = 0; i < k; ++i)
        if ((j >> (k - 1 - i)) & 1) off |= uint64_t(1) << targets[i];
    return off;
}

template <typename R>
static int launch_op_t(void *psi_v, int n, const Op &op, cudaStream_t st, void *mat_dev) {
    using C = typename CT<R>::T;
    C *psi = static_cast<C *>(psi_v);
    const double S = sizeof(C);
    const int k = op.k, c = op.c;
    switch (op.type) {
        case Op::IDENTITY:
            return QSIM_OK;
        case Op::DENSE: {
            const IndexMap map = make_index_map(op.targets, k, op.controls, c);
            const uint64_t ngroups = uint64_t(1) << (n - k - c);
            const double bytes = 2.0 * S * double(ngroups << k);
            if (k == 1) {
                Mat2<R> m{to_c<R>(op.m[0]), to_c<R>(op.m[1]), to_c<R>(op.m[2]), to_c<R>(op.m[3])};
                constexpr int PER = 4, T = 256;
                const uint64_t blocks = (ngroups + T * PER - 1) / (T * PER);
                LaunchScope ls(K_DENSE1, st, bytes, 16.0 * double(ngroups << 1));
                k_dense1<R, PER><<<unsigned(blocks), T, 0, st>>>(psi, ngroups, map,
                                                                  uint64_t(1) << op.targets[0], m);
            } else if (k <= 3) {
                constexpr int T = 256;
                const double flops = 8.0 * double(1 << k) * double(ngroups << k);
                LaunchScope ls(K_DENSEK, st, bytes, flops);
                if (k == 2) {
                    SmallDense<R, 2> G{};
                    for (int e = 0; e < 16; ++e) G.m[e] = to_c<R>(op.m[size_t(e)]);
                    for (int j = 0; j < 4; ++j) G.off[j] = target_offset(j, op.targets, k);
                    constexpr int PER = 2;
                    k_dense_small<R, 2, PER><<<unsigned((ngroups + T * PER - 1) / (T * PER)), T, 0, st>>>(psi, ngroups,
                                                                                                         map, G);
                } else {
                    SmallDense<R, 3> G{};
                    for (int e = 0; e < 64; ++e) G.m[e] = to_c<R>(op.m[size_t(e)]);
                    for (int j = 0; j < 8; ++j) G.off[j] = target_offset(j, op.targets, k);
                    k_dense_small<R, 3, 1><<<unsigned((ngroups + T - 1) / T), T, 0, st>>>(psi, ngroups, map, G);
                }
            } else if (k <= (sizeof(R) == 4 ? 6 : 5)) {
                if (!mat_dev) return set_error(QSIM_EINVAL, "dense k>3 needs the matrix on the device");
                Offsets offs{};
                for (int j = 0; j < (1 << k); ++j) offs.o[j] = target_offset(j, op.targets, k);
                const C *mat = static_cast<const C *>(mat_dev);
                const size_t smem = (size_t(1) << (2 * k)) * sizeof(C);
                const int T = 128;
                const uint64_t want = (ngroups + T - 1) / T;
                const unsigned blocks = unsigned(std::min<uint64_t>(want, uint64_t(sm_count()) * 8));
                LaunchScope ls(K_DENSEK, st, bytes, 8.0 * double(1 << k) * double(ngroups << k));
                auto launch = [&](auto kern) -> int {
                    static bool attr[7] = {};
                    if (!attr[k]) {
                        QSIM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                                      "dense smem attribute");
                        attr[k] = true;
                    }
                    kern<<<blocks, T, smem, st>>>(psi, ngroups, map, mat, offs);
                    return QSIM_OK;
                };
                if (k == 4) QSIM_TRY(launch(k_dense_big<R, 4>));
                else if (k == 5) QSIM_TRY(launch(k_dense_big<R, 5>));
                else QSIM_TRY(launch(k_dense_big<R, (sizeof(R) == 4 ? 6 : 5)>));
            } else {
                if (!mat_dev) return set_error(QSIM_EINVAL, "dense k>1 needs the matrix on the device");
                Offsets offs{};
                for (int j = 0; j < (1 << k); ++j) offs.o[j] = target_offset(j, op.targets, k);
                const C *mat = static_cast<const C *>(mat_dev);
                constexpr int GPB = 32;
                const uint64_t blocks = (ngroups + GPB - 1) / GPB;
                LaunchScope ls(K_DENSEK, st, bytes, 8.0 * double(1 << k) * double(ngroups << k));
                switch (k) {
                    case 2: k_densek<R, 2, GPB><<<unsigned(blocks), 128, 0, st>>>(psi, ngroups, map, mat, offs); break;
                    case 3: k_densek<R, 3, GPB><<<unsigned(blocks), 256, 0, st>>>(psi, ngroups, map, mat, offs); break;
                    case 4: k_densek<R, 4, GPB><<<unsigned(blocks), 256, 0, st>>>(psi, ngroups, map, mat, offs); break;
                    case 5: k_densek<R, 5, GPB><<<unsigned(blocks), 256, 0, st>>>(psi, ngroups, map, mat, offs); break;
                    case 6: k_densek<R, 6, 16><<<unsigned((ngroups + 15) / 16), 256, 0, st>>>(psi, ngroups, map, mat, offs); break;
                    default: return set_error(QSIM_EINVAL, "dense k=%d unsupported", k);
                }
            }
            break;
        }
        case Op::DIAG: {
            const IndexMap map = make_index_map(nullptr, 0, op.controls, c);
            const uint64_t count = uint64_t(1) << (n - c);
            DiagParams<R> p{};
            p.k = k;
            for (int i = 0; i < k; ++i) p.tbits[i] = op.targets[i];
            for (int j = 0; j < (1 << k); ++j) p.d[j] = to_c<R>(op.m[j]);
            constexpr int PER = 4, T = 256;
            const uint64_t blocks = (count + T * PER - 1) / (T * PER);
            LaunchScope ls(K_DIAG, st, 2.0 * S * double(count), 6.0 * double(count));
            k_diag<R, PER><<<unsigned(blocks), T, 0, st>>>(psi, count, map, p);
            break;
        }
        case Op::MONO: {
            const IndexMap map = make_index_map(op.targets, k, op.controls, c);
            const uint64_t ngroups = uint64_t(1) << (n - k - c);
            MonoParams<R> p{};
            for (int r = 0; r < (1 << k); ++r) {
                if (op.perm[r] == r && op.phase[r] == cd(1.0)) continue;
                p.dst[p.na] = target_offset(r, op.targets, k);
                p.src[p.na] = target_offset(op.perm[r], op.targets, k);
                p.ph[p.na] = to_c<R>(op.phase[r]);
                ++p.na;
            }
            const int T = 256;
            LaunchScope ls(K_MONO, st, 2.0 * S * double(ngroups) * p.na);
            if (p.na <= 2) {
                constexpr int PER = 4;
                k_mono<R, 2, PER><<<unsigned((ngroups + T * PER - 1) / (T * PER)), T, 0, st>>>(psi, ngroups, map, p);
            } else {
                k_mono<R, 8, 1><<<unsigned((ngroups + T - 1) / T), T, 0, st>>>(psi, ngroups, map, p);
            }
            break;
        }
    }
    QSIM_CUDA_TRY(cudaGetLastError(), "sweep launch");
    return QSIM_OK;
}

int launch_op(void *psi, int n, int dtype, const Op &op, cudaStream_t st, void *mat_dev) {
    if (n - op.k - op.c < 0) return set_error(QSIM_EINVAL, "gate wider than the state");
    if ((uint64_t(1) << (n - op.k - op.c)) / 256 >= (uint64_t(1) << 31))
        return set_error(QSIM_EUNSUPPORTED, "state too large for one launch");
    return dtype == QSIM_C64 ? launch_op_t<float>(psi, n, op, st, mat_dev)
                             : launch_op_t<double>(psi, n, op, st, mat_dev);
}

}  // namespace qsim

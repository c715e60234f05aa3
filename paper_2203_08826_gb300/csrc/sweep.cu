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

#include "dfloat.cuh"
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

#ifdef QSIM_DEBUG
static __device__ unsigned long long g_sweep_oob;
#endif

// True when index x (the largest a group will touch) lies inside the state; in
// a QSIM_DEBUG build an index outside is counted and its group skipped, in a
// release build nothing is checked.
__device__ __forceinline__ bool in_state(uint64_t x, const IndexMap &m) {
#ifdef QSIM_DEBUG
    if (m.limit && x >= m.limit) {
        atomicAdd(&g_sweep_oob, 1ull);
        return false;
    }
#endif
    return true;
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
        if (g < npairs && !in_state(idx[j] + stride, map)) idx[j] = ~uint64_t(0);
        if (idx[j] != ~uint64_t(0)) {
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

// Complex128 form of the same update, mostly on the FP32 pipes: each double
// of a and b is split into a float pair, the four outputs are compensated dot
// products (double-float, about 48 bits), and the results are rounded back
// to doubles.  A pair with an element outside the float pair's range takes
// the FP64 formula instead (a warp-divergent branch that exact or near-zero
// amplitudes never take; zero is in range), and so do the pairs of the first
// DF_FP64_WARPS warps of each CTA, which keeps the FP64 pipe busy alongside.
// Warps 0 .. DF_FP64_WARPS - 1 of every 8 compute their pairs in FP64, the
// others in double-float: the FP64 pipe and the FP32/integer pipes then work
// side by side.  Measured on the 30-qubit random circuit (dense 1-qubit
// sweeps, complex128): 0 -> 7.98 ms, 2 -> 6.63 ms, 3 -> 6.22 ms (5.5 TB/s),
// 4 -> 8.19 ms per sweep (the FP64 pipe becomes the limit).
constexpr int DF_FP64_WARPS = 3;

struct DfMat2 {
    float v[16];  // m00, m01, m10, m11: (re.hi, re.lo, im.hi, im.lo)
};

// y = mA * a + mB * b (complex), every part a float pair
__device__ __forceinline__ void df_row(const float *mA, const float *mB, const float (&a)[4], const float (&b)[4],
                                       double &yr, double &yi) {
    // a = (re.hi, re.lo, im.hi, im.lo)
    dfl::Dot re, im;
    re.first(mA[0], mA[1], a[0], a[1]);
    re.add(-mA[2], -mA[3], a[2], a[3]);
    re.add(mB[0], mB[1], b[0], b[1]);
    re.add(-mB[2], -mB[3], b[2], b[3]);
    im.first(mA[0], mA[1], a[2], a[3]);
    im.add(mA[2], mA[3], a[0], a[1]);
    im.add(mB[0], mB[1], b[2], b[3]);
    im.add(mB[2], mB[3], b[0], b[1]);
    float h, l;
    re.result(h, l);
    yr = dfl::join(h, l);
    im.result(h, l);
    yi = dfl::join(h, l);
}

template <int PER>
__global__ void __launch_bounds__(256) k_dense1_df(double2 *__restrict__ psi, uint64_t npairs,
                                                   const __grid_constant__ IndexMap map, uint64_t stride,
                                                   const __grid_constant__ DfMat2 m, Mat2<double> md, int fp64_warps) {
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    const bool use64 = int(threadIdx.x >> 5) < fp64_warps;  // warp-uniform
    double2 a[PER], b[PER];
    uint64_t idx[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        idx[j] = g < npairs ? expand_index(g, map) : ~uint64_t(0);
        if (g < npairs && !in_state(idx[j] + stride, map)) idx[j] = ~uint64_t(0);
        if (idx[j] != ~uint64_t(0)) {
            a[j] = psi[idx[j]];
            b[j] = psi[idx[j] + stride];
        }
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
        float fa[4], fb[4];
        bool ok = !use64;
        if (ok) {
            ok &= dfl::split(a[j].x, fa[0], fa[1]);
            ok &= dfl::split(a[j].y, fa[2], fa[3]);
            ok &= dfl::split(b[j].x, fb[0], fb[1]);
            ok &= dfl::split(b[j].y, fb[2], fb[3]);
        }
        double2 o0, o1;
        if (ok) {
            df_row(m.v + 0, m.v + 4, fa, fb, o0.x, o0.y);
            df_row(m.v + 8, m.v + 12, fa, fb, o1.x, o1.y);
        } else {
            o0 = cfma(md.m01, b[j], cmul(md.m00, a[j]));
            o1 = cfma(md.m11, b[j], cmul(md.m10, a[j]));
        }
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
        if (g < ngroups && !in_state(idx[j] | G.off[D - 1], map)) idx[j] = ~uint64_t(0);
        if (idx[j] != ~uint64_t(0)) {
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
        if (!in_state(x | offs.o[D - 1], map)) continue;
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
        if (g < ngroups && in_state(expand_index(g, map) | offs.o[D - 1], map))
            v[gl][j] = psi[expand_index(g, map) | offs.o[j]];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < GPB * D; i += blockDim.x) {
        const int gl = i % GPB, r = i / GPB;
        const uint64_t g = g0 + gl;
        if (g >= ngroups || !in_state(expand_index(g, map) | offs.o[D - 1], map)) continue;
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
        if (g < count && !in_state(idx[j], map)) idx[j] = ~uint64_t(0);
        if (idx[j] != ~uint64_t(0)) a[j] = psi[idx[j]];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
        int sel = 0;
        for (int i = 0; i < p.k; ++i) sel = (sel << 1) | int((idx[j] >> p.tbits[i]) & 1);
        psi[idx[j]] = cmul(p.d[sel], a[j]);
    }
}

// Complex128 diagonal on the FP32 pipes: psi[x] *= d[j(x)] as a
// double-float product (two compensated two-term dot products per
// amplitude), FP64 for an amplitude outside the float pair's range.
template <int PER>
__global__ void __launch_bounds__(256) k_diag_df(double2 *__restrict__ psi, uint64_t count,
                                                 const __grid_constant__ IndexMap map,
                                                 const __grid_constant__ DiagParams<double> p) {
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    double2 a[PER];
    uint64_t idx[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        idx[j] = g < count ? expand_index(g, map) : ~uint64_t(0);
        if (g < count && !in_state(idx[j], map)) idx[j] = ~uint64_t(0);
        if (idx[j] != ~uint64_t(0)) a[j] = psi[idx[j]];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
        int sel = 0;
        for (int i = 0; i < p.k; ++i) sel = (sel << 1) | int((idx[j] >> p.tbits[i]) & 1);
        const double2 d = p.d[sel];
        float x[4], dd[4];
        bool ok = dfl::split(a[j].x, x[0], x[1]);
        ok &= dfl::split(a[j].y, x[2], x[3]);
        ok &= dfl::split(d.x, dd[0], dd[1]);
        ok &= dfl::split(d.y, dd[2], dd[3]);
        double2 o;
        if (ok) {
            dfl::Dot re, im;
            re.first(dd[0], dd[1], x[0], x[1]);
            re.add(-dd[2], -dd[3], x[2], x[3]);
            im.first(dd[0], dd[1], x[2], x[3]);
            im.add(dd[2], dd[3], x[0], x[1]);
            float h, l;
            re.result(h, l);
            o.x = dfl::join(h, l);
            im.result(h, l);
            o.y = dfl::join(h, l);
        } else {
            o = cmul(d, a[j]);
        }
        psi[idx[j]] = o;
    }
}

// Diagonal whose entries are all +1 or -1 (CZ, Z, controlled Z): the sign
// bits of the selected amplitudes flip; no arithmetic, exact in any precision.
template <typename R, int PER>
__global__ void __launch_bounds__(256) k_diag_sign(typename CT<R>::T *__restrict__ psi, uint64_t count,
                                                   const __grid_constant__ IndexMap map, int k, uint64_t neg_table, int nt0, int nt1, int nt2, int nt3, int nt4,
                                                   int nt5) {
    using C = typename CT<R>::T;
    const int tb[6] = {nt0, nt1, nt2, nt3, nt4, nt5};
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
    C a[PER];
    uint64_t idx[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t g = base + uint64_t(j) * blockDim.x;
        idx[j] = g < count ? expand_index(g, map) : ~uint64_t(0);
        if (g < count && !in_state(idx[j], map)) idx[j] = ~uint64_t(0);
        if (idx[j] != ~uint64_t(0)) a[j] = psi[idx[j]];
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        if (idx[j] == ~uint64_t(0)) continue;
        int sel = 0;
        for (int i = 0; i < k; ++i) sel = (sel << 1) | int((idx[j] >> tb[i]) & 1);
        if ((neg_table >> sel) & 1) {
            a[j].x = -a[j].x;
            a[j].y = -a[j].y;
            psi[idx[j]] = a[j];
        }
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
// UNIT: every phase is exactly 1 (X, SWAP, CNOT): a pure move, no arithmetic.
template <typename R, int NA, int PER, bool UNIT>
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
            bool ok = true;
#pragma unroll
            for (int a = 0; a < NA; ++a)
                if (a < p.na) ok = ok && in_state(x[j] | p.src[a] | p.dst[a], map);
            if (!ok) x[j] = ~uint64_t(0);
        }
        if (x[j] != ~uint64_t(0)) {
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
            if (a < p.na) psi[x[j] | p.dst[a]] = UNIT ? v[j][a] : cmul(p.ph[a], v[j][a]);
    }
}

// ------------------------------------------------------------------ dispatch
template <typename R> static typename CT<R>::T to_c(const cd &z) {
    typename CT<R>::T r;
    r.x = R(z.real());
    r.y = R(z.imag());
    return r;
}

// hi + lo with hi = x rounded to float and lo = x - hi rounded to float
// (host; the matrix entries of the double-float sweeps)
static void df_parts(double x, float &hi, float &lo) {
    hi = float(x);
    lo = float(x - double(hi));
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
            IndexMap map = make_index_map(op.targets, k, op.controls, c);
            map.limit = uint64_t(1) << n;
            const uint64_t ngroups = uint64_t(1) << (n - k - c);
            const double bytes = 2.0 * S * double(ngroups << k);
            if (k == 1) {
                Mat2<R> m{to_c<R>(op.m[0]), to_c<R>(op.m[1]), to_c<R>(op.m[2]), to_c<R>(op.m[3])};
                constexpr int PER = 4, T = 256;
                const uint64_t blocks = (ngroups + T * PER - 1) / (T * PER);
                LaunchScope ls(K_DENSE1, st, bytes, 16.0 * double(ngroups << 1));
                if constexpr (sizeof(R) == 8) {
                    constexpr int PD = 2;
                    DfMat2 dm{};
                    for (int e = 0; e < 4; ++e) {
                        df_parts(op.m[size_t(e)].real(), dm.v[4 * e], dm.v[4 * e + 1]);
                        df_parts(op.m[size_t(e)].imag(), dm.v[4 * e + 2], dm.v[4 * e + 3]);
                    }
                    k_dense1_df<PD><<<unsigned((ngroups + T * PD - 1) / (T * PD)), T, 0, st>>>(
                        reinterpret_cast<double2 *>(psi), ngroups, map, uint64_t(1) << op.targets[0], dm, m,
                        DF_FP64_WARPS);
                } else {
                    k_dense1<R, PER><<<unsigned(blocks), T, 0, st>>>(psi, ngroups, map,
                                                                      uint64_t(1) << op.targets[0], m);
                }
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
            IndexMap map = make_index_map(nullptr, 0, op.controls, c);
            map.limit = uint64_t(1) << n;
            const uint64_t count = uint64_t(1) << (n - c);
            DiagParams<R> p{};
            p.k = k;
            for (int i = 0; i < k; ++i) p.tbits[i] = op.targets[i];
            for (int j = 0; j < (1 << k); ++j) p.d[j] = to_c<R>(op.m[j]);
            constexpr int PER = 4, T = 256;
            const uint64_t blocks = (count + T * PER - 1) / (T * PER);
            bool signs = true;  // every entry exactly +1 or -1
            uint64_t neg = 0;
            for (int j = 0; j < (1 << k); ++j) {
                if (op.m[j] == cd(-1.0)) neg |= uint64_t(1) << j;
                else if (op.m[j] != cd(1.0)) signs = false;
            }
            if (signs) {
                // only the flipped amplitudes are written: bytes read S * count,
                // written S * (flipped share of count)
                const double flipped = double(__builtin_popcountll(neg)) / double(1 << k);
                LaunchScope ls(K_DIAG, st, S * double(count) * (1.0 + flipped));
                int tb[6] = {0, 0, 0, 0, 0, 0};
                for (int i = 0; i < k; ++i) tb[i] = op.targets[i];
                k_diag_sign<R, PER><<<unsigned(blocks), T, 0, st>>>(psi, count, map, k, neg, tb[0], tb[1], tb[2],
                                                                    tb[3], tb[4], tb[5]);
                break;
            }
            LaunchScope ls(K_DIAG, st, 2.0 * S * double(count), 6.0 * double(count));
            if constexpr (sizeof(R) == 8) {
                constexpr int PD = 2;
                k_diag_df<PD><<<unsigned((count + T * PD - 1) / (T * PD)), T, 0, st>>>(
                    reinterpret_cast<double2 *>(psi), count, map, p);
            } else {
                k_diag<R, PER><<<unsigned(blocks), T, 0, st>>>(psi, count, map, p);
            }
            break;
        }
        case Op::MONO: {
            IndexMap map = make_index_map(op.targets, k, op.controls, c);
            map.limit = uint64_t(1) << n;
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
            bool unit = true;  // no phase to apply: the moved amplitudes are copied exactly
            for (int r = 0; r < (1 << k); ++r) unit &= op.phase[r] == cd(1.0);
            LaunchScope ls(K_MONO, st, 2.0 * S * double(ngroups) * p.na);
            const unsigned b4 = unsigned((ngroups + T * 4 - 1) / (T * 4)), b1 = unsigned((ngroups + T - 1) / T);
            if (p.na <= 2) {
                if (unit) k_mono<R, 2, 4, true><<<b4, T, 0, st>>>(psi, ngroups, map, p);
                else k_mono<R, 2, 4, false><<<b4, T, 0, st>>>(psi, ngroups, map, p);
            } else {
                if (unit) k_mono<R, 8, 1, true><<<b1, T, 0, st>>>(psi, ngroups, map, p);
                else k_mono<R, 8, 1, false><<<b1, T, 0, st>>>(psi, ngroups, map, p);
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

namespace qsim {
unsigned long long sweep_debug_oob(bool clear) {
#ifdef QSIM_DEBUG
    unsigned long long v = 0;
    cudaMemcpyFromSymbol(&v, g_sweep_oob, sizeof v);
    if (clear) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_sweep_oob, &z, sizeof z);
    }
    return v;
#else
    (void)clear;
    return 0;
#endif
}
}  // namespace qsim

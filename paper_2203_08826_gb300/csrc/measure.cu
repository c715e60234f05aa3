// Measurement kernels: probabilities, marginals, squared norm, Pauli
// expectations (double accumulation, warp-shuffle trees) and the inverse-CDF
// shot sampler with Philox4x32-10 (measurement operators, Sec. 2).
#include "internal.h"

namespace qsim {

// |psi|^2 in double, rounded once from the exact value re^2 + im^2.
// complex64: both squares of fp32 values are exact in double (48-bit
// products), so one fused multiply-add gives the same double as the separate
// product-and-sum; complex128 keeps the two roundings of the product-and-sum
// without contraction, so the result does not depend on scheduling.
__device__ __forceinline__ double prob_of(float2 a) {
    const double re = a.x, im = a.y;
    return __fma_rn(re, re, __dmul_rn(im, im));
}
__device__ __forceinline__ double prob_of(double2 a) {
    return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}

// ---- complex64 weights in integer arithmetic
// floor(p * 2^62) for p = RN_double(re^2 + im^2), the value prob_c64 gives,
// without fp64 (GB300's fp64 rate made the fp64 form the sampler's limit).
// re^2 and im^2 are exact products of the 24-bit significands (subnormals
// normalised first); the larger is shifted left by at most 15 bits onto the
// smaller, bits of the smaller that fall below the 64-bit window are kept as
// one sticky bit, and the sum is rounded to 53 bits, nearest-even.  Every
// step is 64-bit integer arithmetic.
__host__ __device__ inline int clz64_hd(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __clzll(static_cast<long long>(v));
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

__host__ __device__ inline void square_of_float(uint32_t u, uint64_t &M, int &E) {
    const uint32_t e = u >> 23, m = u & 0x7FFFFFu;
    uint64_t mant;
    int ex;
    if (e == 0) {
        const int sh = (clz64_hd(m) - 32) - 8;  // leading bit to position 23
        mant = uint64_t(m) << sh;
        ex = -149 - sh;
    } else {
        mant = m | 0x800000u;
        ex = int(e) - 150;
    }
    M = mant * mant;
    E = 2 * ex;
}

// RN_double(re^2 + im^2) as M53 * 2^E53 (M53 < 2^53); returns 0 for zero,
// 1 for a finite positive value, 2 for NaN, 3 for infinity.
__host__ __device__ inline int sumsq_rn(float re, float im, uint64_t &M53, int &E53) {
    uint32_t ux, uy;
    memcpy(&ux, &re, 4);
    memcpy(&uy, &im, 4);
    ux &= 0x7FFFFFFFu;
    uy &= 0x7FFFFFFFu;
    if (ux > 0x7F800000u || uy > 0x7F800000u) return 2;
    if (ux == 0x7F800000u || uy == 0x7F800000u) return 3;
    if (ux < uy) {  // |re| >= |im|, which orders the normalised exponents too
        const uint32_t t = ux;
        ux = uy;
        uy = t;
    }
    if (ux == 0) return 0;
    uint64_t M1, M2;
    int E1, E2;
    square_of_float(ux, M1, E1);
    if (uy == 0) {
        M53 = M1;
        E53 = E1;
        return 1;
    }
    square_of_float(uy, M2, E2);
    // re^2 + im^2 = 2^(E1 - c) (M1 2^c + M2 2^-r + ...) with c = min(d, 15),
    // r = d - c: the M2 bits shifted out only decide ties, so they are folded
    // into bit 0 (a sticky bit; when r > 0, T >= 2^61 keeps >= 9 bits below
    // the rounding point).  T < 2^63 + 2^48.
    const int d = E1 - E2;
    const int c = d < 15 ? d : 15;
    const int r = d - c < 63 ? d - c : 63;
    const uint64_t sticky = (M2 & ((uint64_t(1) << r) - 1)) != 0 ? 1 : 0;
    const uint64_t T = ((M1 << c) + (M2 >> r)) | sticky;
    const int L = 64 - clz64_hd(T);
    if (L <= 53) {  // exact (no sticky bit is possible here)
        M53 = T;
        E53 = E1 - c;
        return 1;
    }
    int sh = L - 53;
    uint64_t q = T >> sh;
    const uint64_t rem = T & ((uint64_t(1) << sh) - 1), half = uint64_t(1) << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q >> 53) {
        q >>= 1;
        ++sh;
    }
    M53 = q;
    E53 = E1 - c + sh;
    return 1;
}

__host__ __device__ inline uint64_t weight_c64_exact(float re, float im) {
    uint32_t ux, uy;
    memcpy(&ux, &re, 4);
    memcpy(&uy, &im, 4);
    ux &= 0x7FFFFFFFu;
    uy &= 0x7FFFFFFFu;
    if (ux > 0x7F800000u || uy > 0x7F800000u) return 0;         // NaN
    const uint32_t big = ux > uy ? ux : uy;
    if (big >= 0x3F800000u) return uint64_t(1) << 62;           // a part >= 1 (or infinite): p >= 1
    if (big < (95u << 23)) return 0;                             // both parts < 2^-32: p <= 2^-63
    uint64_t M53;
    int E53;
    sumsq_rn(re, im, M53, E53);
    const int s = E53 + 62;
    if (s >= 0) return (64 - clz64_hd(M53)) + s > 62 ? uint64_t(1) << 62 : (M53 << s);  // p >= 1: 2^62
    return -s < 64 ? (M53 >> -s) : 0;
}

// The same weight by a shorter route where it applies.  With |re|, |im|
// below 2^-10, A = (re^2 + im^2) 2^62 is below 2^43, so rounding to double
// moves it by at most 2^-11 and changes floor(A) only if A's fraction is at
// least 1 - 2^-11.  V = floor(re^2 2^73) + floor(im^2 2^73) is floor(A 2^11)
// or one less; when V's low 11 bits are below 0x7FE, both candidates have
// the same floor(A) and a fraction below 1 - 2^-11, so the weight is V >> 11.
// Otherwise (about one element in a thousand), and for larger parts, the
// exact rule above decides.  Parts below 2^-32 give p <= 2^-63: weight 0.
__host__ __device__ inline uint64_t weight_c64(float re, float im) {
    uint32_t ux, uy;
    memcpy(&ux, &re, 4);
    memcpy(&uy, &im, 4);
    ux &= 0x7FFFFFFFu;
    uy &= 0x7FFFFFFFu;
    if (ux < uy) {  // a NaN or infinity ends up in ux and goes to the exact rule
        const uint32_t t = ux;
        ux = uy;
        uy = t;
    }
    const uint32_t ex = ux >> 23, ey = uy >> 23;
    if (ex < 95) return 0;
    if (ex > 116) return weight_c64_exact(re, im);
    // significands and the exponents of their squares in units of 2^-73
    // (a subnormal im has no implicit bit and the scale of exponent 1)
    const uint64_t mx = (ux & 0x7FFFFFu) | 0x800000u, my = (uy & 0x7FFFFFu) | (ey ? 0x800000u : 0u);
    const int u1 = 2 * int(ex) - 227, u2 = 2 * int(ey ? ey : 1) - 227;
    const uint64_t M1 = mx * mx, M2 = my * my;
    const uint64_t t1 = u1 >= 0 ? (M1 << u1) : (M1 >> -u1);
    const uint64_t t2 = u2 >= 0 ? (M2 << u2) : (-u2 < 64 ? (M2 >> -u2) : 0);
    const uint64_t V = t1 + t2;
    if ((V & 0x7FFu) >= 0x7FEu) return weight_c64_exact(re, im);
    return V >> 11;
}

// The same value as a double, assembled from its bits (complex64 inputs give
// normal doubles: a nonzero square is at least 2^-298).
__host__ __device__ inline double prob_c64(float re, float im) {
    uint64_t M53;
    int E53;
    const int kind = sumsq_rn(re, im, M53, E53);
    uint64_t bits;
    if (kind == 0) {
        bits = 0;
    } else if (kind == 2) {
        bits = 0x7FF8000000000000ull;
    } else if (kind == 3) {
        bits = 0x7FF0000000000000ull;
    } else {
        const int lz = clz64_hd(M53) - 11;  // shift the leading bit to position 52
        const uint64_t M = M53 << lz;
        const int E = E53 - lz;             // value = M 2^E, 2^52 <= M < 2^53
        bits = (uint64_t(E + 1075) << 52) | (M & ((uint64_t(1) << 52) - 1));
    }
    double p;
    memcpy(&p, &bits, 8);
    return p;
}


static int sm_count() { return device_sm_count(); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum, result valid in thread 0.  blockDim.x must be a multiple of 32.
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

// Block-wide maximum of non-negative values, result valid in thread 0.
__device__ double block_max(double v) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = 0;
    if (w == 0) {
        v = lane < int(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// ------------------------------------------------------------------ probabilities
template <typename C>
__global__ void k_probs(const C *__restrict__ psi, uint64_t N, double *__restrict__ out) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride)
        out[i] = prob_of(psi[i]);
}

// complex64: the same doubles as prob_of, formed with integer operations
// (no fp64 per amplitude), two amplitudes per 16-byte load
__global__ void __launch_bounds__(256) k_probs_c64(const float4 *__restrict__ psi4, uint64_t n4,
                                                   double2 *__restrict__ out2) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 v = psi4[i];
        out2[i] = make_double2(prob_c64(v.x, v.y), prob_c64(v.z, v.w));
    }
}

int launch_probs(const void *psi, int n, int dtype, double *out, cudaStream_t st) {
    const uint64_t N = uint64_t(1) << n;
    const int T = 256;
    const int blocks = int(std::min<uint64_t>((N + T - 1) / T, uint64_t(sm_count()) * 16));
    LaunchScope ls(K_PROBS, st, double(N) * ((dtype == QSIM_C64 ? 8 : 16) + 8));
    if (dtype == QSIM_C64 && N >= 2 && (reinterpret_cast<uintptr_t>(out) & 15) == 0)
        k_probs_c64<<<blocks, T, 0, st>>>(static_cast<const float4 *>(psi), N / 2, reinterpret_cast<double2 *>(out));
    else if (dtype == QSIM_C64)
        k_probs<<<blocks, T, 0, st>>>(static_cast<const float2 *>(psi), N, out);
    else
        k_probs<<<blocks, T, 0, st>>>(static_cast<const double2 *>(psi), N, out);
    QSIM_CUDA_TRY(cudaGetLastError(), "probabilities launch");
    return QSIM_OK;
}

// ------------------------------------------------------------------ marginals
// Output bit (m-1-i) of y is amplitude bit qubits[i].
struct MargParams {
    int m;
    int q[64];
};

__device__ __forceinline__ uint64_t gather_bits(uint64_t x, const MargParams &p) {
    uint64_t y = 0;
    for (int i = 0; i < p.m; ++i) y = (y << 1) | ((x >> p.q[i]) & 1);
    return y;
}

// few bins: per-CTA shared-memory histogram, then per-CTA rows in scratch
template <typename C>
__global__ void k_marg_hist(const C *__restrict__ psi, uint64_t N, const __grid_constant__ MargParams p, double *__restrict__ rows) {
    extern __shared__ double hist[];
    const int nb = 1 << p.m;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < N; x += stride)
        atomicAdd(&hist[gather_bits(x, p)], prob_of(psi[x]));
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) rows[uint64_t(blockIdx.x) * nb + i] = hist[i];
}

__global__ void k_marg_rows(const double *__restrict__ rows, int nrows, int nb, double *__restrict__ out) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= nb) return;
    double s = 0;
    for (int r = 0; r < nrows; ++r) s += rows[uint64_t(r) * nb + y];
    out[y] = s;
}

// many bins: one thread per output, summing over the complementary bits
template <typename C>
__global__ void k_marg_many(const C *__restrict__ psi, uint64_t nout, uint64_t nrest, const __grid_constant__ MargParams p,
                            IndexMap zero_at_listed, double *__restrict__ out) {
    const uint64_t y = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (y >= nout) return;
    uint64_t ybits = 0;
    for (int i = 0; i < p.m; ++i)
        if ((y >> (p.m - 1 - i)) & 1) ybits |= uint64_t(1) << p.q[i];
    double s = 0;
    for (uint64_t z = 0; z < nrest; ++z) {
        uint64_t x = z;
        for (int i = 0; i < zero_at_listed.nins; ++i) {
            const uint64_t low = x & ((uint64_t(1) << zero_at_listed.ins[i]) - 1);
            x = ((x ^ low) << 1) | low;
        }
        s += prob_of(psi[x | ybits]);
    }
    out[y] = s;
}

static int marg_blocks() { return sm_count() * 2; }

size_t marginal_scratch_doubles(int n, int m) {
    (void)n;
    return m <= 12 ? size_t(marg_blocks()) << m : 0;
}

int launch_marginal(const void *psi, int n, int dtype, const int *qubits, int m, double *out,
                    double *scratch, size_t scratch_doubles, cudaStream_t st) {
    if (m > 62) return set_error(QSIM_EINVAL, "too many qubits");
    MargParams p{};
    p.m = m;
    for (int i = 0; i < m; ++i) p.q[i] = qubits[i];
    const uint64_t N = uint64_t(1) << n;
    const double bytes = double(N) * (dtype == QSIM_C64 ? 8 : 16);
    if (m <= 12) {
        const int blocks = marg_blocks(), T = 256, nb = 1 << m;
        if (scratch_doubles < size_t(blocks) * nb) return set_error(QSIM_EINVAL, "marginal scratch too small");
        {
            LaunchScope ls(K_MARGINAL, st, bytes);
            if (dtype == QSIM_C64)
                k_marg_hist<<<blocks, T, nb * sizeof(double), st>>>(static_cast<const float2 *>(psi), N, p, scratch);
            else
                k_marg_hist<<<blocks, T, nb * sizeof(double), st>>>(static_cast<const double2 *>(psi), N, p, scratch);
            QSIM_CUDA_TRY(cudaGetLastError(), "marginal launch");
        }
        LaunchScope ls(K_REDUCE, st, double(blocks) * nb * 8);
        k_marg_rows<<<(nb + 255) / 256, 256, 0, st>>>(scratch, blocks, nb, out);
        QSIM_CUDA_TRY(cudaGetLastError(), "marginal rows launch");
        return QSIM_OK;
    }
    int sorted[64];
    for (int i = 0; i < m; ++i) sorted[i] = qubits[i];
    if (m > MAX_INS) {
        // more listed qubits than an IndexMap holds: fall back to a wider map
        return set_error(QSIM_EUNSUPPORTED, "marginals over more than %d qubits with m > 12", MAX_INS);
    }
    const IndexMap zmap = make_index_map(sorted, m, nullptr, 0);
    const uint64_t nout = uint64_t(1) << m, nrest = uint64_t(1) << (n - m);
    LaunchScope ls(K_MARGINAL, st, bytes);
    if (dtype == QSIM_C64)
        k_marg_many<<<unsigned((nout + 255) / 256), 256, 0, st>>>(static_cast<const float2 *>(psi), nout, nrest, p,
                                                                   zmap, out);
    else
        k_marg_many<<<unsigned((nout + 255) / 256), 256, 0, st>>>(static_cast<const double2 *>(psi), nout, nrest, p,
                                                                   zmap, out);
    QSIM_CUDA_TRY(cudaGetLastError(), "marginal launch");
    return QSIM_OK;
}

// ------------------------------------------------------------------ reductions
static int reduce_blocks() { return sm_count() * 4; }
size_t reduce_partials_needed(int n) {
    (void)n;
    return size_t(reduce_blocks());
}

// Squared norm, accumulated in double per thread, per warp and per block.
template <typename C>
__global__ void __launch_bounds__(256) k_norm2(const C *__restrict__ psi, uint64_t N, double *__restrict__ partials) {
    double acc = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        const C a = psi[i];
        acc += double(a.x) * double(a.x) + double(a.y) * double(a.y);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Squared 2-norm and largest modulus of a - b (double), per block; a and b
// may differ in precision (a complex64 result against a complex128 reference).
template <typename CA, typename CB>
__global__ void __launch_bounds__(256) k_diff2(const CA *__restrict__ a, const CB *__restrict__ b, uint64_t N,
                                               double *__restrict__ partials, double *__restrict__ maxes) {
    double acc = 0, mx = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
        const double dx = double(a[i].x) - double(b[i].x), dy = double(a[i].y) - double(b[i].y);
        const double d2 = dx * dx + dy * dy;
        acc += d2;
        mx = fmax(mx, d2);
    }
    acc = block_sum(acc);
    mx = block_max(mx);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = acc;
        maxes[blockIdx.x] = mx;
    }
}

// result (+)= sum of partials, in a fixed order (one block)
__global__ void k_sum_partials(const double *__restrict__ partials, int np, double *__restrict__ result,
                               int accumulate) {
    double acc = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partials[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *result = accumulate ? *result + acc : acc;
}

__global__ void k_max_partials(const double *__restrict__ partials, int np, double *__restrict__ result) {
    double mx = 0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) mx = fmax(mx, partials[i]);
    mx = block_max(mx);
    if (threadIdx.x == 0) *result = mx;
}

int launch_diff_norm2(const void *a, const void *b, int n, int dtype, double *partials, double *result,
                      cudaStream_t st) {
    const uint64_t N = uint64_t(1) << n;
    const int blocks = reduce_blocks(), T = 256;
    {
        LaunchScope ls(K_REDUCE, st, 2.0 * double(N) * (dtype == QSIM_C64 ? 8 : 16));
        if (dtype == QSIM_C64)
            k_diff2<<<blocks, T, 0, st>>>(static_cast<const float2 *>(a), static_cast<const float2 *>(b), N, partials,
                                          partials + blocks);
        else
            k_diff2<<<blocks, T, 0, st>>>(static_cast<const double2 *>(a), static_cast<const double2 *>(b), N,
                                          partials, partials + blocks);
        QSIM_CUDA_TRY(cudaGetLastError(), "difference launch");
    }
    LaunchScope ls(K_REDUCE, st, blocks * 16.0);
    k_sum_partials<<<1, 256, 0, st>>>(partials, blocks, result, 0);
    k_max_partials<<<1, 256, 0, st>>>(partials + blocks, blocks, result + 1);
    QSIM_CUDA_TRY(cudaGetLastError(), "difference sum launch");
    return QSIM_OK;
}

int launch_diff_norm2_c64_c128(const void *a, const void *b, int n, double *partials, double *result,
                               cudaStream_t st) {
    const uint64_t N = uint64_t(1) << n;
    const int blocks = reduce_blocks(), T = 256;
    {
        LaunchScope ls(K_REDUCE, st, 24.0 * double(N));
        k_diff2<<<blocks, T, 0, st>>>(static_cast<const float2 *>(a), static_cast<const double2 *>(b), N, partials,
                                      partials + blocks);
        QSIM_CUDA_TRY(cudaGetLastError(), "difference launch");
    }
    LaunchScope ls(K_REDUCE, st, blocks * 16.0);
    k_sum_partials<<<1, 256, 0, st>>>(partials, blocks, result, 0);
    k_max_partials<<<1, 256, 0, st>>>(partials + blocks, blocks, result + 1);
    QSIM_CUDA_TRY(cudaGetLastError(), "difference sum launch");
    return QSIM_OK;
}

// complex64 squared norm without FP64 per amplitude: each square is split
// exactly into p + e (p = x*x, e = fma(x, x, -p)); the p's are summed in a
// float-float pair (Knuth's two-sum), the small e's in float.  Eight 16-byte
// loads per thread are in flight per iteration.
constexpr int RED_U = 4;

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float a) {
    const float s = hi + a;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (a - bp);
    hi = s;
}

__global__ void __launch_bounds__(256) k_norm2_c64(const float4 *__restrict__ psi4, uint64_t n4,
                                                   double *__restrict__ partials) {
    float hi = 0.f, lo = 0.f, el = 0.f;
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x * RED_U;
    for (uint64_t b = uint64_t(blockIdx.x) * blockDim.x * RED_U + threadIdx.x; b < n4; b += step) {
        float4 v[RED_U];
#pragma unroll
        for (int u = 0; u < RED_U; ++u) {
            const uint64_t i = b + uint64_t(u) * blockDim.x;
            v[u] = i < n4 ? psi4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < RED_U; ++u) {
            const float c[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float sq = c[t] * c[t];
                el += fmaf(c[t], c[t], -sq);
                two_sum_add(hi, lo, sq);
            }
        }
    }
    double acc = double(hi) + double(lo) + double(el);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

int launch_norm2(const void *psi, int n, int dtype, double *partials, double *result, cudaStream_t st) {
    const uint64_t N = uint64_t(1) << n;
    const int blocks = reduce_blocks(), T = 256;
    {
        LaunchScope ls(K_REDUCE, st, double(N) * (dtype == QSIM_C64 ? 8 : 16));
        if (dtype == QSIM_C64 && N >= 2)
            k_norm2_c64<<<blocks, T, 0, st>>>(static_cast<const float4 *>(psi), N / 2, partials);
        else if (dtype == QSIM_C64)
            k_norm2<<<blocks, T, 0, st>>>(static_cast<const float2 *>(psi), N, partials);
        else
            k_norm2<<<blocks, T, 0, st>>>(static_cast<const double2 *>(psi), N, partials);
        QSIM_CUDA_TRY(cudaGetLastError(), "norm launch");
    }
    LaunchScope ls(K_REDUCE, st, blocks * 8.0);
    k_sum_partials<<<1, 256, 0, st>>>(partials, blocks, result, 0);
    QSIM_CUDA_TRY(cudaGetLastError(), "norm sum launch");
    return QSIM_OK;
}

// ------------------------------------------------------------------ Pauli expectation
// One pass per distinct xmask X.  With f(y) = sum_t c_t (-1)^{popcount(y & z_t)}
// (c_t = coeff_t * i^{#Y_t}) the group contributes sum_y conj(psi[y ^ X]) f(y) psi[y].
// For X != 0 the pass visits each pair {y, y ^ X} once (bit h = top bit of X is 0).
constexpr int EXP_TERMS = 64;
struct ExpParams {
    uint64_t X;
    int h;        // highest set bit of X, -1 for X == 0
    int nt;
    int uniform;  // every term of the pass has the same coefficient (ur, ui)
    double ur, ui;
    // uniform 2-qubit Z parts: term (a, a + d) contributes bit a of (y ^ (y >> d)),
    // so one popcount per distinct distance d counts the odd terms
    int ndist;
    int dist[EXP_TERMS];
    uint64_t dmask[EXP_TERMS];
    uint64_t z[EXP_TERMS];
    double cr[EXP_TERMS];
    double ci[EXP_TERMS];
};

__device__ __forceinline__ int odd_terms(uint64_t y, const ExpParams &p) {
    int odd = 0;
    if (p.ndist > 0) {
        for (int i = 0; i < p.ndist; ++i) odd += __popcll((y ^ (y >> p.dist[i])) & p.dmask[i]);
    } else {
        for (int t = 0; t < p.nt; ++t) odd += __popcll(y & p.z[t]) & 1;
    }
    return odd;
}

// f(y) = sum_t c_t (-1)^{popcount(y & z_t)}.  With one shared coefficient the
// signs are counted in integers: f = c (nt - 2 * #odd).
__device__ __forceinline__ void f_of(uint64_t y, const ExpParams &p, double &fr, double &fi) {
    if (p.uniform) {
        const double s = double(p.nt - 2 * odd_terms(y, p));
        fr = s * p.ur;
        fi = s * p.ui;
        return;
    }
    fr = 0;
    fi = 0;
    for (int t = 0; t < p.nt; ++t) {
        const double s = (__popcll(y & p.z[t]) & 1) ? -1.0 : 1.0;
        fr += s * p.cr[t];
        fi += s * p.ci[t];
    }
}

// Diagonal pass of a complex64 state with one real coefficient: |psi|^2 times
// the integer sign sum is formed in fp32 (the precision of the complex64
// amplitudes themselves) for the eight amplitudes of one iteration and
// accumulated in double; 16-byte loads, several in flight per thread.
__global__ void __launch_bounds__(256) k_expect_diag_c64(const float4 *__restrict__ psi4, uint64_t n4, const __grid_constant__ ExpParams p,
                                                         double *__restrict__ partials) {
    double acc = 0;
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x * RED_U;
    for (uint64_t b = uint64_t(blockIdx.x) * blockDim.x * RED_U + threadIdx.x; b < n4; b += step) {
        float4 v[RED_U];
#pragma unroll
        for (int u = 0; u < RED_U; ++u) {
            const uint64_t i = b + uint64_t(u) * blockDim.x;
            v[u] = i < n4 ? psi4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < RED_U; ++u) {
            const uint64_t g = 2 * (b + uint64_t(u) * blockDim.x);  // amplitude index of .xy (and g + 1 of .zw)
            part = fmaf(fmaf(v[u].x, v[u].x, v[u].y * v[u].y), float(p.nt - 2 * odd_terms(g, p)), part);
            part = fmaf(fmaf(v[u].z, v[u].z, v[u].w * v[u].w), float(p.nt - 2 * odd_terms(g + 1, p)), part);
        }
        acc += double(part);
    }
    acc = block_sum(acc * p.ur);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Any pass of a complex64 state: products in fp32, eight pairs per iteration
// summed in fp32 and accumulated in double.
__device__ __forceinline__ void f_of_f(uint64_t y, const ExpParams &p, float &fr, float &fi) {
    if (p.uniform) {
        const float s = float(p.nt - 2 * odd_terms(y, p));
        fr = s * float(p.ur);
        fi = s * float(p.ui);
        return;
    }
    fr = 0.f;
    fi = 0.f;
    for (int t = 0; t < p.nt; ++t) {
        const bool odd = __popcll(y & p.z[t]) & 1;
        fr += odd ? -float(p.cr[t]) : float(p.cr[t]);
        fi += odd ? -float(p.ci[t]) : float(p.ci[t]);
    }
}

constexpr int EXP_U = 8;

__global__ void __launch_bounds__(256) k_expect_c64(const float2 *__restrict__ psi, uint64_t count, const __grid_constant__ ExpParams p,
                                                    double *__restrict__ partials) {
    double acc = 0;
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x * EXP_U;
    for (uint64_t b = uint64_t(blockIdx.x) * blockDim.x * EXP_U + threadIdx.x; b < count; b += step) {
        float2 a[EXP_U], c[EXP_U];
        uint64_t y[EXP_U];
#pragma unroll
        for (int u = 0; u < EXP_U; ++u) {
            const uint64_t g = b + uint64_t(u) * blockDim.x;
            if (p.h < 0) {
                y[u] = g;
            } else {
                const uint64_t low = g & ((uint64_t(1) << p.h) - 1);
                y[u] = ((g ^ low) << 1) | low;  // bit h of y is 0
            }
            a[u] = g < count ? psi[y[u]] : make_float2(0.f, 0.f);
            c[u] = (g < count && p.h >= 0) ? psi[y[u] ^ p.X] : make_float2(0.f, 0.f);
        }
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < EXP_U; ++u) {
            float fr, fi;
            f_of_f(y[u], p, fr, fi);
            if (p.h < 0) {
                part = fmaf(fmaf(a[u].x, a[u].x, a[u].y * a[u].y), fr, part);
            } else {
                float gr, gi;
                f_of_f(y[u] ^ p.X, p, gr, gi);
                const float bar = fmaf(c[u].x, a[u].x, c[u].y * a[u].y);   // Re(conj(b) a)
                const float bai = fmaf(c[u].x, a[u].y, -c[u].y * a[u].x);  // Im(conj(b) a)
                part += (fr + gr) * bar + (gi - fi) * bai;
            }
        }
        acc += double(part);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// X-group pass of a complex64 state (X != 0): for the pair (y, y ^ X) with
// bit h of y clear, a = psi[y], b = psi[y ^ X], the group contributes
// Re(conj(b) a) sum_t s_t A_t + Im(conj(b) a) sum_t s_t B_t with
// s_t = (-1)^popcount(y & z_t); the host folded the sign change of each term
// between y and y ^ X into A_t = Re c_t (1 + sigma_t), B_t = Im c_t (sigma_t - 1),
// sigma_t = (-1)^popcount(X & z_t).
struct ExpXParams {
    uint64_t X;
    int h, nt;
    uint64_t z[EXP_TERMS];
    float A[EXP_TERMS], B[EXP_TERMS];
};

__global__ void __launch_bounds__(256) k_expect_x_c64(const float2 *__restrict__ psi, uint64_t count,
                                                      const __grid_constant__ ExpXParams p,
                                                      double *__restrict__ partials) {
    double acc = 0;
    const uint64_t lowmask = (uint64_t(1) << p.h) - 1;
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x * EXP_U;
    for (uint64_t b = uint64_t(blockIdx.x) * blockDim.x * EXP_U + threadIdx.x; b < count; b += step) {
        float2 va[EXP_U], vb[EXP_U];
        uint64_t y[EXP_U];
#pragma unroll
        for (int u = 0; u < EXP_U; ++u) {
            const uint64_t g = b + uint64_t(u) * blockDim.x;
            const uint64_t low = g & lowmask;
            y[u] = ((g ^ low) << 1) | low;
            const bool in = g < count;
            va[u] = in ? psi[y[u]] : make_float2(0.f, 0.f);
            vb[u] = in ? psi[y[u] ^ p.X] : make_float2(0.f, 0.f);
        }
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < EXP_U; ++u) {
            float sa = 0.f, sb = 0.f;
            for (int t = 0; t < p.nt; ++t) {
                const bool odd = __popcll(y[u] & p.z[t]) & 1;
                sa += odd ? -p.A[t] : p.A[t];
                sb += odd ? -p.B[t] : p.B[t];
            }
            const float bar = fmaf(vb[u].x, va[u].x, vb[u].y * va[u].y);
            const float bai = fmaf(vb[u].x, va[u].y, -vb[u].y * va[u].x);
            part = fmaf(bar, sa, fmaf(bai, sb, part));
        }
        acc += double(part);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename C>
__global__ void __launch_bounds__(256) k_expect(const C *__restrict__ psi, uint64_t count, const __grid_constant__ ExpParams p,
                                                double *__restrict__ partials) {
    double acc = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t g = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; g < count; g += stride) {
        if (p.h < 0) {
            const C a = psi[g];
            double fr, fi;
            f_of(g, p, fr, fi);
            acc += (double(a.x) * a.x + double(a.y) * a.y) * fr;
        } else {
            const uint64_t low = g & ((uint64_t(1) << p.h) - 1);
            const uint64_t y = ((g ^ low) << 1) | low;  // bit h of y is 0
            const uint64_t y2 = y ^ p.X;
            const C a = psi[y], b = psi[y2];
            double fr, fi, gr, gi;
            f_of(y, p, fr, fi);
            f_of(y2, p, gr, gi);
            // Re[conj(b) f(y) a + conj(a) f(y2) b]
            const double bar = double(b.x) * a.x + double(b.y) * a.y;   // Re(conj(b) a)
            const double bai = double(b.x) * a.y - double(b.y) * a.x;   // Im(conj(b) a)
            acc += fr * bar - fi * bai;
            acc += gr * bar + gi * bai;  // conj(a) b = conj(conj(b) a)
        }
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

int launch_expect(const void *psi, int n, int dtype, int nterms, const uint64_t *xmask, const uint64_t *zmask,
                  const double *coeff, double *partials, size_t npartials, double *result, cudaStream_t st) {
    const uint64_t N = uint64_t(1) << n;
    const int blocks = reduce_blocks(), T = 256;
    if (npartials < size_t(blocks)) return set_error(QSIM_EINVAL, "expectation scratch too small");
    QSIM_CUDA_TRY(cudaMemsetAsync(result, 0, sizeof(double), st), "expectation zero");
    std::vector<bool> done(nterms, false);
    for (int t0 = 0; t0 < nterms; ++t0) {
        if (done[t0]) continue;
        ExpParams p{};
        p.X = xmask[t0];
        p.h = p.X ? 63 - __builtin_clzll(p.X) : -1;
        for (int t = t0; t < nterms && p.nt < EXP_TERMS; ++t) {
            if (done[t] || xmask[t] != p.X) continue;
            done[t] = true;
            const int ny = __builtin_popcountll(xmask[t] & zmask[t]);
            // i^{#Y}: 1, i, -1, -i
            const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
            p.z[p.nt] = zmask[t];
            p.cr[p.nt] = coeff[t] * re[ny & 3];
            p.ci[p.nt] = coeff[t] * im[ny & 3];
            ++p.nt;
        }
        const uint64_t count = p.h < 0 ? N : N / 2;
        p.uniform = 1;
        p.ur = p.cr[0];
        p.ui = p.ci[0];
        for (int t = 1; t < p.nt; ++t)
            if (p.cr[t] != p.ur || p.ci[t] != p.ui) p.uniform = 0;
        // two-bit Z parts grouped by distance (ZZ chains and couplings)
        bool two_bit = p.uniform != 0;
        for (int t = 0; t < p.nt && two_bit; ++t) two_bit = __builtin_popcountll(p.z[t]) == 2;
        if (two_bit) {
            for (int t = 0; t < p.nt; ++t) {
                const int a = __builtin_ctzll(p.z[t]), b = 63 - __builtin_clzll(p.z[t]);
                int i = 0;
                while (i < p.ndist && p.dist[i] != b - a) ++i;
                if (i == p.ndist) {
                    p.dist[p.ndist] = b - a;
                    p.dmask[p.ndist] = 0;
                    ++p.ndist;
                }
                p.dmask[i] |= uint64_t(1) << a;
            }
        }
        {
            LaunchScope ls(K_EXPECT, st, double(N) * (dtype == QSIM_C64 ? 8 : 16));
            if (dtype == QSIM_C64 && p.h < 0 && p.uniform && p.ui == 0.0 && N >= 2)
                k_expect_diag_c64<<<blocks, T, 0, st>>>(static_cast<const float4 *>(psi), N / 2, p, partials);
            else if (dtype == QSIM_C64 && p.h >= 0) {
                ExpXParams xp{};
                xp.X = p.X;
                xp.h = p.h;
                xp.nt = p.nt;
                for (int t = 0; t < p.nt; ++t) {
                    const double sigma = (__builtin_popcountll(p.X & p.z[t]) & 1) ? -1.0 : 1.0;
                    xp.z[t] = p.z[t];
                    xp.A[t] = float(p.cr[t] * (1.0 + sigma));
                    xp.B[t] = float(p.ci[t] * (sigma - 1.0));
                }
                k_expect_x_c64<<<blocks, T, 0, st>>>(static_cast<const float2 *>(psi), count, xp, partials);
            } else if (dtype == QSIM_C64)
                k_expect_c64<<<blocks, T, 0, st>>>(static_cast<const float2 *>(psi), count, p, partials);
            else
                k_expect<<<blocks, T, 0, st>>>(static_cast<const double2 *>(psi), count, p, partials);
            QSIM_CUDA_TRY(cudaGetLastError(), "expectation launch");
        }
        LaunchScope ls(K_REDUCE, st, blocks * 8.0);
        k_sum_partials<<<1, 256, 0, st>>>(partials, blocks, result, 1);
        QSIM_CUDA_TRY(cudaGetLastError(), "expectation sum launch");
        // terms beyond EXP_TERMS with this xmask stay !done and start their own pass
    }
    return QSIM_OK;
}

// ------------------------------------------------------------------ sampler
// Philox4x32-10, Salmon et al., SC'11: ten rounds of the 4x32 S-box
// (multipliers 0xD2511F53, 0xCD9E8D57), key bumped by 0x9E3779B9 / 0xBB67AE85
// between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

constexpr int CHUNK = 2048;  // amplitudes per first-level CDF entry

// floor(p * 2^62) for 0 < p < 1, read off the binary representation: with
// p = m 2^(e-52) (m the 53-bit significand) the weight is m shifted by e + 10.
__device__ __forceinline__ uint64_t weight_of(double p) {
    // integer tests on the bits: negative, zero, subnormal -> 0; NaN -> 0; >= 1 -> 2^62
    const uint64_t bits = uint64_t(__double_as_longlong(p));
    if (bits >> 63) return 0;
    const int ex = int((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;  // zero or subnormal: far below 2^-62
    if (ex == 0x7FF) return (bits & ((uint64_t(1) << 52) - 1)) ? 0 : (uint64_t(1) << 62);
    if (ex >= 1023) return uint64_t(1) << 62;
    const uint64_t m = (bits & ((uint64_t(1) << 52) - 1)) | (uint64_t(1) << 52);
    const int sh = ex - 1023 + 10;  // <= 9 because p < 1
    return sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0);
}

template <int SRC>
__device__ __forceinline__ double src_prob(const void *src, uint64_t x) {
    if (SRC == SRC_C64) return prob_of(static_cast<const float2 *>(src)[x]);
    if (SRC == SRC_C128) return prob_of(static_cast<const double2 *>(src)[x]);
    return static_cast<const double *>(src)[x];
}

template <int SRC>
__device__ __forceinline__ uint64_t src_weight(const void *src, uint64_t x) {
    if (SRC == SRC_C64) {
        const float2 a = static_cast<const float2 *>(src)[x];
        return weight_c64(a.x, a.y);
    }
    return weight_of(src_prob<SRC>(src, x));
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// chunk sums of the integer weights: one warp per chunk of CHUNK
// probabilities (lane l takes elements l, l + 32, ...), 8 chunks per CTA; the
// probability sum only guards against inputs summing above 1.5, so it is
// accumulated in fp32 per warp and once per CTA in double
template <int SRC>
__global__ void __launch_bounds__(256) k_sample_chunk(const void *__restrict__ src, uint64_t N, uint64_t nchunks,
                                                      uint64_t *__restrict__ sums, double *__restrict__ psum,
                                                      int vec) {
    __shared__ float ps[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t c = uint64_t(blockIdx.x) * 8 + w;
    uint64_t wsum = 0;
    float pf = 0.f;
    if (SRC == SRC_C64 && vec && c < nchunks) {
        // whole chunks of a 16-byte aligned complex64 state: lane l takes the
        // amplitude pairs l, l + 32, ... of the chunk, eight 16-byte loads in
        // flight before their weights are formed (the integer weights add up
        // exactly in any order)
        const float4 *p4 = reinterpret_cast<const float4 *>(static_cast<const float2 *>(src) + c * CHUNK);
        constexpr int U = 8, PER_LANE = CHUNK / 2 / 32;
#pragma unroll 1
        for (int j0 = 0; j0 < PER_LANE; j0 += U) {
            float4 a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] = __ldcs(p4 + (j0 + u) * 32 + lane);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                wsum += weight_c64(a[u].x, a[u].y) + weight_c64(a[u].z, a[u].w);
                pf += a[u].x * a[u].x + a[u].y * a[u].y + a[u].z * a[u].z + a[u].w * a[u].w;
            }
        }
    } else if (c < nchunks) {
        const uint64_t x0 = c * CHUNK;
#pragma unroll 8
        for (int j = 0; j < CHUNK / 32; ++j) {
            const uint64_t x = x0 + uint64_t(j) * 32 + lane;
            if (x < N) {
                if (SRC == SRC_C64) {
                    const float2 a = static_cast<const float2 *>(src)[x];
                    wsum += weight_c64(a.x, a.y);
                    pf += a.x * a.x + a.y * a.y;
                } else {
                    const double p = src_prob<SRC>(src, x);
                    wsum += weight_of(p);
                    pf += p > 0.0 ? float(p) : 0.f;
                }
            }
        }
    }
    wsum = warp_sum_u64(wsum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pf += __shfl_xor_sync(0xffffffffu, pf, o);
    if (lane == 0) {
        if (c < nchunks) sums[c] = wsum;
        ps[w] = pf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < 8; ++i) t += ps[i];
        atomicAdd(psum, t);
    }
}

// Inclusive prefix over the chunk sums in place, in three launches: each
// block scans a tile of SCAN_TILE sums (coalesced, shuffles then shared
// memory); one block forms the exclusive offsets of the tiles (from their last
// elements) and the total (-> sums[nchunks]); every block then adds its tile's
// offset.
constexpr int SCAN_T = 1024, SCAN_PER = 4, SCAN_TILE = SCAN_T * SCAN_PER;

__device__ __forceinline__ uint64_t block_incl_scan_u64(uint64_t x, uint64_t *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < int(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const uint64_t r = x + (warp ? wsum[warp - 1] : 0);
    __syncthreads();  // wsum may be reused
    return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(uint64_t *__restrict__ sums, uint64_t n) {
    __shared__ uint64_t wsum[32];
    const uint64_t base = uint64_t(blockIdx.x) * SCAN_TILE + uint64_t(threadIdx.x) * SCAN_PER;
    uint64_t v[SCAN_PER];
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) v[k] = base + k < n ? sums[base + k] : 0;
#pragma unroll
    for (int k = 1; k < SCAN_PER; ++k) v[k] += v[k - 1];
    const uint64_t incl = block_incl_scan_u64(v[SCAN_PER - 1], wsum);
    const uint64_t excl = incl - v[SCAN_PER - 1];
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k)
        if (base + k < n) sums[base + k] = v[k] + excl;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_offsets(uint64_t *__restrict__ sums, uint64_t n, uint64_t ntiles,
                                                         uint64_t *__restrict__ offs) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t round_total;
    uint64_t carry = 0;
    for (uint64_t t0 = 0; t0 < ntiles; t0 += SCAN_T) {
        const uint64_t t = t0 + threadIdx.x;
        uint64_t last = 0;
        if (t < ntiles) {
            const uint64_t e = (t + 1) * SCAN_TILE < n ? (t + 1) * SCAN_TILE : n;
            last = sums[e - 1];  // the tile's total (its inclusive scan ends there)
        }
        const uint64_t incl = block_incl_scan_u64(last, wsum);
        if (t < ntiles) offs[t] = carry + incl - last;
        if (threadIdx.x == SCAN_T - 1) round_total = incl;
        __syncthreads();
        carry += round_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[n] = carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(uint64_t *__restrict__ sums, uint64_t n,
                                                     const uint64_t *__restrict__ offs) {
    const uint64_t off = offs[blockIdx.x];
    if (off == 0) return;
    const uint64_t base = uint64_t(blockIdx.x) * SCAN_TILE + uint64_t(threadIdx.x) * SCAN_PER;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k)
        if (base + k < n) sums[base + k] += off;
}

// one warp per shot: binary search over the chunk prefix, then a warp scan
// through the chunk in index order
template <int SRC>
__global__ void __launch_bounds__(256) k_sample_draw(const void *__restrict__ src, uint64_t N,
                                                     const uint64_t *__restrict__ prefix, uint64_t nchunks,
                                                     uint64_t nshots, uint64_t seed, uint64_t counter0,
                                                     uint64_t *__restrict__ out) {
    const uint64_t shot = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (shot >= nshots) return;
    const uint64_t T = prefix[nchunks];
    if (T == 0) {
        if (lane == 0) out[shot] = 0;
        return;
    }
    const uint64_t cs = counter0 + shot;
    const uint4 o = philox4x32_10(make_uint4(unsigned(cs), unsigned(cs >> 32), 0u, 0u),
                                  make_uint2(unsigned(seed), unsigned(seed >> 32)));
    const uint64_t u = (uint64_t(o.y) << 32) | o.x;
    const uint64_t r = __umul64hi(u, T);
    // smallest chunk c with prefix[c] > r
    uint64_t lo = 0, hi = nchunks - 1;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (prefix[mid] > r) hi = mid;
        else lo = mid + 1;
    }
    const uint64_t c = lo;
    uint64_t run = c ? prefix[c - 1] : 0;  // CDF just before the chunk
    const uint64_t x0 = c * CHUNK;
    uint64_t found = ((x0 + CHUNK < N) ? x0 + CHUNK : N) - 1;
    for (int j = 0; j < CHUNK / 32; ++j) {
        const uint64_t x = x0 + uint64_t(j) * 32 + lane;
        uint64_t w = x < N ? src_weight<SRC>(src, x) : 0;
        // inclusive warp scan
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t v = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += v;
        }
        const uint64_t cdf = run + w;
        const unsigned hit = __ballot_sync(0xffffffffu, cdf > r);
        if (hit) {
            found = x0 + uint64_t(j) * 32 + (__ffs(hit) - 1);
            break;
        }
        run += __shfl_sync(0xffffffffu, w, 31);
    }
    if (lane == 0) out[shot] = found;
}

size_t sample_scratch_u64(uint64_t N) { return size_t((N + CHUNK - 1) / CHUNK) + 1; }
size_t sample_offsets_u64(uint64_t N) { return size_t(((N + CHUNK - 1) / CHUNK + SCAN_TILE - 1) / SCAN_TILE); }

template <int SRC>
static int launch_sample_t(const void *src, uint64_t N, uint64_t nshots, uint64_t seed, uint64_t counter0,
                           uint64_t *out, uint64_t *scratch, uint64_t *offs, double *psum, cudaStream_t st) {
    const uint64_t nchunks = (N + CHUNK - 1) / CHUNK;
    const double S = SRC == SRC_C64 ? 8 : 16;
    QSIM_CUDA_TRY(cudaMemsetAsync(psum, 0, sizeof(double), st), "sampler zero");
    {
        LaunchScope ls(K_SAMPLE_CHUNK, st, double(N) * S);
        // 16-byte loads when every chunk is whole and the state 16-byte aligned
        const int vec = N % CHUNK == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
        k_sample_chunk<SRC><<<unsigned((nchunks + 7) / 8), 256, 0, st>>>(src, N, nchunks, scratch, psum, vec);
        QSIM_CUDA_TRY(cudaGetLastError(), "sampler chunk launch");
    }
    {
        LaunchScope ls(K_SAMPLE_SCAN, st, double(nchunks) * 16);
        const uint64_t ntiles = (nchunks + SCAN_TILE - 1) / SCAN_TILE;
        k_scan_tiles<<<unsigned(ntiles), SCAN_T, 0, st>>>(scratch, nchunks);
        k_scan_offsets<<<1, SCAN_T, 0, st>>>(scratch, nchunks, ntiles, offs);
        k_scan_add<<<unsigned(ntiles), SCAN_T, 0, st>>>(scratch, nchunks, offs);
        QSIM_CUDA_TRY(cudaGetLastError(), "sampler scan launch");
    }
    if (nshots) {
        const uint64_t threads = nshots * 32;
        LaunchScope ls(K_SAMPLE_DRAW, st, double(nshots) * CHUNK * S);
        k_sample_draw<SRC><<<unsigned((threads + 255) / 256), 256, 0, st>>>(src, N, scratch, nchunks, nshots, seed,
                                                                             counter0, out);
        QSIM_CUDA_TRY(cudaGetLastError(), "sampler draw launch");
    }
    return QSIM_OK;
}

int launch_sample(const void *src, int src_kind, uint64_t N, uint64_t nshots, uint64_t seed, uint64_t counter0,
                  uint64_t *out_dev, uint64_t *scratch, uint64_t *offs, double *psum_dev, cudaStream_t st) {
    if (nshots > (uint64_t(1) << 30)) return set_error(QSIM_EINVAL, "at most 2^30 shots per call");
    switch (src_kind) {
        case SRC_C64: return launch_sample_t<SRC_C64>(src, N, nshots, seed, counter0, out_dev, scratch, offs, psum_dev, st);
        case SRC_C128: return launch_sample_t<SRC_C128>(src, N, nshots, seed, counter0, out_dev, scratch, offs, psum_dev, st);
        default: return launch_sample_t<SRC_PROBS>(src, N, nshots, seed, counter0, out_dev, scratch, offs, psum_dev, st);
    }
}

}  // namespace qsim

// ------------------------------------------------------------------ sampler without allocation
// Some callers may not allocate device memory at all: a framework whose
// caching allocator owns the whole device pool, a service that fixes its
// memory budget at start-up, or a latency-sensitive loop that cannot afford
// the implicit device synchronisation cudaMalloc and cudaFree may bring.
// qsim_sample_probs_static serves them: its scratch (the chunk prefix sums,
// the total weight and the probability sum) lives in this file-scope device
// array, which every GPU that loads the library holds until the process exits.
#include <mutex>

namespace qsim {

constexpr uint64_t STATIC_SAMPLE_MAX_N = uint64_t(1) << 27;         // probabilities
constexpr size_t STATIC_SAMPLE_CHUNKS = size_t(STATIC_SAMPLE_MAX_N / CHUNK);
// [0, chunks]: inclusive chunk prefix + total; [chunks + 1]: probability sum
constexpr size_t STATIC_SAMPLE_WORDS = (STATIC_SAMPLE_CHUNKS + 2 + 31) / 32 * 32;  // 512.25 KiB
// the scan's tile offsets use the array's last words (the padding above)
constexpr size_t STATIC_SCAN_TILES = (STATIC_SAMPLE_CHUNKS + SCAN_TILE - 1) / SCAN_TILE;
static_assert(STATIC_SAMPLE_CHUNKS + 2 + STATIC_SCAN_TILES <= STATIC_SAMPLE_WORDS, "static sampler scratch too small");

static __device__ __align__(256) uint64_t g_sample_scratch[STATIC_SAMPLE_WORDS];

namespace {
std::mutex g_static_mu;
constexpr int MAX_DEVICES = 256;
uint64_t *g_static_ptr[MAX_DEVICES] = {};

// Device address of g_sample_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current.
int static_scratch(uint64_t **out) {
    int dev = 0;
    QSIM_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(QSIM_EUNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        QSIM_CUDA_TRY(cudaGetSymbolAddress(&p, g_sample_scratch), "cudaGetSymbolAddress(sampler scratch)");
        g_static_ptr[dev] = static_cast<uint64_t *>(p);
    }
    *out = g_static_ptr[dev];
    return QSIM_OK;
}
}  // namespace

}  // namespace qsim

extern "C" QSIM_API int qsim_sample_probs_static(const double *p_dev, uint64_t N, uint64_t nshots, uint64_t seed,
                                                 uint64_t counter0, uint64_t *out_dev, void *cuda_stream) {
    using namespace qsim;
    if (!p_dev || (nshots && !out_dev)) return set_error(QSIM_EINVAL, "NULL argument");
    if (N == 0 || N > STATIC_SAMPLE_MAX_N)
        return set_error(QSIM_EINVAL, "N=%llu outside 1..2^27, the capacity of the static sampler scratch",
                         (unsigned long long)N);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    uint64_t *scratch = nullptr;
    QSIM_TRY(static_scratch(&scratch));
    const uint64_t nchunks = (N + CHUNK - 1) / CHUNK;
    double *psum = reinterpret_cast<double *>(scratch + STATIC_SAMPLE_CHUNKS + 1);
    uint64_t *offs = scratch + STATIC_SAMPLE_WORDS - STATIC_SCAN_TILES;
    // the chunk kernel overwrites every prefix entry it uses; the probability
    // sum is accumulated and is cleared by the launcher's memset
    QSIM_TRY(launch_sample(p_dev, SRC_PROBS, N, nshots, seed, counter0, out_dev, scratch, offs, psum, st));
    double hp = 0.0;
    uint64_t total = 0;
    QSIM_CUDA_TRY(cudaMemcpyAsync(&hp, psum, sizeof(double), cudaMemcpyDeviceToHost, st), "psum copy");
    QSIM_CUDA_TRY(cudaMemcpyAsync(&total, scratch + nchunks, sizeof(uint64_t), cudaMemcpyDeviceToHost, st),
                  "total copy");
    QSIM_CUDA_TRY(cudaStreamSynchronize(st), "static sampler sync");
    if (!(hp <= 1.5) || total == 0)
        return set_error(QSIM_EINVAL, "probabilities must sum to a value in (0, 1.5] (got %g)", hp);
    return QSIM_OK;
}

// ------------------------------------------------------------------ collapse
// Measurement collapse (Sec. 2: the operator that collapses and
// re-normalises a state): P = sum of |psi(x)|^2 over the x whose listed bits
// spell the outcome; those amplitudes are divided by sqrt(P), the others set
// to zero.
namespace qsim {
namespace {

template <typename C>
__global__ void __launch_bounds__(256) k_outcome_prob(const C *__restrict__ psi, uint64_t N, uint64_t qmask,
                                                      uint64_t omask, double *__restrict__ partials) {
    double acc = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < N; x += stride)
        if ((x & qmask) == omask) acc += double(psi[x].x) * psi[x].x + double(psi[x].y) * psi[x].y;
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename C>
__global__ void __launch_bounds__(256) k_collapse(C *__restrict__ psi, uint64_t N, uint64_t qmask, uint64_t omask,
                                                  const double *__restrict__ prob) {
    const double inv = 1.0 / sqrt(*prob);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < N; x += stride) {
        C a = psi[x];
        if ((x & qmask) == omask) {
            a.x = a.x * inv;
            a.y = a.y * inv;
        } else {
            a.x = 0;
            a.y = 0;
        }
        psi[x] = a;
    }
}

}  // namespace
}  // namespace qsim

// test support: the complex64 sampler weight rule evaluated on the host
extern "C" uint64_t qsim_sampler_weight_c64(float re, float im) { return qsim::weight_c64(re, im); }
extern "C" double qsim_prob_c64(float re, float im) { return qsim::prob_c64(re, im); }

extern "C" QSIM_API int qsim_collapse(qsim_state *s, const int *qubits, int m, uint64_t outcome, double *prob_out) {
    using namespace qsim;
    if (!s || (m > 0 && !qubits)) return set_error(QSIM_EINVAL, "NULL argument");
    if (m < 1 || m > s->n) return set_error(QSIM_EINVAL, "m=%d outside 1..n", m);
    if (outcome >> m) return set_error(QSIM_EINVAL, "outcome has more than %d bits", m);
    uint64_t qmask = 0, omask = 0;
    for (int i = 0; i < m; ++i) {
        if (qubits[i] < 0 || qubits[i] >= s->n || (qmask >> qubits[i] & 1))
            return set_error(QSIM_EINVAL, "bad or repeated qubit %d", qubits[i]);
        qmask |= uint64_t(1) << qubits[i];
        if ((outcome >> (m - 1 - i)) & 1) omask |= uint64_t(1) << qubits[i];  // qubits[0] = MSB
    }
    const int blocks = reduce_blocks();
    QSIM_TRY(s->ensure_scratch((size_t(blocks) + 8) * sizeof(double)));
    double *part = static_cast<double *>(s->scratch), *res = part + blocks;
    const uint64_t N = s->size();
    {
        LaunchScope ls(K_REDUCE, s->stream, double(N) * s->amp_bytes());
        if (s->dtype == QSIM_C64)
            k_outcome_prob<<<blocks, 256, 0, s->stream>>>(static_cast<const float2 *>(s->amps), N, qmask, omask, part);
        else
            k_outcome_prob<<<blocks, 256, 0, s->stream>>>(static_cast<const double2 *>(s->amps), N, qmask, omask, part);
        QSIM_CUDA_TRY(cudaGetLastError(), "collapse probability launch");
        k_sum_partials<<<1, 256, 0, s->stream>>>(part, blocks, res, 0);
        QSIM_CUDA_TRY(cudaGetLastError(), "collapse sum launch");
    }
    double p = 0;
    QSIM_CUDA_TRY(cudaMemcpyAsync(&p, res, sizeof(double), cudaMemcpyDeviceToHost, s->stream), "collapse copy");
    QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "collapse sync");
    if (prob_out) *prob_out = p;
    if (!(p > 0.0)) return set_error(QSIM_EINVAL, "the outcome has probability 0");
    LaunchScope ls(K_REDUCE, s->stream, 2.0 * double(N) * s->amp_bytes());
    if (s->dtype == QSIM_C64)
        k_collapse<<<blocks, 256, 0, s->stream>>>(static_cast<float2 *>(s->amps), N, qmask, omask, res);
    else
        k_collapse<<<blocks, 256, 0, s->stream>>>(static_cast<double2 *>(s->amps), N, qmask, omask, res);
    QSIM_CUDA_TRY(cudaGetLastError(), "collapse launch");
    return QSIM_OK;
}

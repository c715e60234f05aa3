// Diagonal Pauli-sum evolution: psi <- exp(-i theta D) psi with
// D = sum_t c_t Z(z_t), the diagonal factor of a Trotter step (Sec. 3.3
// turns the evolution into a circuit by the Trotter product; for the TFIM
// the sum of Z_i Z_{i+1} terms is diagonal and its exponential is one phase
// per amplitude).  One HBM pass per call whatever the number of terms:
// D(x) = sum_t c_t (-1)^popcount(x & z_t).
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <complex>
#include <vector>
#include <cstring>

#include "internal.h"

namespace qsim {
namespace {

constexpr int MAX_PHASE_TERMS = 128;
constexpr int GROUP_TERMS = 8;     // terms per sign-pattern table

template <typename R> struct CTe;
template <> struct CTe<float> { using T = float2; };
template <> struct CTe<double> { using T = double2; };

// Up to 64 terms: the parity of every term for an index x is one XOR of
// per-byte tables, P(x) = XOR_b T_b[byte b of x] (bit t of T_b[v] is the
// parity of the part of z_t in byte b for byte value v).  Then
//   equal coefficients: D(x) = c (T - 2 popcount(P)), phase from a table of T + 1;
//   general: the phase is a product over groups of 8 terms of a table entry
//   indexed by the group's 8 parity bits (all 256 sign patterns precomputed).
// Every table is built on the host, copied to the device with the call and
// loaded into shared memory by each (persistent) block.  More than 64 terms:
// one popcount per term and a sine/cosine per amplitude.
constexpr int PAR_TERMS = 64;
constexpr int MAX_BYTES = 8;  // index bytes (n <= 64)

template <typename R> struct PhaseParams {
    using C = typename CTe<R>::T;
    int mode;      // 0 uniform table, 1 group tables, 2 direct (per term)
    int nterms, nbytes, ngroups;
    R theta;
    const uint64_t *ptab;  // [nbytes][256] parity masks (modes 0, 1)
    const C *ftab;         // mode 0: T + 1 phases; mode 1: [ngroups][256] phases
    uint64_t z[MAX_PHASE_TERMS];  // mode 2
    R c[MAX_PHASE_TERMS];
};

__device__ __forceinline__ void sincos_r(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_r(double a, double *s, double *c) { sincos(a, s, c); }

template <typename R, int PER>
__global__ void __launch_bounds__(256) k_pauli_phase(typename CTe<R>::T *__restrict__ psi, uint64_t N,
                                                     const __grid_constant__ PhaseParams<R> p) {
    using C = typename CTe<R>::T;
    __shared__ uint64_t ptab[MAX_BYTES * 256];
    __shared__ C ftab[(PAR_TERMS / GROUP_TERMS) * 256];
    if (p.mode != 2) {
        for (int i = threadIdx.x; i < p.nbytes * 256; i += blockDim.x) ptab[i] = p.ptab[i];
        const int nf = p.mode == 0 ? p.nterms + 1 : p.ngroups * 256;
        for (int i = threadIdx.x; i < nf; i += blockDim.x) ftab[i] = p.ftab[i];
    }
    __syncthreads();
    const uint64_t step = uint64_t(gridDim.x) * blockDim.x * PER;
    for (uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x; base < N; base += step) {
        C a[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint64_t x = base + uint64_t(j) * blockDim.x;
            if (x < N) a[j] = psi[x];
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const uint64_t x = base + uint64_t(j) * blockDim.x;
            if (x >= N) continue;
            C f;
            if (p.mode != 2) {
                uint64_t P = 0;
                for (int b = 0; b < p.nbytes; ++b) P ^= ptab[b * 256 + int((x >> (8 * b)) & 255)];
                if (p.mode == 0) {
                    f = ftab[__popcll(P)];
                } else {
                    f = ftab[int(P & 255)];
                    for (int g = 1; g < p.ngroups; ++g) {
                        const C h = ftab[g * 256 + int((P >> (8 * g)) & 255)];
                        const R fx = f.x * h.x - f.y * h.y;
                        f.y = f.x * h.y + f.y * h.x;
                        f.x = fx;
                    }
                }
            } else {
                R e = 0;
                for (int t = 0; t < p.nterms; ++t) e += (__popcll(x & p.z[t]) & 1) ? -p.c[t] : p.c[t];
                R sn, cs;
                sincos_r(-p.theta * e, &sn, &cs);
                f.x = cs;
                f.y = sn;
            }
            C o;
            o.x = f.x * a[j].x - f.y * a[j].y;
            o.y = f.x * a[j].y + f.y * a[j].x;
            psi[x] = o;
        }
    }
}

template <typename R>
int launch_pauli_phase(qsim_state *s, int nterms, const uint64_t *zmask, const double *coeff, double theta) {
    using C = typename CTe<R>::T;
    const int n = s->n;
    PhaseParams<R> p;
    memset(&p, 0, sizeof p);
    p.nterms = nterms;
    p.theta = R(theta);
    bool uniform = true;
    for (int t = 0; t < nterms; ++t)
        if (coeff[t] != coeff[0]) uniform = false;
    p.nbytes = (n + 7) / 8;
    if (nterms <= PAR_TERMS) {
        p.mode = uniform ? 0 : 1;
        p.ngroups = (nterms + GROUP_TERMS - 1) / GROUP_TERMS;
        std::vector<uint64_t> pt(size_t(p.nbytes) * 256, 0);
        for (int b = 0; b < p.nbytes; ++b)
            for (int v = 0; v < 256; ++v) {
                uint64_t m = 0;
                for (int t = 0; t < nterms; ++t)
                    if (__builtin_popcountll((zmask[t] >> (8 * b)) & uint64_t(v)) & 1) m |= uint64_t(1) << t;
                pt[size_t(b) * 256 + size_t(v)] = m;
            }
        std::vector<C> ft;
        auto phase = [&](double e) {
            const std::complex<double> f = std::exp(std::complex<double>(0.0, -theta * e));
            C z;
            z.x = R(f.real());
            z.y = R(f.imag());
            return z;
        };
        if (uniform) {
            for (int k = 0; k <= nterms; ++k) ft.push_back(phase(coeff[0] * double(nterms - 2 * k)));
        } else {
            for (int g = 0; g < p.ngroups; ++g)
                for (int m = 0; m < 256; ++m) {
                    double e = 0;
                    for (int t = g * GROUP_TERMS; t < std::min(nterms, (g + 1) * GROUP_TERMS); ++t)
                        e += ((m >> (t - g * GROUP_TERMS)) & 1) ? -coeff[t] : coeff[t];
                    ft.push_back(phase(e));
                }
        }
        const size_t pbytes = pt.size() * sizeof(uint64_t), fbytes = ft.size() * sizeof(C);
        QSIM_TRY(s->ensure_scratch(pbytes + fbytes + 256));
        char *buf = static_cast<char *>(s->scratch);
        QSIM_CUDA_TRY(cudaMemcpyAsync(buf, pt.data(), pbytes, cudaMemcpyHostToDevice, s->stream), "phase tables");
        QSIM_CUDA_TRY(cudaMemcpyAsync(buf + ((pbytes + 255) & ~size_t(255)), ft.data(), fbytes,
                                      cudaMemcpyHostToDevice, s->stream),
                      "phase tables");
        // pageable sources: the copies are staged before the calls return, and
        // stream order keeps a later call's tables behind this launch
        p.ptab = reinterpret_cast<const uint64_t *>(buf);
        p.ftab = reinterpret_cast<const C *>(buf + ((pbytes + 255) & ~size_t(255)));
    } else {
        p.mode = 2;
        for (int t = 0; t < nterms; ++t) {
            p.z[t] = zmask[t];
            p.c[t] = R(coeff[t]);
        }
    }
    const uint64_t N = uint64_t(1) << n;
    constexpr int PER = 4, T = 256;
    const int sms = device_sm_count();
    const uint64_t blocks = std::min<uint64_t>((N + T * PER - 1) / (T * PER), uint64_t(std::max(sms, 1)) * 8);
    LaunchScope ls(K_PAULI_PHASE, s->stream, 2.0 * double(N) * sizeof(C), 6.0 * double(N));
    k_pauli_phase<R, PER><<<unsigned(blocks), T, 0, s->stream>>>(static_cast<C *>(s->amps), N, p);
    QSIM_CUDA_TRY(cudaGetLastError(), "pauli phase launch");
    return QSIM_OK;
}

}  // namespace
}  // namespace qsim

using namespace qsim;

extern "C" int qsim_apply_pauli_phase(qsim_state *s, int nterms, const uint64_t *zmask, const double *coeff,
                                      double theta) {
    if (!s) return set_error(QSIM_EINVAL, "state is NULL");
    if (nterms < 0 || nterms > MAX_PHASE_TERMS)
        return set_error(QSIM_EINVAL, "nterms=%d outside 0..%d", nterms, MAX_PHASE_TERMS);
    if (nterms > 0 && (!zmask || !coeff)) return set_error(QSIM_EINVAL, "NULL term arrays");
    const uint64_t full = (uint64_t(1) << s->n) - 1;
    for (int t = 0; t < nterms; ++t)
        if (zmask[t] & ~full) return set_error(QSIM_EINVAL, "term %d acts outside the state", t);
    if (nterms == 0) return QSIM_OK;
    return s->dtype == QSIM_C64 ? launch_pauli_phase<float>(s, nterms, zmask, coeff, theta)
                                : launch_pauli_phase<double>(s, nterms, zmask, coeff, theta);
}

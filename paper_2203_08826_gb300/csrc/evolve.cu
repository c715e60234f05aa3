// Diagonal Pauli-sum evolution: psi <- exp(-i theta D) psi with
// D = sum_t c_t Z(z_t), the diagonal factor of a Trotter step (Sec. 3.3: the
// time evolution is decomposed into a circuit of unitary gates; for the TFIM
// the sum of Z_i Z_{i+1} terms is diagonal and its exponential is one phase
// per amplitude).  One HBM pass per call whatever the number of terms:
// D(x) = sum_t c_t (-1)^popcount(x & z_t).  When every coefficient is the
// same, D(x) = c (T - 2 k(x)) with k(x) the number of terms of odd parity, and
// the T + 1 possible phases come from a table built on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>

#include "internal.h"

namespace qsim {
namespace {

constexpr int MAX_PHASE_TERMS = 128;

template <typename R> struct CTe;
template <> struct CTe<float> { using T = float2; };
template <> struct CTe<double> { using T = double2; };

template <typename R> struct PhaseParams {
    using C = typename CTe<R>::T;
    int nterms;
    int uniform;                    // 1: the table path
    uint64_t z[MAX_PHASE_TERMS];
    R c[MAX_PHASE_TERMS];
    R theta;
    C table[MAX_PHASE_TERMS + 1];   // uniform: exp(-i theta c (T - 2k)), k = 0..T
};

__device__ __forceinline__ void sincos_r(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_r(double a, double *s, double *c) { sincos(a, s, c); }

template <typename R, int PER>
__global__ void __launch_bounds__(256) k_pauli_phase(typename CTe<R>::T *__restrict__ psi, uint64_t N,
                                                     const __grid_constant__ PhaseParams<R> p) {
    using C = typename CTe<R>::T;
    const uint64_t base = uint64_t(blockIdx.x) * (blockDim.x * PER) + threadIdx.x;
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
        if (p.uniform) {
            int k = 0;
            for (int t = 0; t < p.nterms; ++t) k += __popcll(x & p.z[t]) & 1;
            f = p.table[k];
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

template <typename R>
int launch_pauli_phase(void *psi, int n, int nterms, const uint64_t *zmask, const double *coeff, double theta,
                       cudaStream_t st) {
    using C = typename CTe<R>::T;
    PhaseParams<R> p;
    memset(&p, 0, sizeof p);
    p.nterms = nterms;
    p.theta = R(theta);
    bool uniform = nterms > 0;
    for (int t = 0; t < nterms; ++t) {
        p.z[t] = zmask[t];
        p.c[t] = R(coeff[t]);
        if (coeff[t] != coeff[0]) uniform = false;
    }
    p.uniform = uniform ? 1 : 0;
    if (uniform)
        for (int k = 0; k <= nterms; ++k) {
            const std::complex<double> f = std::exp(std::complex<double>(0.0, -theta * coeff[0] * double(nterms - 2 * k)));
            p.table[k].x = R(f.real());
            p.table[k].y = R(f.imag());
        }
    const uint64_t N = uint64_t(1) << n;
    constexpr int PER = 4, T = 256;
    const uint64_t blocks = (N + T * PER - 1) / (T * PER);
    LaunchScope ls(K_PAULI_PHASE, st, 2.0 * double(N) * sizeof(C), 6.0 * double(N));
    k_pauli_phase<R, PER><<<unsigned(blocks), T, 0, st>>>(static_cast<C *>(psi), N, p);
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
    return s->dtype == QSIM_C64 ? launch_pauli_phase<float>(s->amps, s->n, nterms, zmask, coeff, theta, s->stream)
                                : launch_pauli_phase<double>(s->amps, s->n, nterms, zmask, coeff, theta, s->stream);
}

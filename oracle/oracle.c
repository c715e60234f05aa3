/*
 * Plain complex128 CPU oracle for the state-vector gate-application path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header or table with the CUDA
 * path.  It is written to be checked by eye against the paper, not to be fast:
 * every function loops over the full index space in the most literal order.
 *
 * Conventions (the paper fixes none of them; they are the library's):
 *   - qubit q is bit q of the amplitude index (qubit 0 is the least
 *     significant bit), as in the single-qubit kernel listing of Sec. 2 where
 *     the partner index is found by adding 1 << target;
 *   - for a k-qubit gate with targets[0..k-1], targets[0] is the MOST
 *     significant bit of the row/column index of G, so G(tau_1..tau_k,
 *     tau_1'..tau_k') of Eq. (1) reads tau_1 from targets[0];
 *   - a control qubit must be 1 for the gate to act.
 */
#include <complex.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_MAX_TARGETS 10

/* offset of the amplitude that carries matrix index j (targets[0] = MSB) */
static uint64_t target_offset(uint64_t j, const int *targets, int k) {
    uint64_t off = 0;
    for (int i = 0; i < k; ++i)
        if ((j >> (k - 1 - i)) & 1u) off |= (uint64_t)1 << targets[i];
    return off;
}

static int check_qubits(int n, const int *targets, int k, const int *controls,
                        int c) {
    if (n < 1 || n > 40 || k < 0 || k > ORC_MAX_TARGETS || c < 0 || c > n)
        return -1;
    uint64_t seen = 0;
    for (int i = 0; i < k; ++i) {
        if (targets[i] < 0 || targets[i] >= n) return -1;
        if (seen >> targets[i] & 1u) return -1;
        seen |= (uint64_t)1 << targets[i];
    }
    for (int i = 0; i < c; ++i) {
        if (controls[i] < 0 || controls[i] >= n) return -1;
        if (seen >> controls[i] & 1u) return -1;
        seen |= (uint64_t)1 << controls[i];
    }
    return 0;
}

/*
 * Eq. (1): psi'(..tau..) = sum_tau' G(tau, tau') psi(..tau'..), restricted to
 * the indices whose control bits are all 1 (controlled gates, Sec. 2).
 * For every index x whose target bits are all 0 (and control bits all 1) the
 * 2^k amplitudes x | bits(tau') are gathered, multiplied by G and written back
 * in place.  G is row-major complex128, 2^k x 2^k.
 */
int orc_apply_gate(cplx *psi, int n, const cplx *G, const int *targets, int k,
                   const int *controls, int c) {
    if (check_qubits(n, targets, k, controls, c)) return -1;
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t d = (uint64_t)1 << k;
    uint64_t tmask = 0, cmask = 0;
    for (int i = 0; i < k; ++i) tmask |= (uint64_t)1 << targets[i];
    for (int i = 0; i < c; ++i) cmask |= (uint64_t)1 << controls[i];
    uint64_t offs[1 << ORC_MAX_TARGETS];
    for (uint64_t j = 0; j < d; ++j) offs[j] = target_offset(j, targets, k);

#pragma omp parallel for schedule(static)
    for (int64_t xs = 0; xs < (int64_t)N; ++xs) {
        const uint64_t x = (uint64_t)xs;
        if (x & tmask) continue;
        if ((x & cmask) != cmask) continue;
        cplx v[1 << ORC_MAX_TARGETS];
        cplx w[1 << ORC_MAX_TARGETS];
        for (uint64_t j = 0; j < d; ++j) v[j] = psi[x | offs[j]];
        for (uint64_t r = 0; r < d; ++r) {
            cplx acc = 0;
            for (uint64_t j = 0; j < d; ++j) acc += G[r * d + j] * v[j];
            w[r] = acc;
        }
        for (uint64_t r = 0; r < d; ++r) psi[x | offs[r]] = w[r];
    }
    return 0;
}

/*
 * Marginal probabilities of the qubits listed in qubits[0..m-1]:
 * out[y] = sum over x whose listed bits spell y of |psi(x)|^2, where
 * qubits[0] is the most significant bit of y (the same order as targets).
 * With m = n and qubits = (n-1, ..., 0) this is p(x) = |psi(x)|^2.
 */
int orc_marginal_probs(const cplx *psi, int n, const int *qubits, int m,
                       double *out) {
    if (n < 1 || n > 40 || m < 0 || m > n || m > 30) return -1;
    uint64_t seen = 0;
    for (int i = 0; i < m; ++i) {
        if (qubits[i] < 0 || qubits[i] >= n || (seen >> qubits[i] & 1u)) return -1;
        seen |= (uint64_t)1 << qubits[i];
    }
    const uint64_t N = (uint64_t)1 << n;
    memset(out, 0, sizeof(double) * ((size_t)1 << m));
    for (uint64_t x = 0; x < N; ++x) {
        uint64_t y = 0;
        for (int i = 0; i < m; ++i) y = (y << 1) | ((x >> qubits[i]) & 1u);
        const double re = creal(psi[x]), im = cimag(psi[x]);
        out[y] += re * re + im * im;
    }
    return 0;
}

/*
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11, Sec. 4): ten rounds of the 4x32 Philox S-box with the
 * multipliers 0xD2511F53 and 0xCD9E8D57 and the Weyl key increments
 * 0x9E3779B9 and 0xBB67AE85 applied between rounds.
 */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n1 = lo1;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        const uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    memcpy(out, c, sizeof c);
}

/* integer weight of one probability: floor(p * 2^62), 0 for p <= 0 or NaN */
static uint64_t prob_weight(double p) {
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 62;
    return (uint64_t)(p * 4611686018427387904.0); /* 2^62, exact scaling */
}

/*
 * Shot sampling by inverse CDF.  Sec. 2 samples shots with a Metropolis
 * chain, whose output is not unique; inverse-CDF sampling over integer
 * weights with a counter-based generator gives shots that two
 * implementations can reproduce bit for bit.
 *   w(x)   = floor(p(x) 2^62)              (integer weights)
 *   CDF(x) = w(0) + ... + w(x),  T = CDF(N-1)
 *   shot s: (o0,o1,o2,o3) = Philox4x32-10(counter = (lo32(c0+s), hi32(c0+s), 0, 0),
 *                                       key = (lo32(seed), hi32(seed)))
 *           u = o1 * 2^32 + o0,   r = floor(u * T / 2^64)
 *           out[s] = smallest x with CDF(x) > r
 * Returns -1 if the probabilities sum to more than 1.5 or to zero.
 */
int orc_sample(const double *p, uint64_t N, uint64_t nshots, uint64_t seed,
               uint64_t counter0, uint64_t *out) {
    if (N == 0) return -1;
    double psum = 0.0;
    for (uint64_t x = 0; x < N; ++x) psum += (p[x] > 0.0 ? p[x] : 0.0);
    if (!(psum <= 1.5)) return -1;
    uint64_t *cdf = (uint64_t *)malloc(sizeof(uint64_t) * N);
    if (!cdf) return -2;
    uint64_t run = 0;
    for (uint64_t x = 0; x < N; ++x) {
        run += prob_weight(p[x]);
        cdf[x] = run;
    }
    const uint64_t T = run;
    if (T == 0) {
        free(cdf);
        return -1;
    }
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint64_t s = 0; s < nshots; ++s) {
        const uint64_t cs = counter0 + s;
        const uint32_t ctr[4] = {(uint32_t)cs, (uint32_t)(cs >> 32), 0u, 0u};
        uint32_t o[4];
        orc_philox4x32_10(ctr, key, o);
        const uint64_t u = ((uint64_t)o[1] << 32) | o[0];
        const uint64_t r = (uint64_t)(((unsigned __int128)u * T) >> 64);
        /* smallest x with cdf[x] > r: plain binary search on the sorted CDF */
        uint64_t lo = 0, hi = N - 1;
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > r) hi = mid;
            else lo = mid + 1;
        }
        out[s] = lo;
    }
    free(cdf);
    return 0;
}

/* Threads used by the Eq. (1) loop from now on (timing the oracle on one core
 * or on all of them); returns the previous setting. */
int orc_set_threads(int nthreads) {
    const int prev = omp_get_max_threads();
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return prev;
}

// Tensor-core fused k-qubit blocks (QSIM_FUSE_TC), complex64 states.
//
// A dense k-qubit block on the k lowest bits of the index is the contraction
// of Eq. (1) for every row of the (2^(n-k) x 2^k) matrix view of the state:
// psi'[r, c] = sum_c' G[c, c'] psi[r, c'].  With amplitudes interleaved
// (re, im) a row is 2^(k+1) reals and the complex product becomes one real
// GEMM  D = A * B^T  with A = rows (M = 128 per tile, K = 2^(k+1)) and the
// real-ified gate B[N = 2^(k+1), K]:
//   B[2c  ][2c'] =  Re G[c,c'],  B[2c  ][2c'+1] = -Im G[c,c'],
//   B[2c+1][2c'] =  Im G[c,c'],  B[2c+1][2c'+1] =  Re G[c,c'].
// The fp32 state is split into two low-precision parts a = a_hi + a_lo and
// the product is taken as A_hi B_hi + A_hi B_lo + A_lo B_hi (the a_lo b_lo term
// is below fp32 rounding of the result's scale), on the 5th-generation tensor
// cores: tcgen05.mma with operands in shared memory (128-byte swizzled K-major
// layout), the fp32 accumulator in tensor memory, completion signalled through
// an mbarrier.  Two splits are built: BF16x3 (kind::f16) and 3xTF32
// (kind::tf32).
//
// Each pass writes its output with the index rotated right by k bits,
// out[(c << (n-k)) | r] = D[r, c], into a second buffer: the next pass then
// finds the next k qubits in the low bits, and the warp that owns 32
// consecutive rows stores 32 consecutive amplitudes per column.  A plan is a
// sequence of such passes whose widths add up to a multiple of n, so the
// final index order is the natural one.  Diagonal gates whose qubits straddle
// the block are applied to the output in the epilogue, where the full index of
// every element is known.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"
#include "plan.h"

namespace qsim {

namespace {

constexpr int TC_M = 128;          // rows per tile (tcgen05 M)
// warp roles: 4 epilogue warps (warp w reads TMEM lanes 32w..32w+31), one
// MMA warp (also allocates TMEM), 8 producer warps
constexpr int TC_EPI_WARPS = 4;
constexpr int TC_MMA_WARP = 4;
constexpr int TC_PROD_WARPS = 8;
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 1 + TC_PROD_WARPS);
constexpr int TC_PROD_THREADS = 32 * TC_PROD_WARPS;
constexpr int MAX_EPI = 48;        // epilogue diagonal ops per pass
constexpr int MAX_EPI_POOL = 256;  // their complex entries
constexpr unsigned long long WAIT_LIMIT = 1ull << 26;  // bounded mbarrier waits

// per-pass arithmetic: BF16x3 or 3xTF32 on the tensor cores, or the same
// contraction in FP32 on the CUDA cores (k_rot_simt)
enum TcPrec { TC_BF16X3 = 0, TC_TF32X3 = 1, TC_FP32 = 2 };

struct EpiOp {
    uint64_t cmask;  // control bits (current index) that must all be 1
    int k;           // selector bits
    int sel[QSIM_MAX_TARGETS];  // current-index bit of selector t (t = 0 is the MSB)
    int moff;        // entries in the pool (2^k complex)
    int neg;         // 1: k == 0 and the factor is exactly -1
};

struct TcParams {
    const float2 *in;
    float2 *out;
    const uint4 *bimg;   // shared-memory image of B_hi then B_lo
    int *err;            // set to 1 when a bounded wait expires
    unsigned long long wait_limit;  // polls of a pipeline wait before it gives up
    uint64_t ntiles;     // 2^(n-k) / 128
    int n;
    int nepi;               // phase ops (evaluated per element)
    int nneg;               // sign flips on a control subspace: row mask + column flip mask
    EpiOp epi[MAX_EPI];
    uint64_t negr[MAX_EPI];  // bits of the row index R that must all be 1
    uint64_t negc[MAX_EPI];  // bit c set: column c is negated (when the row bits hold)
    float2 pool[MAX_EPI_POOL];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFF) >> 4);
    d |= uint64_t(1) << 16;             // leading byte offset (unused with swizzle)
    d |= uint64_t(1024 >> 4) << 32;     // stride byte offset
    d |= uint64_t(1) << 46;             // version
    d |= uint64_t(2) << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor: D fp32, A/B bf16 (1) or tf32 (2), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
template <int PREC>
__host__ __device__ constexpr uint32_t tc_idesc(int N, int M) {
    return (1u << 4) | (uint32_t(PREC == TC_BF16X3 ? 1 : 2) << 7) | (uint32_t(PREC == TC_BF16X3 ? 1 : 2) << 10) |
           (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Byte offset of element (row m, k-element e) in a swizzled K-major operand
// made of 128-byte-wide column blocks, each rows*128 bytes.
template <int EB>
__host__ __device__ inline uint32_t sw128_offset(int m, int e, int rows) {
    const int per_row = 128 / EB;  // elements per 128-byte row of a column block
    const int blk = e / per_row;
    const uint32_t byte = uint32_t(e % per_row) * EB;
    const uint32_t chunk = byte >> 4, within = byte & 15;
    return uint32_t(blk) * uint32_t(rows) * 128u + uint32_t(m / 8) * 1024u + uint32_t(m % 8) * 128u +
           ((chunk ^ uint32_t(m % 8)) << 4) + within;
}

template <int PREC> struct Elem;
template <> struct Elem<TC_BF16X3> {
    static constexpr int EB = 2;
    __device__ static void split(float a, uint16_t &hi, uint16_t &lo) {
        const __nv_bfloat16 h = __float2bfloat16_rn(a);
        const __nv_bfloat16 l = __float2bfloat16_rn(a - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
};
// Round a float to the nearest tf32 value (10 fraction bits; ties away from
// zero in magnitude): add half of the dropped range to the magnitude bits,
// then clear them.  The tensor cores read only the top 19 bits of a tf32
// operand, so a part given with more bits would be truncated toward zero;
// rounding both parts here keeps the split unbiased.
__host__ __device__ inline uint32_t tf32_rn(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }

template <> struct Elem<TC_TF32X3> {
    static constexpr int EB = 4;
    __device__ static void split(float a, uint32_t &hi, uint32_t &lo) {
        const uint32_t h = tf32_rn(__float_as_uint(a));
        hi = h;
        lo = tf32_rn(__float_as_uint(a - __uint_as_float(h)));  // a - hi is exact in fp32
    }
};

template <int K, int PREC>
struct TcShape {
    static constexpr int KR = 2 << K;                   // reals per row (GEMM K and N)
    static constexpr int EB = Elem<PREC>::EB;
    static constexpr int OPND = TC_M * KR * EB;         // bytes of one A split
    static constexpr int BOPND = KR * KR * EB;          // bytes of one B split
    static constexpr int STAGES = 2;                    // A operand buffers (hi + lo each)
    static constexpr int BAR_OFF = 2 * BOPND + STAGES * 2 * OPND;
    static constexpr int EPI_OFF = BAR_OFF + 128;       // epilogue ops copied from the parameters
    static constexpr int EPI_BYTES = 2 * MAX_EPI * 8 + MAX_EPI * int(sizeof(EpiOp)) + MAX_EPI_POOL * 8;
    static constexpr int SMEM = EPI_OFF + EPI_BYTES + 1024;  // + alignment slack
    static constexpr int TCOLS = 2 * KR < 32 ? 32 : 2 * KR;  // two accumulators (power of 2)
    static constexpr int KSTEP = 32 / EB;               // K elements per MMA
    static constexpr int NV = TC_M * KR / 4;            // float4 per fp32 tile
    static constexpr int PER = NV / TC_PROD_THREADS;    // float4 per producer thread
    static_assert(SMEM <= 227 * 1024, "tensor-core tile does not fit shared memory");
    static_assert(NV % TC_PROD_THREADS == 0, "tile not divisible among producers");
};

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (unsigned long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Bounded wait that also gives up as soon as another role has given up
// (*abort set); on its own expiry it sets *abort.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t mbar, uint32_t parity, volatile int *abort,
                                             unsigned long long limit) {
    for (unsigned long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 31) == 31 && *abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Every lane of a warp waits; the warp goes on only if all lanes saw the
// phase complete, so its lanes never leave a loop in different iterations.
__device__ __forceinline__ bool warp_wait(uint32_t mbar, uint32_t parity, volatile int *abort,
                                          unsigned long long limit) {
    const bool ok = mbar_wait_ab(mbar, parity, abort, limit);
    return __all_sync(0xffffffffu, ok);
}

// Persistent, warp-specialised CTA (one per SM).  Tile i (rows of the
// (2^(n-k) x 2^k) view, CTAs take every gridDim.x-th tile) moves through
//   producers: global fp32 -> registers -> hi/lo split -> A stage i % 2
//   MMA thread: A stage + B -> accumulator i % 2 in TMEM (3 products)
//   epilogue:   accumulator -> diagonal epilogue ops -> rotated global store
// with one mbarrier per hand-off and direction: full_a / empty_a per A stage
// (producers -> MMA, MMA commit -> producers), full_acc / empty_acc per
// accumulator (MMA commit -> epilogue, epilogue -> MMA).  Two of each let the
// loads of tile i + 1 and the stores of tile i - 1 overlap the MMAs of tile i.
template <int K, int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_block(const __grid_constant__ TcParams p) {
    using S = TcShape<K, PREC>;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    unsigned char *b_hi = sm;
    unsigned char *b_lo = sm + S::BOPND;
    auto a_hi = [&](int st) { return sm + 2 * S::BOPND + st * 2 * S::OPND; };
    auto a_lo = [&](int st) { return sm + 2 * S::BOPND + st * 2 * S::OPND + S::OPND; };
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + S::BAR_OFF);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 8);
    volatile int *abort_f = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t full_a0 = smem_u32(&bars[0]), empty_a0 = smem_u32(&bars[2]);
    const uint32_t full_acc0 = smem_u32(&bars[4]), empty_acc0 = smem_u32(&bars[6]);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    uint64_t *s_negr = reinterpret_cast<uint64_t *>(sm + S::EPI_OFF);
    uint64_t *s_negc = s_negr + MAX_EPI;
    EpiOp *s_epi = reinterpret_cast<EpiOp *>(s_negc + MAX_EPI);
    float2 *s_pool = reinterpret_cast<float2 *>(s_epi + MAX_EPI);
    {  // B (both splits): the host built the swizzled image
        const uint4 *src = p.bimg;
        uint4 *dst = reinterpret_cast<uint4 *>(b_hi);
        for (int i = tid; i < 2 * S::BOPND / 16; i += TC_THREADS) dst[i] = src[i];
        for (int i = tid; i < p.nneg; i += TC_THREADS) {
            s_negr[i] = p.negr[i];
            s_negc[i] = p.negc[i];
        }
        for (int i = tid; i < p.nepi; i += TC_THREADS) s_epi[i] = p.epi[i];
        for (int i = tid; i < MAX_EPI_POOL; i += TC_THREADS) s_pool[i] = p.pool[i];
    }
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full_a0 + 8 * st), "r"(TC_PROD_WARPS));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty_a0 + 8 * st));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full_acc0 + 8 * st));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty_acc0 + 8 * st), "r"(TC_EPI_WARPS));
        }
        *abort_f = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == TC_MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(S::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B image -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const int n = p.n;
    const uint64_t my_tiles = blockIdx.x < p.ntiles ? (p.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (warp > TC_MMA_WARP) {
        // ---------------- producers
        // Software-pipelined by half tiles: while one half of tile i is split
        // into the operands, the same half of tile i + 1 is already loading.
        const int pt = tid - 32 * (TC_MMA_WARP + 1);
        constexpr int PH = S::PER / 2;
        static_assert(S::PER % 2 == 0, "half tiles");
        auto load_half = [&](float4 (&v)[PH], uint64_t i, int h) {
            const uint64_t tile = blockIdx.x + i * gridDim.x;
            const float4 *src = reinterpret_cast<const float4 *>(p.in) + tile * uint64_t(S::NV);
#pragma unroll
            for (int j = 0; j < PH; ++j) v[j] = __ldcs(src + pt + (h * PH + j) * TC_PROD_THREADS);
        };
        auto convert_half = [&](const float4 (&v)[PH], int st, int h) {
            unsigned char *ah = a_hi(st), *al = a_lo(st);
#pragma unroll
            for (int j = 0; j < PH; ++j) {
                const int vi = pt + (h * PH + j) * TC_PROD_THREADS;
                const int m = (vi * 4) / S::KR, e = (vi * 4) % S::KR;
                if (PREC == TC_BF16X3) {
                    uint16_t hh[4], ll[4];
                    Elem<TC_BF16X3>::split(v[j].x, hh[0], ll[0]);
                    Elem<TC_BF16X3>::split(v[j].y, hh[1], ll[1]);
                    Elem<TC_BF16X3>::split(v[j].z, hh[2], ll[2]);
                    Elem<TC_BF16X3>::split(v[j].w, hh[3], ll[3]);
                    const uint32_t off = sw128_offset<2>(m, e, TC_M);
                    *reinterpret_cast<uint2 *>(ah + off) =
                        make_uint2(hh[0] | (uint32_t(hh[1]) << 16), hh[2] | (uint32_t(hh[3]) << 16));
                    *reinterpret_cast<uint2 *>(al + off) =
                        make_uint2(ll[0] | (uint32_t(ll[1]) << 16), ll[2] | (uint32_t(ll[3]) << 16));
                } else {
                    uint32_t hh[4], ll[4];
                    Elem<TC_TF32X3>::split(v[j].x, hh[0], ll[0]);
                    Elem<TC_TF32X3>::split(v[j].y, hh[1], ll[1]);
                    Elem<TC_TF32X3>::split(v[j].z, hh[2], ll[2]);
                    Elem<TC_TF32X3>::split(v[j].w, hh[3], ll[3]);
                    const uint32_t off = sw128_offset<4>(m, e, TC_M);
                    *reinterpret_cast<uint4 *>(ah + off) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
                    *reinterpret_cast<uint4 *>(al + off) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
                }
            }
        };
        float4 v0[PH], v1[PH];
        if (my_tiles > 0) {
            load_half(v0, 0, 0);
            load_half(v1, 0, 1);
        }
        for (uint64_t i = 0; i < my_tiles; ++i) {
            const int st = int(i & 1);
            const uint32_t u = uint32_t(i >> 1);
            const bool more = i + 1 < my_tiles;
            if (i >= 2 && !warp_wait(empty_a0 + 8 * st, (u - 1) & 1, abort_f, p.wait_limit)) break;
            convert_half(v0, st, 0);
            if (more) load_half(v0, i + 1, 0);
            convert_half(v1, st, 1);
            // generic-proxy writes -> visible to the tensor core (async proxy)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(full_a0 + 8 * st);
            if (more) load_half(v1, i + 1, 1);
        }
    } else if (warp == TC_MMA_WARP) {
        // ---------------- MMA issue (one thread)
        if (lane == 0) {
            constexpr uint32_t IDESC = tc_idesc<PREC>(S::KR, TC_M);
            constexpr int PERB = 128 / S::EB;  // elements per 128-byte column block
            const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
            uint64_t issued = 0;
            for (uint64_t i = 0; i < my_tiles; ++i) {
                const int st = int(i & 1);
                const uint32_t u = uint32_t(i >> 1);
                if (!mbar_wait_ab(full_a0 + 8 * st, u & 1, abort_f, p.wait_limit)) break;
                if (i >= 2 && !mbar_wait_ab(empty_acc0 + 8 * st, (u - 1) & 1, abort_f, p.wait_limit)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t ah = smem_u32(a_hi(st)), al = smem_u32(a_lo(st));
                const uint32_t dacc = tmem + uint32_t(st * S::KR);
                int acc = 0;
#pragma unroll
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t A = pass == 2 ? al : ah;
                    const uint32_t B = pass == 1 ? bl : bh;
#pragma unroll
                    for (int ks = 0; ks < S::KR / S::KSTEP; ++ks) {
                        const int e = ks * S::KSTEP;
                        const uint32_t aoff = uint32_t(e / PERB) * TC_M * 128 + uint32_t(e % PERB) * S::EB;
                        const uint32_t boff = uint32_t(e / PERB) * S::KR * 128 + uint32_t(e % PERB) * S::EB;
                        const uint64_t ad = sw128_desc(A + aoff), bd = sw128_desc(B + boff);
                        if (PREC == TC_BF16X3)
                            asm volatile(
                                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(dacc),
                                "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                        else
                            asm volatile(
                                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}" ::"r"(dacc),
                                "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
                        acc = 1;
                    }
                }
                // completion frees the A stage and fills the accumulator
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 empty_a0 + 8 * st)
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 full_acc0 + 8 * st)
                             : "memory");
                issued = i + 1;
            }
            // no MMA may be in flight at teardown: wait (bounded) for the last
            // commit of each stage
            for (uint64_t i = issued >= 2 ? issued - 2 : 0; i < issued; ++i)
                mbar_wait(empty_a0 + 8 * int(i & 1), uint32_t(i >> 1) & 1);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: TMEM lane = row of the tile
        const int m = warp * 32 + lane;
        for (uint64_t i = 0; i < my_tiles; ++i) {
            const uint64_t tile = blockIdx.x + i * gridDim.x;
            const int st = int(i & 1);
            const uint32_t u = uint32_t(i >> 1);
            if (!warp_wait(full_acc0 + 8 * st, u & 1, abort_f, p.wait_limit)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t R = tile * TC_M + m;  // row index = bits K.. of the current index
            const uint32_t trow = tmem + uint32_t(st * S::KR) + (uint32_t(warp * 32) << 16);
            // sign flips: one 64-bit column mask per row
            uint64_t flip = 0;
            for (int e = 0; e < p.nneg; ++e)
                if ((R & s_negr[e]) == s_negr[e]) flip ^= s_negc[e];
            const int nph = p.nepi;
#pragma unroll 1
            for (int c0 = 0; c0 < S::KR; c0 += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(trow + uint32_t(c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float2 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = c0 / 2 + j;  // complex column = low K bits of the current index
                    v[j] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
                    if ((flip >> c) & 1) {
                        v[j].x = -v[j].x;
                        v[j].y = -v[j].y;
                    }
                    if (nph) {
                        const uint64_t x = (R << K) | uint64_t(c);
                        for (int e = 0; e < nph; ++e) {
                            const EpiOp &op = s_epi[e];
                            if ((x & op.cmask) != op.cmask) continue;
                            int s = 0;
                            for (int t = 0; t < op.k; ++t) s = (s << 1) | int((x >> op.sel[t]) & 1);
                            const float2 f = s_pool[op.moff + s];
                            v[j] = make_float2(f.x * v[j].x - f.y * v[j].y, f.x * v[j].y + f.y * v[j].x);
                        }
                    }
                }
                // 16-byte stores of two consecutive rows: lanes 2m and 2m+1
                // trade one value per column pair (c, c + 1); the even lane
                // writes column c, the odd lane column c + 1, both at row 2m
                const bool odd = lane & 1;
                const uint64_t R0 = R & ~uint64_t(1);
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    const int c = c0 / 2 + j;
                    const float2 send = odd ? v[j] : v[j + 1];
                    float2 recv;
                    recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
                    recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
                    const float4 w = odd ? make_float4(recv.x, recv.y, v[j + 1].x, v[j + 1].y)
                                         : make_float4(v[j].x, v[j].y, recv.x, recv.y);
                    const uint64_t col = uint64_t(odd ? c + 1 : c);
                    __stcs(reinterpret_cast<float4 *>(&p.out[(col << (n - K)) | R0]), w);
                }
            }
            // the accumulator may be overwritten by the MMAs of tile i + 2
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_acc0 + 8 * st);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0 && *abort_f) atomicExch(p.err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == TC_MMA_WARP)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TCOLS));
}

// The FP32 CUDA-core form of a pass: the same contraction, epilogue and
// rotated store as k_tc_block, with the block matrix (complex64, row-major)
// broadcast from shared memory.  A CTA of 128 threads loads 128 consecutive
// rows (one contiguous run of 128 * 2^K amplitudes) into a padded shared
// tile, each thread takes one row into registers and forms its 2^K outputs;
// for each output column the 128 threads store 128 consecutive amplitudes.
template <int K>
__global__ void __launch_bounds__(128) k_rot_simt(const __grid_constant__ TcParams p, const float2 *__restrict__ G) {
    constexpr int D = 1 << K;
    constexpr int ROWS = 128;
    extern __shared__ __align__(16) unsigned char simt_smem[];
    float2 *gm = reinterpret_cast<float2 *>(simt_smem);
    float2 *tile = gm + D * D;  // ROWS x (D + 1)
    uint64_t *s_negr = reinterpret_cast<uint64_t *>(tile + ROWS * (D + 1));
    uint64_t *s_negc = s_negr + MAX_EPI;
    EpiOp *s_epi = reinterpret_cast<EpiOp *>(s_negc + MAX_EPI);
    float2 *s_pool = reinterpret_cast<float2 *>(s_epi + MAX_EPI);
    for (int i = threadIdx.x; i < D * D; i += ROWS) gm[i] = G[i];
    for (int i = threadIdx.x; i < p.nneg; i += ROWS) {
        s_negr[i] = p.negr[i];
        s_negc[i] = p.negc[i];
    }
    for (int i = threadIdx.x; i < p.nepi; i += ROWS) s_epi[i] = p.epi[i];
    for (int i = threadIdx.x; i < MAX_EPI_POOL; i += ROWS) s_pool[i] = p.pool[i];
    const int n = p.n;
    const uint64_t nrows = uint64_t(1) << (n - K);
    const int m = threadIdx.x;
    for (uint64_t r0 = uint64_t(blockIdx.x) * ROWS; r0 < nrows; r0 += uint64_t(gridDim.x) * ROWS) {
        __syncthreads();  // the matrix and tables are in place; the previous tile is consumed
        const float2 *src = p.in + (r0 << K);
        for (int i = threadIdx.x; i < ROWS * D; i += ROWS) tile[(i >> K) * (D + 1) + (i & (D - 1))] = __ldcs(src + i);
        __syncthreads();
        float2 v[D];
#pragma unroll
        for (int c = 0; c < D; ++c) v[c] = tile[m * (D + 1) + c];
        const uint64_t R = r0 + uint64_t(m);
        uint64_t flip = 0;
        for (int e = 0; e < p.nneg; ++e)
            if ((R & s_negr[e]) == s_negr[e]) flip ^= s_negc[e];
#pragma unroll 1
        for (int c = 0; c < D; ++c) {
            const float2 *row = gm + c * D;
            float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
            for (int j = 0; j < D; j += 2) {
                const float2 g0 = row[j], g1 = row[j + 1];
                ax = fmaf(g0.x, v[j].x, ax);
                ax = fmaf(-g0.y, v[j].y, ax);
                ay = fmaf(g0.x, v[j].y, ay);
                ay = fmaf(g0.y, v[j].x, ay);
                bx = fmaf(g1.x, v[j + 1].x, bx);
                bx = fmaf(-g1.y, v[j + 1].y, bx);
                by = fmaf(g1.x, v[j + 1].y, by);
                by = fmaf(g1.y, v[j + 1].x, by);
            }
            float2 o = make_float2(ax + bx, ay + by);
            if ((flip >> c) & 1) {
                o.x = -o.x;
                o.y = -o.y;
            }
            const uint64_t x = (R << K) | uint64_t(c);
            for (int e = 0; e < p.nepi; ++e) {
                const EpiOp &op = s_epi[e];
                if ((x & op.cmask) != op.cmask) continue;
                int sel = 0;
                for (int t = 0; t < op.k; ++t) sel = (sel << 1) | int((x >> op.sel[t]) & 1);
                const float2 f = s_pool[op.moff + sel];
                o = make_float2(f.x * o.x - f.y * o.y, f.x * o.y + f.y * o.x);
            }
            __stcs(&p.out[(uint64_t(c) << (n - K)) | R], o);
        }
    }
}

template <int K> constexpr int simt_smem_bytes() {
    return int(((1 << K) * (1 << K) + 128 * ((1 << K) + 1)) * sizeof(float2) + 2 * MAX_EPI * sizeof(uint64_t) +
               MAX_EPI * sizeof(EpiOp) + MAX_EPI_POOL * sizeof(float2));
}

}  // namespace

// ------------------------------------------------------------------ plan
struct TcPass {
    bool plain = false;          // a gate no window can hold, applied by a plain sweep
    Op op;                       // plain: the classified gate (original qubits)
    int k = 6;
    int off = 0;                 // original qubit held by bit 0 of the current index
    std::vector<cd> block;       // 2^k x 2^k on the window (index bit i = qubit off + i)
    struct Diag {
        std::vector<int> targets;  // original qubits (targets[0] = MSB of the entry index)
        std::vector<int> controls;
        std::vector<cd> d;
    };
    std::vector<Diag> epi;
    int ngates = 0;
    int prec = TC_BF16X3;        // arithmetic of this pass (TcPrec)
};

struct TcPlan {
    int prec = TC_BF16X3;
    std::vector<TcPass> passes;
    struct Dev {
        bool ready = false;
        void *bimg = nullptr;
        std::vector<size_t> boff;
        std::vector<TcParams> params;
        int *err = nullptr;
    } dev;
    ~TcPlan() {
        if (dev.bimg) cudaFree(dev.bimg);
        if (dev.err) cudaFree(dev.err);
    }
};

namespace {

// widths of consecutive passes: 6s and 5s (every total >= 20 is a sum of them)
bool split56(int total, std::vector<int> &out) {
    for (int b = total / 6; b >= 0; --b) {
        const int rest = total - 6 * b;
        if (rest % 5 == 0) {
            out.assign(b, 6);
            out.insert(out.end(), rest / 5, 5);
            return true;
        }
    }
    return false;
}

}  // namespace

int build_tc(const qsim_circuit &c, qsim_plan &p) {
    const int n = c.n;
    const int kw = p.kmax >= 6 ? 6 : 5;
    // a tile is 128 rows of the (2^(n-k) x 2^k) view
    if (n < kw + 7 || n > 34) return set_error(QSIM_EUNSUPPORTED, "tensor-core plans need %d <= n <= 34 qubits", kw + 7);
    TcPlan *tp = new TcPlan();
    p.tc = tp;
    tp->prec = kw == 6 ? TC_BF16X3 : TC_TF32X3;
    // classify gates
    std::vector<Op> ops(c.gates.size()), orig(c.gates.size());
    std::vector<bool> diag(c.gates.size());
    for (size_t i = 0; i < c.gates.size(); ++i) {
        const GateRec &g = c.gates[i];
        QSIM_TRY(classify(g.m, g.targets, g.k, g.controls, g.nc, ops[i]));
        orig[i] = ops[i];
        diag[i] = ops[i].type == Op::DIAG || ops[i].type == Op::IDENTITY;
        if (ops[i].type == Op::MONO) {
            const size_t d = size_t(1) << ops[i].k;
            ops[i].m.assign(d * d, cd(0.0));
            for (size_t r = 0; r < d; ++r) ops[i].m[r * d + ops[i].perm[r]] = ops[i].phase[r];
            ops[i].type = Op::DENSE;
        }
    }
    std::vector<int> remaining(c.gates.size());
    for (size_t i = 0; i < remaining.size(); ++i) remaining[i] = int(i);
    // does a gate fit one of the windows the planner will visit from offset
    // `from` on (offsets from + t k mod n)?
    auto fits_orbit = [&](const Op &op, int from, int k) {
        uint64_t q = 0;
        for (int t = 0; t < op.k; ++t) q |= uint64_t(1) << op.targets[t];
        for (int t = 0; t < op.c; ++t) q |= uint64_t(1) << op.controls[t];
        int o = from;
        for (int t = 0; t < n; ++t) {
            uint64_t w = 0;
            for (int i = 0; i < k; ++i) w |= uint64_t(1) << ((o + i) % n);
            if ((q & ~w) == 0) return true;
            o = (o + k) % n;
        }
        return false;
    };
    int off = 0, rotated = 0;
    int stall = 0;
    while (!remaining.empty()) {
        const int k = kw;
        {
            // the earliest pending gate fits no window (a SWAP or a 2- or
            // 3-qubit gate on distant qubits): one plain sweep, here, on the
            // current index order; the gates already taken past it act on
            // other qubits
            const int g0 = remaining.front();
            const Op &o0 = ops[g0];
            if (!diag[g0] && !fits_orbit(o0, off, k)) {
                const Op &og = orig[g0];
                if (og.type == Op::DENSE && og.k > 3)
                    return set_error(QSIM_EUNSUPPORTED, "tensor-core planner: a %d-qubit gate spans more than %d qubits",
                                     og.k, k);
                TcPass ps;
                ps.plain = true;
                ps.op = og;
                ps.off = off;
                ps.ngates = 1;
                tp->passes.push_back(std::move(ps));
                remaining.erase(remaining.begin());
                continue;
            }
        }
        TcPass ps;
        ps.k = k;
        ps.off = off;
        std::vector<int> win(k);
        uint64_t wmask = 0;
        for (int i = 0; i < k; ++i) {
            win[i] = (off + i) % n;
            wmask |= uint64_t(1) << win[i];
        }
        std::vector<int> qs(k);  // embedding order: MSB first
        for (int i = 0; i < k; ++i) qs[i] = win[k - 1 - i];
        ps.block.assign(size_t(1) << (2 * k), cd(0.0));
        for (size_t i = 0; i < (size_t(1) << k); ++i) ps.block[i * ((size_t(1) << k) + 1)] = 1.0;
        uint64_t blocked = 0;
        std::vector<int> rest;
        for (int gi : remaining) {
            const Op &op = ops[gi];
            uint64_t q = 0;
            for (int t = 0; t < op.k; ++t) q |= uint64_t(1) << op.targets[t];
            for (int t = 0; t < op.c; ++t) q |= uint64_t(1) << op.controls[t];
            if (q & blocked) {
                blocked |= q;
                rest.push_back(gi);
                continue;
            }
            if ((q & ~wmask) == 0) {
                // inside the window: multiply into the block (later gates on the left)
                GateRec gr;
                gr.k = op.k;
                gr.nc = op.c;
                for (int t = 0; t < op.k; ++t) gr.targets[t] = op.targets[t];
                for (int t = 0; t < op.c; ++t) gr.controls[t] = op.controls[t];
                if (op.type == Op::DENSE) {
                    gr.m = op.m;
                } else if (op.type == Op::DIAG) {
                    const size_t d = size_t(1) << op.k;
                    gr.m.assign(d * d, cd(0.0));
                    for (size_t r = 0; r < d; ++r) gr.m[r * d + r] = op.m[r];
                } else {
                    ps.ngates++;
                    continue;  // identity
                }
                ps.block = matmul(embed_gate(gr, qs), ps.block, size_t(1) << k);
                ps.ngates++;
                continue;
            }
            if (diag[gi] && ops[gi].type != Op::IDENTITY) {
                if (int(ps.epi.size()) >= MAX_EPI) {
                    blocked |= q;
                    rest.push_back(gi);
                    continue;
                }
                // straddles the window: applied after the block, so the
                // window qubits it touches take no further block gates
                TcPass::Diag dg;
                dg.targets.assign(op.targets, op.targets + op.k);
                dg.controls.assign(op.controls, op.controls + op.c);
                dg.d = op.m;
                ps.epi.push_back(dg);
                ps.ngates++;
                blocked |= q & wmask;
                continue;
            }
            if (ops[gi].type == Op::IDENTITY) {
                ps.ngates++;
                continue;
            }
            blocked |= q;
            rest.push_back(gi);
        }
        stall = ps.ngates ? 0 : stall + 1;
        if (stall > 2 * n) {
            const Op &o = ops[remaining.front()];
            return set_error(QSIM_EUNSUPPORTED,
                             "tensor-core planner: gate %d (%d targets, %d controls, first qubit %d) fits no %d-qubit window",
                             remaining.front(), o.k, o.c, o.k ? o.targets[0] : o.controls[0], k);
        }
        tp->passes.push_back(std::move(ps));
        remaining.swap(rest);
        off = (off + k) % n;
        rotated += k;
    }
    // close the rotation: extra identity passes until the total is a multiple
    // of n (3xTF32 plans use width 5 only: width 6 does not fit shared memory)
    for (int extra = (n - rotated % n) % n;; extra += n) {
        std::vector<int> widths;
        if (extra == 0) break;
        const bool fits = kw == 5 ? (extra % 5 == 0 && (widths.assign(extra / 5, 5), true)) : split56(extra, widths);
        if (fits) {
            for (int w : widths) {
                TcPass ps;
                ps.k = w;
                ps.off = off;
                ps.block.assign(size_t(1) << (2 * w), cd(0.0));
                for (size_t i = 0; i < (size_t(1) << w); ++i) ps.block[i * ((size_t(1) << w) + 1)] = 1.0;
                tp->passes.push_back(std::move(ps));
                off = (off + w) % n;
            }
            break;
        }
    }
    for (TcPass &ps : tp->passes) ps.prec = tp->prec;
    return QSIM_OK;
}

// Arithmetic of each pass (TcPrec values, one per pass; plain passes ignore
// theirs).  3xTF32 needs a 5-wide window (6-wide operands do not fit shared
// memory).  The device images are rebuilt at the next run.
int tc_set_precisions(qsim_plan &p, const std::vector<int> &prec) {
    if (!p.tc) return set_error(QSIM_EINVAL, "not a tensor-core plan");
    TcPlan &tp = *p.tc;
    if (prec.size() != tp.passes.size()) return set_error(QSIM_EINVAL, "one precision per pass");
    for (size_t i = 0; i < prec.size(); ++i) {
        if (prec[i] < TC_BF16X3 || prec[i] > TC_FP32) return set_error(QSIM_EINVAL, "pass %zu: bad precision", i);
        if (prec[i] == TC_TF32X3 && !tp.passes[i].plain && tp.passes[i].k != 5)
            return set_error(QSIM_EINVAL, "pass %zu: 3xTF32 passes are 5 qubits wide", i);
    }
    for (size_t i = 0; i < prec.size(); ++i) tp.passes[i].prec = prec[i];
    if (tp.dev.bimg) cudaFree(tp.dev.bimg);
    tp.dev.bimg = nullptr;
    tp.dev.ready = false;
    return QSIM_OK;
}

int tc_pass_precision(const qsim_plan &p, int i) { return p.tc->passes[size_t(i)].prec; }

namespace {

template <int EB>
void build_bimage(const std::vector<cd> &G, int k, std::vector<unsigned char> &img, int prec) {
    const int KR = 2 << k;
    const int d = 1 << k;
    const size_t opnd = size_t(KR) * KR * EB;
    img.assign(2 * opnd, 0);
    for (int nn = 0; nn < KR; ++nn)
        for (int kk = 0; kk < KR; ++kk) {
            const int c = nn >> 1, s = nn & 1, cp = kk >> 1, t = kk & 1;
            const cd g = G[size_t(c) * d + cp];
            const double v = s == 0 ? (t == 0 ? g.real() : -g.imag()) : (t == 0 ? g.imag() : g.real());
            const uint32_t off = sw128_offset<EB>(nn, kk, KR);
            const float f = float(v);
            if (prec == TC_BF16X3) {
                // round-to-nearest-even bf16 split of the fp32 value
                auto bf = [](float x) {
                    uint32_t u;
                    memcpy(&u, &x, 4);
                    const uint32_t lsb = (u >> 16) & 1;
                    u += 0x7FFF + lsb;
                    return uint16_t(u >> 16);
                };
                const uint16_t h = bf(f);
                uint32_t hu = uint32_t(h) << 16;
                float hf;
                memcpy(&hf, &hu, 4);
                const uint16_t l = bf(f - hf);
                memcpy(&img[off], &h, 2);
                memcpy(&img[opnd + off], &l, 2);
            } else {
                uint32_t u;
                memcpy(&u, &f, 4);
                const uint32_t hu = tf32_rn(u);
                float hf;
                memcpy(&hf, &hu, 4);
                const float lf = f - hf;
                uint32_t lu;
                memcpy(&lu, &lf, 4);
                lu = tf32_rn(lu);
                memcpy(&img[off], &hu, 4);
                memcpy(&img[opnd + off], &lu, 4);
            }
        }
}

template <int K, int PREC> constexpr int smem_bytes() { return TcShape<K, PREC>::SMEM; }

int prepare_tc(qsim_plan &p, int n) {
    TcPlan &tp = *p.tc;
    if (tp.dev.ready) return QSIM_OK;
    std::vector<unsigned char> all, img;
    tp.dev.boff.clear();
    tp.dev.params.clear();
    for (const TcPass &ps : tp.passes) {
        if (ps.plain) {  // no tensor-core work: placeholders keep the indices aligned
            tp.dev.boff.push_back(0);
            TcParams prm;
            memset(&prm, 0, sizeof prm);
            tp.dev.params.push_back(prm);
            continue;
        }
        if (ps.prec == TC_FP32) {  // the block itself, complex64 row-major
            const size_t d2 = size_t(1) << (2 * ps.k);
            img.resize(d2 * sizeof(float2));
            for (size_t e = 0; e < d2; ++e) {
                const float2 v = make_float2(float(ps.block[e].real()), float(ps.block[e].imag()));
                memcpy(&img[e * sizeof(float2)], &v, sizeof v);
            }
        } else if (ps.prec == TC_BF16X3) {
            build_bimage<2>(ps.block, ps.k, img, ps.prec);
        } else {
            build_bimage<4>(ps.block, ps.k, img, ps.prec);
        }
        tp.dev.boff.push_back(all.size());
        all.insert(all.end(), img.begin(), img.end());
        while (all.size() % 256) all.push_back(0);
        TcParams prm;
        memset(&prm, 0, sizeof prm);
        prm.n = n;
        prm.ntiles = (uint64_t(1) << (n - ps.k)) / TC_M;
        int pool = 0;
        for (const TcPass::Diag &dg : ps.epi) {
            auto cur = [&](int q) { return (q - ps.off + n) % n; };
            uint64_t cmask = 0;
            for (int q : dg.controls) cmask |= uint64_t(1) << cur(q);
            if (dg.targets.empty() && dg.d[0] == cd(-1.0)) {
                // -1 on the control subspace: rows whose control bits are set
                // negate the columns whose control bits are set
                const uint64_t cm = cmask & ((uint64_t(1) << ps.k) - 1);
                uint64_t cols = 0;
                for (uint64_t c = 0; c < (uint64_t(1) << ps.k); ++c)
                    if ((c & cm) == cm) cols |= uint64_t(1) << c;
                prm.negr[prm.nneg] = cmask >> ps.k;
                prm.negc[prm.nneg] = cols;
                ++prm.nneg;
                continue;
            }
            EpiOp &e = prm.epi[prm.nepi++];
            e.cmask = cmask;
            e.k = int(dg.targets.size());
            for (int t = 0; t < e.k; ++t) e.sel[t] = cur(dg.targets[t]);
            e.neg = 0;
            e.moff = pool;
            if (pool + int(dg.d.size()) > MAX_EPI_POOL) return set_error(QSIM_EUNSUPPORTED, "epilogue pool overflow");
            for (const cd &v : dg.d) prm.pool[pool++] = make_float2(float(v.real()), float(v.imag()));
        }
        tp.dev.params.push_back(prm);
    }
    QSIM_CUDA_TRY(dev_alloc(&tp.dev.bimg, all.size()), "tc B images");
    QSIM_CUDA_TRY(cudaMemcpy(tp.dev.bimg, all.data(), all.size(), cudaMemcpyHostToDevice), "tc B upload");
    QSIM_CUDA_TRY(dev_alloc(&tp.dev.err, sizeof(int)), "tc error flag");
    QSIM_CUDA_TRY(cudaMemset(tp.dev.err, 0, sizeof(int)), "tc error flag clear");
    tp.dev.ready = true;
    return QSIM_OK;
}

int sm_count_tc() { return device_sm_count(); }

template <int K, int PREC>
int launch_tc_k(const TcParams &prm, cudaStream_t st) {
    constexpr int smem = TcShape<K, PREC>::SMEM;
    static bool attr = false;
    if (!attr) {
        QSIM_CUDA_TRY(cudaFuncSetAttribute(k_tc_block<K, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                      "tc smem attribute");
        attr = true;
    }
    const uint64_t want = uint64_t(sm_count_tc());
    const unsigned grid = unsigned(std::min<uint64_t>(want, prm.ntiles));
    // useful flops: a dense k-qubit block is 2^k complex multiply-adds per amplitude
    LaunchScope ls(K_TC_BLOCK, st, 2.0 * double(prm.ntiles) * TC_M * (2 << K) * 4.0,
                   8.0 * double(1 << K) * double(prm.ntiles) * TC_M * double(1 << K));
    k_tc_block<K, PREC><<<grid, TC_THREADS, smem, st>>>(prm);
    QSIM_CUDA_TRY(cudaGetLastError(), "tc launch");
    return QSIM_OK;
}

template <int K>
int launch_rot_simt(const TcParams &prm, cudaStream_t st) {
    constexpr int smem = simt_smem_bytes<K>();
    static bool attr = false;
    if (!attr) {
        QSIM_CUDA_TRY(cudaFuncSetAttribute(k_rot_simt<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                      "fp32 pass smem attribute");
        attr = true;
    }
    const uint64_t rows = uint64_t(1) << (prm.n - K);
    const unsigned grid = unsigned(std::min<uint64_t>(uint64_t(sm_count_tc()) * 2, (rows + 127) / 128));
    LaunchScope ls(K_TC_BLOCK, st, 2.0 * double(rows << K) * 8.0, 8.0 * double(1 << K) * double(rows << K));
    k_rot_simt<K><<<grid, 128, smem, st>>>(prm, reinterpret_cast<const float2 *>(prm.bimg));
    QSIM_CUDA_TRY(cudaGetLastError(), "fp32 pass launch");
    return QSIM_OK;
}

}  // namespace

// polls before a pipeline wait gives up (test support can shorten it)
static std::atomic<unsigned long long> g_wait_limit{WAIT_LIMIT};

int run_tc(qsim_state *s, qsim_plan &p) {
    if (s->dtype != QSIM_C64) return set_error(QSIM_EUNSUPPORTED, "tensor-core plans run complex64 states");
    QSIM_TRY(prepare_tc(p, s->n));
    TcPlan &tp = *p.tc;
    const size_t bytes = s->size() * s->amp_bytes();
    // ping-pong partner buffer in the state's scratch (grow-only)
    QSIM_TRY(s->ensure_scratch(bytes));
    float2 *bufs[2] = {static_cast<float2 *>(s->amps), static_cast<float2 *>(s->scratch)};
    int cur = 0;
    for (size_t i = 0; i < tp.passes.size(); ++i) {
        if (tp.passes[i].plain) {
            // in place on the current buffer, qubits moved to their current bits
            Op op = tp.passes[i].op;
            const int off = tp.passes[i].off, n = s->n;
            for (int t = 0; t < op.k; ++t) op.targets[t] = (op.targets[t] - off + n) % n;
            for (int t = 0; t < op.c; ++t) op.controls[t] = (op.controls[t] - off + n) % n;
            QSIM_TRY(launch_op(bufs[cur], n, QSIM_C64, op, s->stream, nullptr));
            continue;
        }
        TcParams prm = tp.dev.params[i];
        prm.in = bufs[cur];
        prm.out = bufs[cur ^ 1];
        prm.bimg = reinterpret_cast<const uint4 *>(static_cast<char *>(tp.dev.bimg) + tp.dev.boff[i]);
        prm.err = tp.dev.err;
        prm.wait_limit = g_wait_limit.load();
        const int k = tp.passes[i].k;
        int rc;
        const int prec = tp.passes[i].prec;
        if (prec == TC_FP32) rc = k == 6 ? launch_rot_simt<6>(prm, s->stream) : launch_rot_simt<5>(prm, s->stream);
        else if (prec == TC_BF16X3) rc = k == 6 ? launch_tc_k<6, TC_BF16X3>(prm, s->stream) : launch_tc_k<5, TC_BF16X3>(prm, s->stream);
        else if (k == 5) rc = launch_tc_k<5, TC_TF32X3>(prm, s->stream);
        else rc = set_error(QSIM_EUNSUPPORTED, "3xTF32 passes are 5 qubits wide");
        QSIM_TRY(rc);
        cur ^= 1;
    }
    if (cur == 1) {
        LaunchScope ls(K_COPY, s->stream, 2.0 * double(bytes));
        QSIM_CUDA_TRY(cudaMemcpyAsync(s->amps, s->scratch, bytes, cudaMemcpyDeviceToDevice, s->stream), "tc result copy");
    }
    int err = 0;
    QSIM_CUDA_TRY(cudaMemcpyAsync(&err, tp.dev.err, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "tc flag read");
    QSIM_CUDA_TRY(cudaStreamSynchronize(s->stream), "tc sync");
    if (err) {
        cudaMemsetAsync(tp.dev.err, 0, sizeof(int), s->stream);
        return set_error(QSIM_ETIMEOUT, "tensor-core pass: an mbarrier wait exceeded its bound");
    }
    return QSIM_OK;
}

int tc_nsweeps(const qsim_plan &p) { return p.tc ? int(p.tc->passes.size()) : 0; }

void tc_describe(const qsim_plan &p, std::string &out) {
    if (!p.tc) return;
    char buf[256];
    snprintf(buf, sizeof buf, "tensor-core plan: %zu passes, default %s\n", p.tc->passes.size(),
             p.tc->prec == TC_BF16X3 ? "BF16x3 (kind::f16)" : "3xTF32 (kind::tf32)");
    out += buf;
    for (size_t i = 0; i < p.tc->passes.size(); ++i) {
        const TcPass &ps = p.tc->passes[i];
        if (ps.plain) {
            snprintf(buf, sizeof buf, "  %3zu plain sweep: %d-target gate (kind %d) on the rotated index\n", i, ps.op.k,
                     int(ps.op.type));
            out += buf;
            continue;
        }
        static const char *pn[3] = {"bf16x3", "3xtf32", "fp32"};
        snprintf(buf, sizeof buf, "  %3zu k=%d qubits %d..%d (mod n) gates=%d epilogue=%zu %s\n", i, ps.k, ps.off,
                 ps.off + ps.k - 1, ps.ngates, ps.epi.size(), pn[ps.prec]);
        out += buf;
    }
}

}  // namespace qsim

// ------------------------------------------------------------------ host inspection
extern "C" {

QSIM_API int qsim_plan_tc_pass(const qsim_plan *p, int i, int *plain, int *k, int *targets, int *nc, int *controls,
                               double *matrix, int *nepi) {
    using namespace qsim;
    if (!p || !p->tc) return set_error(QSIM_EINVAL, "not a tensor-core plan");
    if (i < 0 || i >= int(p->tc->passes.size())) return set_error(QSIM_EINVAL, "pass %d outside the plan", i);
    const TcPass &ps = p->tc->passes[size_t(i)];
    std::vector<int> t, c;
    std::vector<cd> m;
    if (ps.plain) {
        const Op &op = ps.op;
        t.assign(op.targets, op.targets + op.k);
        c.assign(op.controls, op.controls + op.c);
        const size_t d = size_t(1) << op.k;
        m.assign(d * d, cd(0.0));
        if (op.type == Op::DENSE) {
            m = op.m;
        } else {
            for (size_t r = 0; r < d; ++r) {
                if (op.type == Op::DIAG) m[r * d + r] = op.m[r];
                else if (op.type == Op::MONO) m[r * d + size_t(op.perm[r])] = op.phase[r];
                else m[r * d + r] = 1.0;
            }
        }
    } else {
        for (int j = ps.k - 1; j >= 0; --j) t.push_back((ps.off + j) % p->n);  // window, MSB first
        m = ps.block;
    }
    if (plain) *plain = ps.plain ? 1 : 0;
    if (k) *k = int(t.size());
    if (targets)
        for (size_t j = 0; j < t.size(); ++j) targets[j] = t[j];
    if (nc) *nc = int(c.size());
    if (controls)
        for (size_t j = 0; j < c.size(); ++j) controls[j] = c[j];
    if (matrix)
        for (size_t j = 0; j < m.size(); ++j) {
            matrix[2 * j] = m[j].real();
            matrix[2 * j + 1] = m[j].imag();
        }
    if (nepi) *nepi = ps.plain ? 0 : int(ps.epi.size());
    return QSIM_OK;
}

QSIM_API int qsim_plan_tc_epilogue(const qsim_plan *p, int i, int e, int *k, int *targets, int *nc, int *controls,
                                   double *diag) {
    using namespace qsim;
    if (!p || !p->tc) return set_error(QSIM_EINVAL, "not a tensor-core plan");
    if (i < 0 || i >= int(p->tc->passes.size())) return set_error(QSIM_EINVAL, "pass %d outside the plan", i);
    const TcPass &ps = p->tc->passes[size_t(i)];
    if (e < 0 || e >= int(ps.epi.size())) return set_error(QSIM_EINVAL, "epilogue gate %d outside pass %d", e, i);
    const TcPass::Diag &dg = ps.epi[size_t(e)];
    if (k) *k = int(dg.targets.size());
    if (targets)
        for (size_t j = 0; j < dg.targets.size(); ++j) targets[j] = dg.targets[j];
    if (nc) *nc = int(dg.controls.size());
    if (controls)
        for (size_t j = 0; j < dg.controls.size(); ++j) controls[j] = dg.controls[j];
    if (diag)
        for (size_t j = 0; j < dg.d.size(); ++j) {
            diag[2 * j] = dg.d[j].real();
            diag[2 * j + 1] = dg.d[j].imag();
        }
    return QSIM_OK;
}

QSIM_API int qsim_plan_tc_precision(const qsim_plan *p, int i, int *prec) {
    using namespace qsim;
    if (!p || !p->tc || !prec) return set_error(QSIM_EINVAL, "not a tensor-core plan");
    if (i < 0 || i >= int(p->tc->passes.size())) return set_error(QSIM_EINVAL, "pass %d outside the plan", i);
    *prec = tc_pass_precision(*p, i);
    return QSIM_OK;
}

QSIM_API int qsim_plan_tc_set_precision(qsim_plan *p, int npasses, const int *prec) {
    using namespace qsim;
    if (!p || !p->tc || !prec) return set_error(QSIM_EINVAL, "not a tensor-core plan");
    if (npasses != int(p->tc->passes.size())) return set_error(QSIM_EINVAL, "one precision per pass");
    return tc_set_precisions(*p, std::vector<int>(prec, prec + npasses));
}

}  // extern "C"

void qsim_plan::release_tc() {
    delete tc;
    tc = nullptr;
}

extern "C" QSIM_API int qsim_debug_set_wait_limit(unsigned long long polls) {
    qsim::g_wait_limit.store(polls ? polls : qsim::WAIT_LIMIT);
    return QSIM_OK;
}

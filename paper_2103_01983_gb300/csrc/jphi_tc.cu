// bs_jphi on the 5th-generation tensor cores (prec PTROM_TF32X3 and
// PTROM_F16X3).
//
// With K the 2n x 2n matrix of pair blocks K_ij = gamma_j A(x_i - x_j)
// (zero on the block diagonal) and S_i = sum_j K_ij, the J Phi of the LSPG
// Gauss-Newton least squares (Sec. 3.2) is
//     (J Phi)_i = sum_j K_ij (Phi_i - Phi_j) = S_i Phi_i - sum_j K_ij Phi_j,
// and the second term is a dense contraction over the sources.  Its left
// operand is generated on the fly, never stored in global memory:
//
//   * a CTA owns 128 target bodies (MMA rows: their chi dofs in half 0, psi
//     dofs in half 1) and one slice of up to 64 basis columns (MMA N);
//   * a tile is 16 (TF32) or 32 (FP16) source bodies (MMA K = 32 or 64: chi
//     dofs, then psi dofs; either way 8 groups of 16 bytes per row).  A
//     loader warp brings each tile's image -- the sources' positions and
//     gamma, and their Phi rows already split into hi and lo parts in the
//     tensor cores' K-major layout -- into shared memory with one bulk copy
//     (cp.async.bulk, completion on an mbarrier), four tiles ahead;
//   * eight generator warps evaluate the 2x2 blocks of the tile's pairs in
//     FP32, split each entry into hi + lo, and store them in the same layout
//     (two stages);
//   * one thread issues tcgen05.mma kind::tf32 (K = 8 per instruction) or
//     kind::f16 (K = 16), M = 128, for both halves: A_hi B_hi into one
//     accumulator and the cross terms A_hi B_lo + A_lo B_hi (2^-11 smaller)
//     into another -- the 3-term split that keeps products to ~2^-20
//     relative -- both in tensor memory;
//   * every 16 tiles (256 or 512 sources) the generators read both accumulators
//     back with tcgen05.ld and add them to a TwoSum-compensated (hi, lo)
//     total that also lives in tensor memory (tcgen05.st), so the hi*hi sum
//     in FP32 never runs over more than 64 MMA steps before it is folded
//     exactly; the diagonal sums S_i are accumulated per tile in FP32 and
//     folded into compensated pairs in registers.
// FP16 has TF32's 11-bit significand but a 5-bit exponent, so that variant
// scales by powers of two: the blocks by 2^(14 - e) with 2^e bounding
// 3 max|gamma| / delta (no block entry exceeds it, so nothing overflows;
// entries far below it lose only absolute bits ~2^-24 of the bound), each
// basis column by 2^(14 - e_m) from its largest entry; the epilogue divides
// the powers out exactly.  It needs delta > 0 (the bound); at delta = 0 the
// call takes the TF32 variant.  Per MMA instruction FP16 moves twice TF32's
// K, so it issues half as many MMAs per pair.
// The epilogue forms S_i Phi_i - sum_j K_ij Phi_j in FP64.  Source splits
// over gridDim.z write FP64 partials that a second kernel adds in split
// order, as in the SIMT kernel.  Every mbarrier wait is bounded (1 s of
// global time); a CTA that gives up raises a status the host reads, waits
// (bounded) for its copies and MMAs in flight, and frees its tensor memory.
#include <algorithm>
#include <atomic>

#include <cuda_fp16.h>

#include "common.cuh"
#include "scratch.h"
#include "internal.h"

namespace ptrom {
std::atomic<int> g_jphi_tc_withhold{0};
namespace {

constexpr int kTB = 128;       // target bodies per CTA (MMA M = 128 per half)
constexpr int kNC = 64;        // basis columns per slice (MMA N <= 64)
constexpr int kChunk = 16;     // tiles accumulated in tensor memory between folds
constexpr int kStA = 2, kStB = 4;
constexpr int kGenThreads = 256, kMmaWarp = 8, kLoadWarp = 9, kThreads = 320;
// tensor-memory columns: per half (64 columns each) the chunk's hi*hi
// accumulator, its cross-term accumulator, and the running total's hi and lo
constexpr uint32_t kColMain = 0, kColCross = 2 * kNC, kColHi = 4 * kNC, kColLo = 6 * kNC;
constexpr uint32_t kTmemCols = 8 * kNC;  // 512: all of an SM's tensor memory (one CTA per SM)

// K-major, no-swizzle operand layout: 8-row x 16-byte core matrices; rows of
// a core matrix 16 bytes apart, 8-row groups 128 bytes apart (SBO), groups of
// 16 bytes of K (4 TF32 or 8 FP16 elements) LBO apart; a tile row holds 8
// such groups in both formats.
constexpr uint32_t kSbo = 128;
constexpr uint32_t kALbo = (kTB / 8) * 128;               // 2048
constexpr uint32_t kATile = 8 * kALbo;                    // 128 rows x 8 K groups = 16 KB
constexpr uint32_t kAStage = 4 * kATile;                  // (half 0, 1) x (hi, lo)
constexpr uint32_t kBLbo = (kNC / 8) * 128;               // 1024
constexpr uint32_t kBTile = 8 * kBLbo;                    // 64 rows x 8 K groups = 8 KB
constexpr uint32_t kAOff = 0;
constexpr uint32_t kBOff = kAOff + kStA * kAStage;        // 131072
constexpr int kNumBars = 15;
// per format: sources per tile, their records (x, y, gamma, 0), one tile
// image (records, B hi, B lo), the barrier block, the shared memory
template <bool F16> __host__ __device__ constexpr int tile_sources() { return F16 ? 32 : 16; }
template <bool F16> __host__ __device__ constexpr uint32_t rec_bytes() { return tile_sources<F16>() * 16; }
template <bool F16> __host__ __device__ constexpr uint32_t img_bytes() { return rec_bytes<F16>() + 2 * kBTile; }
template <bool F16> __host__ __device__ constexpr uint32_t bar_off() { return kBOff + kStB * img_bytes<F16>(); }
template <bool F16> __host__ __device__ constexpr uint32_t smem_bytes() { return bar_off<F16>() + 256; }
static_assert(kNumBars * 8 + 8 <= 256, "barrier block");
static_assert(img_bytes<false>() % 16 == 0 && img_bytes<true>() % 16 == 0 && kBOff % 16 == 0,
              "bulk copies need 16-byte sizes and addresses");
static_assert(smem_bytes<false>() <= 227 * 1024 && smem_bytes<true>() <= 227 * 1024, "shared memory");
static_assert(2 * 128 * 3 * 8 <= kAStage, "S exchange fits in the A stages");
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_test(uint64_t *b, uint32_t parity) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return r != 0;
}

// Wait for the completion of the phase with this parity: false once the CTA
// has given up (abort set by any thread) or after kWaitNs, which sets abort.
// With follow_abort false it ignores the flag (draining work in flight).
__device__ bool bar_wait(uint64_t *b, uint32_t parity, volatile int *abort_f, bool follow_abort = true) {
    if (bar_test(b, parity)) return true;
    const unsigned long long t0 = gtime();
    while (true) {
        if (bar_test(b, parity)) return true;
        if (follow_abort && *abort_f) return false;
        if (gtime() - t0 > kWaitNs) {
            *abort_f = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(b))
                 : "memory");
}

// Shared-memory matrix descriptor: start, LBO, SBO (all >> 4), the fixed
// 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor: FP32 accumulate (bits 4-5 = 1), A and B of one
// type (bits 7-9, 10-12: TF32 = 2 under kind::tf32, FP16 = 0 under
// kind::f16), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <bool F16>
__host__ __device__ constexpr uint32_t idesc_mma(uint32_t M, uint32_t N) {
    return (1u << 4) | ((F16 ? 0u : 2u) << 7) | ((F16 ? 0u : 2u) << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <bool F16>
__device__ __forceinline__ void mma_issue(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (F16)
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t ta, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(ta),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// TF32 split: hi keeps the top 10 explicit mantissa bits (exact in TF32), lo
// the rest.
__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }

__device__ __forceinline__ void st4(unsigned char *p, float a, float b, float c, float d) {
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}

// FP16 split of a scaled value: hi rounded to nearest, lo the rounded rest.
__device__ __forceinline__ void f16_split(float v, __half &hi, __half &lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}

__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// Power-of-two scale 2^(14 - e) for values bounded by x = 2^e .. 2^(e+1)
// (exponent clamped so the scale stays finite); 1 for x = 0.
__device__ __forceinline__ int scale_exp(float x) {
    if (!(x > 0.f)) return 0;
    int e = (int)((__float_as_uint(x) >> 23) & 0xff) - 127;
    int se = 14 - e;
    return se < -120 ? -120 : (se > 120 ? 120 : se);
}

// Largest |Gamma| (slot 0) and largest |Phi| of each column m (slot 1 + m),
// as the bit patterns of non-negative floats (ordered like the values).
__global__ void k_tc_maxabs(int n, const double *G, const double *phi, int M, unsigned *umax) {
    const int col = blockIdx.y;  // 0 .. M - 1: basis columns; M: Gamma
    const size_t len = col < M ? 2 * (size_t)n : (size_t)n;
    const double *src = col < M ? phi + (size_t)col * 2 * n : G;
    float m = 0.f;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf((float)src[e]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(umax + (col < M ? 1 + col : 0), __float_as_uint(m));
}

// Tile images, per (slice, tile): the tile's source records, then Phi rows of
// the slice's 64 columns (MMA N rows) x the tile's dofs (K), hi then lo, in
// the MMA layout; FP16 rows scaled per column (umax, see k_tc_maxabs).
template <bool F16>
__global__ void k_tc_pack(int n, const double *x, const double *G, const double *phi, int M, int nslices, int ntiles,
                          const unsigned *umax, unsigned char *img) {
    constexpr int kTSx = tile_sources<F16>();
    constexpr int kEsz = F16 ? 2 : 4;                        // element bytes
    constexpr int kPer = 16 / kEsz;                          // K elements per 16-byte group
    constexpr int kRecWords = (int)rec_bytes<F16>() / 4;
    constexpr int kPart = (int)kBTile / kEsz;                // elements per B part
    constexpr int kItems = kRecWords + 2 * kPart;
    const double ox = x[0], oy = x[n];
    const size_t total = (size_t)nslices * ntiles * kItems;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(e % kItems);
        const size_t st = e / kItems;
        const int tile = (int)(st % ntiles), slice = (int)(st / ntiles);
        unsigned char *base = img + st * img_bytes<F16>();
        if (w < kRecWords) {
            const int j = tile * kTSx + w / 4, comp = w % 4;
            float v = 0.f;
            if (j < n) {
                if (comp == 0) v = (float)(x[j] - ox);
                else if (comp == 1) v = (float)(x[n + j] - oy);
                else if (comp == 2) v = (float)(G[j] * kInv2Pi);
            }
            reinterpret_cast<float *>(base)[w] = v;
            continue;
        }
        const int o = w - kRecWords;
        const int part = o / kPart, q = o % kPart;
        // element q = kgroup * (LBO / esize) + row * kPer + k % kPer
        const int kg = q / ((int)kBLbo / kEsz), rem = q % ((int)kBLbo / kEsz);
        const int row = rem / kPer, k = kg * kPer + rem % kPer;
        const int j = tile * kTSx + (k % kTSx), dof = k / kTSx;
        const int m = slice * kNC + row;
        const double d = (j < n && m < M) ? phi[(size_t)m * 2 * n + (size_t)dof * n + j] : 0.0;
        unsigned char *dst = base + rec_bytes<F16>() + part * kBTile;
        if constexpr (F16) {
            const float sc = m < M ? ldexpf(1.f, scale_exp(__uint_as_float(umax[1 + m]))) : 1.f;
            __half hi, lo;
            f16_split((float)(d * sc), hi, lo);
            reinterpret_cast<__half *>(dst)[q] = part == 0 ? hi : lo;
        } else {
            const float hi = tf32_hi((float)d);
            reinterpret_cast<float *>(dst)[q] = part == 0 ? hi : (float)(d - (double)hi);
        }
    }
}

// Fold chunk c (this warp's 32 TMEM lanes = output rows of half sh, 64
// columns) into the running total: total += main + cross with TwoSum, total
// kept as (hi, lo) in tensor memory; then hand the accumulators back to the
// MMA issuer.  Warp-uniform; false when the CTA gave up.
__device__ __forceinline__ bool fold_chunk(int c, int sh, uint32_t tmem, uint32_t lane_base, uint64_t *accfull,
                                           uint64_t *accempty, volatile int *abort_f) {
    bool ok = bar_wait(accfull, c & 1, abort_f);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) return false;
    tc_fence_after();
    const uint32_t base = tmem + lane_base + (uint32_t)(sh * kNC);
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
        const uint32_t col = base + 32 * hh;
        uint32_t m[32], x[32], h[32], l[32];
        tmem_ld32(col + kColMain, m);
        tmem_ld32(col + kColCross, x);
        if (c > 0) {
            tmem_ld32(col + kColHi, h);
            tmem_ld32(col + kColLo, l);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const float v = __uint_as_float(m[k]) + __uint_as_float(x[k]);
            if (c == 0) {
                h[k] = __float_as_uint(v);
                l[k] = 0u;
            } else {
                const float hi = __uint_as_float(h[k]);
                const float sum = hi + v, bb = sum - hi;
                const float err = (hi - (sum - bb)) + (v - bb);
                h[k] = __float_as_uint(sum);
                l[k] = __float_as_uint(__uint_as_float(l[k]) + err);
            }
        }
        tmem_st32(col + kColHi, h);
        tmem_st32(col + kColLo, l);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    bar_arrive(accempty);
    return true;
}

template <bool MASK, bool F16>
__global__ void __launch_bounds__(kThreads, 1)
k_jphi_tc(int n, const double *x, const double *phi, int M, float delta, const unsigned char *img_all, int ntiles,
          const unsigned *umax, double *out, double *part, int *status, int withhold) {
    constexpr uint32_t kImg = img_bytes<F16>(), kRecBytes = rec_bytes<F16>(), kBarOff = bar_off<F16>();
    constexpr int kU = F16 ? 8 : 4;  // sources per 16-byte K group
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tb0 = blockIdx.x * kTB;
    const int slice = blockIdx.y;
    const int ncols = min(kNC, M - slice * kNC);
    const uint32_t nmma = (uint32_t)((ncols + 15) & ~15);
    const int t_begin = (int)(((long long)blockIdx.z * ntiles) / gridDim.z);
    const int t_end = (int)(((long long)(blockIdx.z + 1) * ntiles) / gridDim.z);
    const int T = t_end - t_begin;
    const unsigned char *img = img_all + ((size_t)slice * ntiles + t_begin) * kImg;

    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kBarOff);
    uint64_t *bfull = bars, *emptyB = bars + 4, *afull = bars + 8, *emptyA = bars + 10, *accfull = bars + 12,
             *accempty = bars + 13, *done = bars + 14;
    uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kBarOff + kNumBars * 8);
    volatile int *abort_f = reinterpret_cast<volatile int *>(sm + kBarOff + kNumBars * 8 + 4);
    if (tid == 0) {
        for (int s = 0; s < kStB; ++s) {
            bar_init(bfull + s, 1);
            bar_init(emptyB + s, 1);
        }
        for (int s = 0; s < kStA; ++s) {
            bar_init(afull + s, kGenThreads);
            bar_init(emptyA + s, 1);
        }
        bar_init(accfull, 1);
        bar_init(accempty, kGenThreads);
        bar_init(done, 1);
        *abort_f = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;

    if (warp == kLoadWarp) {
        if (lane == 0) {
            int issued = 0;
            // withhold: the test hook -- no copy is issued, so every wait on
            // one runs out at its bound and the CTA takes its abort path
            for (int t = 0; t < (withhold ? 0 : T); ++t) {
                const int s = t % kStB, use = t / kStB;
                if (use > 0 && !bar_wait(emptyB + s, (use - 1) & 1, abort_f)) break;
                bar_expect_tx(bfull + s, kImg);
                bulk_g2s(sm + kBOff + s * kImg, img + (size_t)t * kImg, kImg, bfull + s);
                issued = t + 1;
            }
            // every copy still landing in shared memory completes before the CTA leaves
            for (int t = max(0, issued - kStB); t < issued; ++t)
                bar_wait(bfull + t % kStB, (t / kStB) & 1, abort_f, false);
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            const uint32_t idesc = idesc_mma<F16>(128, nmma);
            for (int t = 0; t < T; ++t) {
                const int c = t / kChunk;
                const bool first = t % kChunk == 0, last = t % kChunk == kChunk - 1 || t == T - 1;
                // the accumulators are single-buffered: chunk c starts once chunk c - 1 is folded
                if (first && c >= 1 && !bar_wait(accempty, (c - 1) & 1, abort_f)) break;
                if (!bar_wait(bfull + t % kStB, (t / kStB) & 1, abort_f)) break;
                if (!bar_wait(afull + t % kStA, (t / kStA) & 1, abort_f)) break;
                tc_fence_after();
                const uint32_t a0 = su32(sm + kAOff + (t % kStA) * kAStage);
                const uint32_t b0 = su32(sm + kBOff + (t % kStB) * kImg + kRecBytes);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint64_t bh = sdesc(b0 + q * 2 * kBLbo, kBLbo, kSbo);
                    const uint64_t bl = sdesc(b0 + kBTile + q * 2 * kBLbo, kBLbo, kSbo);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t dm = tmem + kColMain + (uint32_t)(h * kNC);
                        const uint32_t dx = tmem + kColCross + (uint32_t)(h * kNC);
                        const uint64_t ah = sdesc(a0 + (2 * h) * kATile + q * 2 * kALbo, kALbo, kSbo);
                        const uint64_t al = sdesc(a0 + (2 * h + 1) * kATile + q * 2 * kALbo, kALbo, kSbo);
                        const uint32_t acc = (first && q == 0) ? 0u : 1u;
                        mma_issue<F16>(dm, ah, bh, idesc, acc);
                        mma_issue<F16>(dx, ah, bl, idesc, acc);
                        mma_issue<F16>(dx, al, bh, idesc, 1u);
                    }
                }
                mma_commit(emptyA + t % kStA);
                mma_commit(emptyB + t % kStB);
                if (last) mma_commit(accfull);
            }
            // every MMA issued has completed before the tensor memory is freed
            mma_commit(done);
            bar_wait(done, 0, abort_f, false);
        }
        __syncwarp();
    } else {
        // generators: target i of this CTA (also the accumulator's TMEM lane),
        // sources 8 sh .. 8 sh + 7 of every tile; in the folds and the
        // epilogue, output row (dof sh, target i)
        const int i = (warp & 3) * 32 + lane, sh = warp >> 2;
        const int ti = tb0 + i;
        const bool tact = ti < n;
        const double ox = x[0], oy = x[n];
        const float tx = tact ? (float)(x[ti] - ox) : 0.f, ty = tact ? (float)(x[n + ti] - oy) : 0.f;
        // FP16: blocks scaled by 2^eA, 2^eA * 3 max|gamma| / delta < 2^15
        const int eA = F16 ? scale_exp(3.f * __uint_as_float(umax[0]) * (float)kInv2Pi / delta) : 0;
        const float sA = ldexpf(1.f, eA);
        CSum2 s0, s1;  // (s00, s01), (s10, -)
        s0.zero();
        s1.zero();
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        bool ok = true;
        int pending = -1;
        for (int t = 0; t < T; ++t) {
            const int sa = t % kStA;
            if (t >= kStA) ok = bar_wait(emptyA + sa, ((t / kStA) - 1) & 1, abort_f);
            if (ok) ok = bar_wait(bfull + t % kStB, (t / kStB) & 1, abort_f);
            ok = __all_sync(0xffffffffu, ok);  // the warp leaves together (tcgen05.ld is warp-wide)
            if (!ok) break;
            const float4 *rec = reinterpret_cast<const float4 *>(sm + kBOff + (t % kStB) * kImg);
            unsigned char *A = sm + kAOff + sa * kAStage;
            float p00 = 0.f, p01 = 0.f, p10 = 0.f;
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                const int jg = 2 * sh + jj;  // K group of these kU sources' chi dofs (psi: 4 + jg)
                float d00[kU], d01[kU], d10[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const float4 r = rec[kU * jg + u];
                    const float a = tx - r.x, b = ty - r.y;
                    const float d2 = fmaf(a, a, b * b);
                    float rr = rcp_approx(d2 + delta);
                    if (MASK) rr = d2 == 0.f ? 0.f : rr;
                    const float q = r.z * rr;
                    const float p2 = 2.f * q * rr;
                    const float pa = p2 * a;
                    d00[u] = pa * b;
                    d01[u] = fmaf(p2 * b, b, -q);
                    d10[u] = fmaf(-pa, a, q);
                    p00 += d00[u];
                    p01 += d01[u];
                    p10 += d10[u];
                }
                const uint32_t rchi = (uint32_t)jg * kALbo + (uint32_t)i * 16;        // chi-dof K group
                const uint32_t rpsi = (uint32_t)(4 + jg) * kALbo + (uint32_t)i * 16;  // psi-dof K group
                // half 0 (target chi rows): [A00 | A01]; half 1 (psi rows): [A10 | -A00]
                if constexpr (F16) {
                    uint32_t h[4][4], l[4][4];  // (A00, A01, A10, -A00) x 4 half pairs
#pragma unroll
                    for (int u = 0; u < kU; u += 2) {
                        __half a0h, a0l, a1h, a1l;
                        const float v0[4] = {d00[u], d01[u], d10[u], -d00[u]};
                        const float v1[4] = {d00[u + 1], d01[u + 1], d10[u + 1], -d00[u + 1]};
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            f16_split(v0[c] * sA, a0h, a0l);
                            f16_split(v1[c] * sA, a1h, a1l);
                            h[c][u / 2] = pack_h2(a0h, a1h);
                            l[c][u / 2] = pack_h2(a0l, a1l);
                        }
                    }
                    auto st16 = [](unsigned char *p, const uint32_t (&w)[4]) {
                        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
                    };
                    st16(A + 0 * kATile + rchi, h[0]);
                    st16(A + 0 * kATile + rpsi, h[1]);
                    st16(A + 2 * kATile + rchi, h[2]);
                    st16(A + 2 * kATile + rpsi, h[3]);
                    st16(A + 1 * kATile + rchi, l[0]);
                    st16(A + 1 * kATile + rpsi, l[1]);
                    st16(A + 3 * kATile + rchi, l[2]);
                    st16(A + 3 * kATile + rpsi, l[3]);
                } else {
                    float h00[kU], h01[kU], h10[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        h00[u] = tf32_hi(d00[u]);
                        h01[u] = tf32_hi(d01[u]);
                        h10[u] = tf32_hi(d10[u]);
                    }
                    st4(A + 0 * kATile + rchi, h00[0], h00[1], h00[2], h00[3]);
                    st4(A + 0 * kATile + rpsi, h01[0], h01[1], h01[2], h01[3]);
                    st4(A + 2 * kATile + rchi, h10[0], h10[1], h10[2], h10[3]);
                    st4(A + 2 * kATile + rpsi, -h00[0], -h00[1], -h00[2], -h00[3]);
                    st4(A + 1 * kATile + rchi, d00[0] - h00[0], d00[1] - h00[1], d00[2] - h00[2], d00[3] - h00[3]);
                    st4(A + 1 * kATile + rpsi, d01[0] - h01[0], d01[1] - h01[1], d01[2] - h01[2], d01[3] - h01[3]);
                    st4(A + 3 * kATile + rchi, d10[0] - h10[0], d10[1] - h10[1], d10[2] - h10[2], d10[3] - h10[3]);
                    st4(A + 3 * kATile + rpsi, h00[0] - d00[0], h00[1] - d00[1], h00[2] - d00[2], h00[3] - d00[3]);
                }
            }
            s0.add(f2(p00, p01));
            s1.add(f2(p10, 0.f));
            // the tensor cores read A through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_arrive(afull + sa);
            if (pending >= 0) {
                if (!(ok = fold_chunk(pending, sh, tmem, lane_base, accfull, accempty, abort_f))) break;
                pending = -1;
            }
            if (t % kChunk == kChunk - 1 || t == T - 1) pending = t / kChunk;
        }
        if (ok && pending >= 0) ok = fold_chunk(pending, sh, tmem, lane_base, accfull, accempty, abort_f);
        ok = __all_sync(0xffffffffu, ok);
        // S_i: the two source halves' sums meet in shared memory (the A
        // stages, idle once the last chunk's MMAs have completed)
        asm volatile("bar.sync 1, %0;" ::"r"(kGenThreads) : "memory");
        double *sx = reinterpret_cast<double *>(sm + kAOff);
        sx[(sh * kTB + i) * 3 + 0] = s0.x();
        sx[(sh * kTB + i) * 3 + 1] = s0.y();
        sx[(sh * kTB + i) * 3 + 2] = s1.x();
        asm volatile("bar.sync 1, %0;" ::"r"(kGenThreads) : "memory");
        const double s00 = sx[i * 3 + 0] + sx[(kTB + i) * 3 + 0];
        const double s01 = sx[i * 3 + 1] + sx[(kTB + i) * 3 + 1];
        const double s10 = sx[i * 3 + 2] + sx[(kTB + i) * 3 + 2];
        // the total's (hi, lo) come back from tensor memory warp-wide
        if (__all_sync(0xffffffffu, ok && !*abort_f)) {
            tc_fence_after();
            double *dst = gridDim.z > 1 ? part + (size_t)blockIdx.z * 2 * n * M : out;
#pragma unroll 1
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t h[32], l[32];
                const uint32_t col = tmem + lane_base + (uint32_t)(sh * kNC + 32 * hh);
                tmem_ld32(col + kColHi, h);
                tmem_ld32(col + kColLo, l);
                if (!tact) continue;
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    const int m = slice * kNC + 32 * hh + k;
                    if (m >= M) continue;
                    const double pc = phi[(size_t)m * 2 * n + ti], pp = phi[(size_t)m * 2 * n + n + ti];
                    const double si = sh == 0 ? s00 * pc + s01 * pp : s10 * pc - s00 * pp;
                    double sum = (double)__uint_as_float(h[k]) + (double)__uint_as_float(l[k]);
                    if (F16) sum = ldexp(sum, -(eA + scale_exp(__uint_as_float(umax[1 + m]))));
                    dst[(size_t)m * 2 * n + (size_t)sh * n + ti] = si - sum;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
    if (tid == 0 && *abort_f) atomicExch(status, 1);
}

__global__ void k_tc_sum(size_t len, int S, const double *__restrict__ part, double *__restrict__ out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < S; ++s) v += part[(size_t)s * len + e];
        out[e] = v;
    }
}

// Source splits: the S in 1..8 minimising waves x (tiles per split + the
// epilogue's cost in tiles), one CTA per SM, plus 2 % per extra split for
// the partials' write and sum.  Every split CTA runs the FP64 epilogue
// (S_i Phi_i - total over 64 columns), worth ~32 tiles on GB300 (fitted to
// measured times at N = 8192 .. 65536, M = 60, both formats); a partly
// filled last wave counts as a whole one.
int pick_split(int ctas, int ntiles) {
    constexpr long long kEpiTiles = 32;
    const int sms = device_sm_count();
    int best = 1;
    long long best_cost = -1;
    for (int S = 1; S <= 8 && S <= ntiles; ++S) {
        const long long waves = ((long long)ctas * S + sms - 1) / sms;
        const long long cost = waves * ((ntiles + S - 1) / S + kEpiTiles) * (100 + 2 * (S - 1));
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = S;
        }
    }
    return best;
}

}  // namespace

namespace {

template <bool F16>
int jphi_tc_run(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out,
                cudaStream_t st, int split, int withhold) {
    constexpr uint32_t kImg = img_bytes<F16>(), kSmem = smem_bytes<F16>();
    constexpr int kTSx = tile_sources<F16>();
    static bool attr_set = false;
    if (!attr_set) {
        PTROM_CUDA(cudaFuncSetAttribute(k_jphi_tc<true, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kSmem));
        PTROM_CUDA(cudaFuncSetAttribute(k_jphi_tc<false, F16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kSmem));
        attr_set = true;
    }
    const int nslices = (M + kNC - 1) / kNC;
    const int ntiles = (n + kTSx - 1) / kTSx;
    const int tblocks = (n + kTB - 1) / kTB;
    const int S = split > 0 ? std::min(split, ntiles) : pick_split(tblocks * nslices, ntiles);
    unsigned char *img = nullptr;
    double *part = nullptr;
    int *status = nullptr;
    unsigned *umax = nullptr;
    const size_t len = 2 * (size_t)n * M;
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&img, (size_t)kImg * nslices * ntiles));
    PTROM_TRY(sc.alloc(&status, sizeof(int)));
    if (F16) PTROM_TRY(sc.alloc(&umax, sizeof(unsigned) * (M + 1)));
    if (S > 1) PTROM_TRY(sc.alloc(&part, sizeof(double) * len * S));
    PTROM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
    if (F16) {
        PTROM_CUDA(cudaMemsetAsync(umax, 0, sizeof(unsigned) * (M + 1), st));
        k_tc_maxabs<<<dim3(std::min(64, (2 * n + 255) / 256), M + 1), 256, 0, st>>>(n, G, phi, M, umax);
        count_launch();
    }
    const size_t items = (size_t)nslices * ntiles * (rec_bytes<F16>() / 4 + 2 * kBTile / (F16 ? 2 : 4));
    const int pgrid = (int)std::min<size_t>((items + 255) / 256, (size_t)8 * device_sm_count());
    k_tc_pack<F16><<<pgrid, 256, 0, st>>>(n, x, G, phi, M, nslices, ntiles, umax, img);
    count_launch();
    dim3 grid(tblocks, nslices, S);
    const int slot = timing_begin(PTROM_K_JPHI, st);
    if (delta == 0.0)
        k_jphi_tc<true, F16><<<grid, kThreads, kSmem, st>>>(n, x, phi, M, (float)delta, img, ntiles, umax, out, part,
                                                            status, withhold);
    else
        k_jphi_tc<false, F16><<<grid, kThreads, kSmem, st>>>(n, x, phi, M, (float)delta, img, ntiles, umax, out,
                                                             part, status, withhold);
    cudaError_t e = cudaGetLastError();
    count_launch();
    if (e == cudaSuccess && S > 1) {
        const int rgrid = (int)std::min<size_t>((len + 255) / 256, (size_t)8 * device_sm_count());
        k_tc_sum<<<rgrid, 256, 0, st>>>(len, S, part, out);
        e = cudaGetLastError();
        count_launch();
    }
    timing_end(slot, st);
    if (e != cudaSuccess) return check_cuda(e, "k_jphi_tc launch");
    int h_status = 0;
    PTROM_CUDA(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sc.release());
    if (h_status) return set_error(PTROM_ETIMEOUT, "bs_jphi: a tensor-core pipeline wait gave up");
    return PTROM_OK;
}

}  // namespace

int jphi_tc(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out,
            cudaStream_t st, int split) {
    return jphi_tc_run<false>(n, x, G, delta, phi, M, out, st, split, g_jphi_tc_withhold.exchange(0));
}

// FP16 operands; the power-of-two scaling of the blocks needs delta > 0, so
// delta = 0 takes the TF32 variant.
int jphi_tc_f16(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out,
                cudaStream_t st, int split) {
    const int withhold = g_jphi_tc_withhold.exchange(0);
    if (delta > 0.0) return jphi_tc_run<true>(n, x, G, delta, phi, M, out, st, split, withhold);
    return jphi_tc_run<false>(n, x, G, delta, phi, M, out, st, split, withhold);
}

}  // namespace ptrom

extern "C" int ptrom_test_withhold_jphi_tc(int on) {
    if (on != 0 && on != 1) return ptrom::set_error(PTROM_EINVAL, "ptrom_test_withhold_jphi_tc: on must be 0 or 1");
    ptrom::g_jphi_tc_withhold.store(on);
    return PTROM_OK;
}

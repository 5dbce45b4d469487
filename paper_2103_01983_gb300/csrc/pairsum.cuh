// All-pairs Biot-Savart sums on sm_103a: the tiled target x source skeleton
// shared by the velocity, J v and J^T w kernels.
//
// Geometry (one launch):
//   * a CTA owns 64 * Op::kSets targets; lane l of every warp holds, for
//     each set s, targets tbase + 64 s + l and tbase + 64 s + 32 + l packed
//     in one 2-wide register pair, so the FP32 path runs on the packed
//     FADD2/FMUL2/FFMA2 instructions and every source record read from shared
//     memory serves 2 * kSets pairs per lane (on GB300 a warp's shared-memory
//     read issues at about one per two cycles per SM, close to the FP32 and
//     MUFU rates of one source against two targets);
//   * a pack kernel first converts every source once into an FP32 record laid
//     out the way the inner loop reads it (positions relative to a common
//     origin, negated and duplicated for the packed instructions, gamma =
//     Gamma/(2 pi)); FP64 arithmetic, slow on GB300, thus never runs per pair
//     or per staged chunk;
//   * the CTA's source range is cut into 8 equal contiguous shares, one per
//     warp; each warp walks its share 32 records at a time, staged in its own
//     shared-memory double buffer (coalesced 16-byte loads of the next 32
//     records are in flight while the current ones are consumed), so no
//     CTA-wide barrier sits in the loop;
//   * gridDim.y = S splits the sources further, with one of two combines of
//     the S partial sums of a target block, both in a fixed order (so the
//     result does not depend on which CTA finishes first):
//       - global: each CTA writes its FP64 partial to scratch and the last
//         CTA of the target block to arrive (a counter per target block, zeroed by
//         the pack kernel) adds the S partials in split order and finalises;
//         S <= 16, CTAs scheduled independently;
//       - cluster: the S CTAs of a target block form a thread-block cluster
//         and add their partials through distributed shared memory (no
//         global scratch); S <= 8, the S CTAs are co-scheduled and wait for
//         one another at the end.
// Accumulation: FP32 pair terms summed plainly inside a chunk, then folded
// into a TwoSum-compensated (hi, lo) pair once per chunk; the FP64 variant
// accumulates in FP64 directly.
#pragma once

#include <cooperative_groups.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ptrom {
namespace cg = cooperative_groups;

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 32;     // record padding granularity
#ifndef PTROM_STEP_RECS
#define PTROM_STEP_RECS 1
#endif
constexpr int kStepRecs = PTROM_STEP_RECS;  // records per lane per warp step
constexpr int kStep = 32 * kStepRecs;       // records per warp step (one compensated fold each)
constexpr int kTB = 64;        // targets per set
constexpr int kMaxSets = 4;    // largest Op::kSets
constexpr int kMaxCluster = 8;
constexpr int kMaxSplit = 16;   // largest source split of the global combine
constexpr int kMaxNacc = 5;     // largest number of scalar sums per target of any op
constexpr int kAutoSplit = 4;  // default source split (cluster size)
#ifndef PTROM_PAIR_UNROLL
#define PTROM_PAIR_UNROLL 8
#endif
constexpr int kPairUnroll = PTROM_PAIR_UNROLL;  // unroll of the per-chunk source loop

// ---- 2-wide vector traits: FP32 (packed instructions) or FP64 -----------------
template <typename T> struct VT;
template <> struct VT<float> {
    using V = float2;
    __device__ static __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
#ifdef PTROM_SCALAR_F32
    __device__ static __forceinline__ V add(V a, V b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
    __device__ static __forceinline__ V mul(V a, V b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
    __device__ static __forceinline__ V fma(V a, V b, V c) {
        return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
    }
#else
    __device__ static __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    __device__ static __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    __device__ static __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
#endif
    __device__ static __forceinline__ V rcp(V a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
};
template <> struct VT<double> {
    using V = double2;
    __device__ static __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
    __device__ static __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    __device__ static __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
    __device__ static __forceinline__ V fma(V a, V b, V c) {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
    __device__ static __forceinline__ V rcp(V a) { return make_double2(1.0 / a.x, 1.0 / a.y); }
};

// Accumulator across chunks: compensated for FP32, plain for FP64.
template <typename T> struct Acc;
template <> struct Acc<float> {
    CSum2 s;
    __device__ __forceinline__ void zero() { s.zero(); }
    __device__ __forceinline__ void add(float2 p) { s.add(p); }
    __device__ __forceinline__ double x() const { return s.x(); }
    __device__ __forceinline__ double y() const { return s.y(); }
};
template <> struct Acc<double> {
    double2 s;
    __device__ __forceinline__ void zero() { s = make_double2(0.0, 0.0); }
    __device__ __forceinline__ void add(double2 p) { s.x += p.x; s.y += p.y; }
    __device__ __forceinline__ double x() const { return s.x; }
    __device__ __forceinline__ double y() const { return s.y; }
};

// Zero q where the pair is an exact self/coincident pair (d2 == 0).
template <typename V>
__device__ __forceinline__ V mask_zero(V q, V d2) {
    q.x = (d2.x == 0) ? 0 : q.x;
    q.y = (d2.y == 0) ? 0 : q.y;
    return q;
}

// ---- the skeleton ---------------------------------------------------------
// Op interface (all static):
//   using Args;                        kernel arguments (trivially copyable)
//   NACC                               scalar sums per target
//   kMinBlocks                         resident CTAs per SM the registers must allow
//   kKind                              enum ptrom_kernel_kind (instrumentation)
//   struct Rec {..}                    one packed source (16-byte multiple)
//   struct Tgt {..}                    the lane's two targets
//   origin(args) -> Origin             common origin subtracted before FP32 rounding
//   pack(args, j, Origin) -> Rec       j >= ns -> zero-strength padding
//   load_tgt(args, t0, t1, Origin, Tgt&) t >= nt -> harmless padding
//   pair(const Rec&, Tgt&, V part[NACC])  add one source's contribution
//   finalize(args, t, const double s[NACC])  write target t's outputs
// skip: optional device flag; when it is nonzero at launch the kernel does
// nothing (a speculatively queued launch whose result is not needed).
// cnt (optional, ncnt ints): the global combine's per-target-block arrival
// counters, zeroed here so that the pair launch that follows on the stream
// starts from zero.
template <class Op>
__global__ void __launch_bounds__(256)
pack_kernel(const typename Op::Args args, typename Op::Rec *__restrict__ out, int ns_pad, int *__restrict__ cnt,
            int ncnt, const int *skip) {
    if (skip && *skip) return;
    const typename Op::Origin org = Op::origin(args);
    const int total = ns_pad > ncnt ? ns_pad : ncnt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += gridDim.x * blockDim.x) {
        if (j < ns_pad) out[j] = Op::pack(args, j, org);
        if (j < ncnt) cnt[j] = 0;
    }
}

// Targets per CTA of an op: 64 per set; lane l of every warp holds targets
// 64 s + l and 64 s + 32 + l of each set s < Op::kSets, so every source record
// loaded from shared memory serves 2 kSets pairs per lane.
template <class Op>
constexpr int op_tb() {
    return 64 * Op::kSets;
}

// Shared memory of one pair CTA: the warps' staging double buffers, which
// the cross-warp reduction reuses, and the reduced sums of the CTA's targets.
template <class Op>
struct PairSmem {
    using Rec = typename Op::Rec;
    struct Chunk { Rec r[kStep]; };
    static constexpr int TB = op_tb<Op>();
    static constexpr size_t kStageBytes = sizeof(Chunk) * kWarps * 2;
    static constexpr size_t kRedBytes = sizeof(double) * kWarps * Op::NACC * TB;
    __align__(16) unsigned char raw[kStageBytes > kRedBytes ? kStageBytes : kRedBytes];
    double fin[Op::NACC][TB];
    __device__ Chunk (&stage())[kWarps][2] { return *reinterpret_cast<Chunk(*)[kWarps][2]>(raw); }
    __device__ double (&red())[kWarps][Op::NACC][TB] { return *reinterpret_cast<double(*)[kWarps][Op::NACC][TB]>(raw); }
};

// Sums of the sources in records [r_a, r_b) into acc, for the lane's targets:
// warp w takes an equal contiguous share (to one record) and walks it 32
// records at a time, the last step possibly short, so the 8 warps finish
// together.
template <class Op>
__device__ __forceinline__ void seg_accumulate(const typename Op::Rec *__restrict__ packed, int r_a, int r_b,
                                               const typename Op::Tgt (&tgt)[Op::kSets],
                                               Acc<typename Op::Real> (&acc)[Op::kSets][Op::NACC], PairSmem<Op> &sm) {
    using R = typename Op::Real;
    using V = typename VT<R>::V;
    using Rec = typename Op::Rec;
    constexpr int NACC = Op::NACC;
    constexpr int KS = Op::kSets;
    auto &stage = sm.stage();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int r_len = r_b - r_a;
    const int w_lo = r_a + (int)(((long long)warp * r_len) / kWarps);
    const int w_hi = r_a + (int)(((long long)(warp + 1) * r_len) / kWarps);
    Rec reg[kStepRecs];
#pragma unroll
    for (int p = 0; p < kStepRecs; ++p) {
        reg[p] = Rec{};
        if (w_lo + 32 * p + lane < w_hi) reg[p] = packed[w_lo + 32 * p + lane];
    }
    int b = 0;
    for (int i = w_lo; i < w_hi; i += kStep) {
        const int kn = min(kStep, w_hi - i);
#pragma unroll
        for (int p = 0; p < kStepRecs; ++p) stage[warp][b].r[32 * p + lane] = reg[p];  // slots >= kn are never read
        __syncwarp();
#pragma unroll
        for (int p = 0; p < kStepRecs; ++p)
            if (i + kStep + 32 * p + lane < w_hi) reg[p] = packed[i + kStep + 32 * p + lane];
        V pa[KS][NACC];
#pragma unroll
        for (int q = 0; q < KS; ++q)
#pragma unroll
            for (int k = 0; k < NACC; ++k) pa[q][k] = VT<R>::mk(0, 0);
#pragma unroll kPairUnroll
        for (int k = 0; k < kn; ++k) {
            const Rec rc = stage[warp][b].r[k];  // one shared-memory read per source for all sets
#pragma unroll
            for (int q = 0; q < KS; ++q) Op::pair(rc, tgt[q], pa[q]);
        }
#pragma unroll
        for (int q = 0; q < KS; ++q)
#pragma unroll
            for (int k = 0; k < NACC; ++k) acc[q][k].add(pa[q][k]);
        b ^= 1;
    }
}

// Adds the 8 warps' sums in warp order (FP64) into dst[k * TB + t]; the
// staging storage is reused, so every warp must be done with it.
template <class Op>
__device__ __forceinline__ void reduce_warps(const Acc<typename Op::Real> (&acc)[Op::kSets][Op::NACC], PairSmem<Op> &sm,
                                             double *dst) {
    constexpr int NACC = Op::NACC;
    constexpr int TB = op_tb<Op>();
    auto &red = sm.red();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Op::kSets; ++q)
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            red[warp][k][64 * q + lane] = acc[q][k].x();
            red[warp][k][64 * q + 32 + lane] = acc[q][k].y();
        }
    __syncthreads();
    for (int e = threadIdx.x; e < NACC * TB; e += kThreads) {
        const int k = e / TB, t = e % TB;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += red[w][k][t];
        dst[e] = s;
    }
}

// Writes the outputs of targets tbase .. tbase + TB - 1 from sm.fin.
template <class Op>
__device__ __forceinline__ void finalize_block(const typename Op::Args &args, int tbase, PairSmem<Op> &sm) {
    for (int tl = threadIdx.x; tl < op_tb<Op>(); tl += kThreads) {
        const int t = tbase + tl;
        if (t < Op::num_targets(args)) {
            double s[Op::NACC];
#pragma unroll
            for (int k = 0; k < Op::NACC; ++k) s[k] = sm.fin[k][tl];
            Op::finalize(args, t, s);
        }
    }
}

// One CTA's work: targets tbase .. tbase + op_tb<Op>() - 1 against the sources
// of this CTA's split (gridDim.y) of `nchunks` packed chunks.
// part/cnt: the global combine's scratch (nullptr: cluster combine when
// gridDim.y > 1); bx: this target block's index into them.
template <class Op>
__device__ __forceinline__ void pair_block(const typename Op::Args &args, const typename Op::Rec *__restrict__ packed,
                                           int nchunks, int tbase, double *__restrict__ part = nullptr,
                                           int *__restrict__ cnt = nullptr, int bx = 0) {
    using R = typename Op::Real;
    constexpr int NACC = Op::NACC;
    constexpr int KS = Op::kSets;
    constexpr int TB = op_tb<Op>();
    __shared__ PairSmem<Op> sm;
    auto &fin = sm.fin;
    const int lane = threadIdx.x & 31;

    const typename Op::Origin org = Op::origin(args);
    typename Op::Tgt tgt[KS];
#pragma unroll
    for (int q = 0; q < KS; ++q) Op::load_tgt(args, tbase + 64 * q + lane, tbase + 64 * q + 32 + lane, org, tgt[q]);

    Acc<R> acc[KS][NACC];
#pragma unroll
    for (int q = 0; q < KS; ++q)
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[q][k].zero();

    const int c_begin = (int)(((long long)blockIdx.y * nchunks) / gridDim.y);
    const int c_end = (int)(((long long)(blockIdx.y + 1) * nchunks) / gridDim.y);
    seg_accumulate<Op>(packed, c_begin * kChunk, c_end * kChunk, tgt, acc, sm);

    const int S = gridDim.y;
    double *mine = (S > 1 && part) ? part + ((size_t)bx * S + blockIdx.y) * (NACC * TB) : nullptr;
    reduce_warps<Op>(acc, sm, mine ? mine : &fin[0][0]);

    if (mine) {
        // global combine: the last of the S CTAs of this target block adds the
        // S partials in split order (release: fence before the counter;
        // acquire: fence after it, loads that bypass L1)
        __shared__ int s_last;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(&cnt[bx], 1) == S - 1;
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        const double *base = part + (size_t)bx * S * (NACC * TB);
        for (int e = threadIdx.x; e < NACC * TB; e += kThreads) {
            double s = 0.0;
            for (int r = 0; r < S; ++r) s += __ldcg(base + (size_t)r * (NACC * TB) + e);
            fin[e / TB][e % TB] = s;
        }
    }
    if (mine || S == 1) {
        __syncthreads();
        finalize_block<Op>(args, tbase, sm);
        return;
    }
    // cluster of S CTAs along y: rank r finalises targets t with t % S == r
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    const int rank = (int)cluster.block_rank();
    for (int tl = rank + (int)threadIdx.x * S; tl < TB; tl += kThreads * S) {
        double s[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) s[k] = 0.0;
        for (int r = 0; r < S; ++r) {
            const double *peer = cluster.map_shared_rank(&fin[0][0], r);
#pragma unroll
            for (int k = 0; k < NACC; ++k) s[k] += peer[k * TB + tl];
        }
        const int t = tbase + tl;
        if (t < Op::num_targets(args)) Op::finalize(args, t, s);
    }
    cluster.sync();
}

template <class Op>
__global__ void __launch_bounds__(kThreads, Op::kMinBlocks)
pair_kernel(const typename Op::Args args, const typename Op::Rec *__restrict__ packed, int nchunks, const int *skip,
            double *part, int *cnt) {
    if (skip && *skip) return;  // uniform over the grid: no CTA reaches a cluster barrier
    pair_block<Op>(args, packed, nchunks, blockIdx.x * op_tb<Op>(), part, cnt, blockIdx.x);
}

// Batched launch: instance b owns CTAs prefix[b] .. prefix[b+1]-1 along x.
template <class Op>
struct BatchItem {
    typename Op::Args args;
    const typename Op::Rec *packed;
    int nchunks;
};

template <class Op>
__global__ void __launch_bounds__(kThreads, Op::kMinBlocks)
pair_kernel_batched(const BatchItem<Op> *__restrict__ items, const int *__restrict__ prefix, int B) {
    int lo = 0, hi = B - 1;  // largest b with prefix[b] <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const BatchItem<Op> it = items[lo];
    pair_block<Op>(it.args, it.packed, it.nchunks, ((int)blockIdx.x - prefix[lo]) * op_tb<Op>());
}

// Batched packing: record e of the flattened list belongs to the instance b
// with rec_prefix[b] <= e < rec_prefix[b+1].
template <class Op>
__global__ void __launch_bounds__(256)
pack_kernel_batched(const BatchItem<Op> *__restrict__ items, const int *__restrict__ rec_prefix, int B,
                    typename Op::Rec *__restrict__ out) {
    const int total = rec_prefix[B];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rec_prefix[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const typename Op::Args &a = items[lo].args;
        out[e] = Op::pack(a, e - rec_prefix[lo], Op::origin(a));
    }
}

// Scratch of one launch with split S: packed records, then (S > 1, global
// combine) the FP64 partials of every (target block, split) and the
// per-target-block counters, each region 256-byte aligned.
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
struct PairScratchLayout {
    size_t rec, part, cnt, total;
};
inline PairScratchLayout pair_scratch_layout(size_t rec_bytes, int nacc, int tb, int nt, int ns, int S,
                                             bool global) {
    const size_t tblocks = ((size_t)nt + tb - 1) / tb;
    const size_t ns_pad = ((size_t)ns + kChunk - 1) / kChunk * kChunk;
    PairScratchLayout L;
    L.rec = 0;
    L.part = align256(rec_bytes * ns_pad);
    const size_t part_bytes = (global && S > 1) ? align256(sizeof(double) * (size_t)nacc * tb * tblocks * S) : 0;
    L.cnt = L.part + part_bytes;
    L.total = L.cnt + ((global && S > 1) ? align256(sizeof(int) * tblocks) : 0);
    return L;
}

// Launch helper: packs the sources (into `scratch` when given, else into a
// stream-ordered allocation freed right after), picks the source split S and
// its combine and launches the pair kernel.
//   * S = 4 (fewer when the warps would run out of chunks), or forced;
//   * global combine (default, S <= 16): used when the scratch has room for
//     the partials (a caller's scratch of pack_scratch_bytes(nt, ns) bytes
//     always has);
//   * cluster combine (S <= 8): used when forced by ptrom_set_split_mode(1)
//     or when a caller's scratch holds the packed records only.
// Measured on GB300 at N = 4096 .. 65536 for every op, S = 4 is within a few
// per cent of the best S in 1..16 with either combine, and the global combine
// is 0-4 % faster than the cluster one (its CTAs need not be co-scheduled nor
// wait for one another).
// One pack + pair launch with split S and the given combine, on buf (at least
// pair_scratch_layout(..., S, global).total bytes).
template <class Op>
cudaError_t launch_pairs_on(const typename Op::Args &args, int nt, int ns, cudaStream_t stream, const LaunchOpts &o,
                            int S, bool global, char *buf) {
    using Rec = typename Op::Rec;
    constexpr int TB = op_tb<Op>();
    const int tblocks = (nt + TB - 1) / TB;
    const int nchunks = (ns + kChunk - 1) / kChunk;
    const int ns_pad = nchunks * kChunk;
    const PairScratchLayout L = pair_scratch_layout(sizeof(Rec), Op::NACC, TB, nt, ns, S, global);
    Rec *packed = reinterpret_cast<Rec *>(buf + L.rec);
    double *part = (global && S > 1) ? reinterpret_cast<double *>(buf + L.part) : nullptr;
    int *cnt = (global && S > 1) ? reinterpret_cast<int *>(buf + L.cnt) : nullptr;
    const int ncnt = cnt ? tblocks : 0;
    const int pwork = ns_pad > ncnt ? ns_pad : ncnt;
    int pgrid = (pwork + 255) / 256;
    if (pgrid > 4 * device_sm_count()) pgrid = 4 * device_sm_count();
    const int pslot = timing_begin(PTROM_K_PACK, stream);
    pack_kernel<Op><<<pgrid, 256, 0, stream>>>(args, packed, ns_pad, cnt, ncnt, o.skip);
    timing_end(pslot, stream);
    if (o.slots) o.slots->add(pslot);
    count_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tblocks, S, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = global ? 1 : S;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = global ? 0 : 1;
    const int slot = timing_begin(Op::kKind, stream);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, pair_kernel<Op>, args, (const Rec *)packed, nchunks, o.skip,
                                             part, cnt);
    timing_end(slot, stream);
    if (o.slots) o.slots->add(slot);
    if (e == cudaSuccess) count_launch();
    return e;
}

// Autotuning of the global combine's split: every candidate S is launched
// three times on the caller's data (the first as warm-up) and timed with CUDA
// events on the stream; the fastest S is cached per (kernel, nt, ns).  The
// outputs are those of the last launch, which the caller's launch overwrites.
template <class Op>
int tune_split(const typename Op::Args &args, int nt, int ns, cudaStream_t stream, const LaunchOpts &o, int *best) {
    using Rec = typename Op::Rec;
    constexpr int TB = op_tb<Op>();
    const int nchunks = (ns + kChunk - 1) / kChunk;
    static const int cands[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16};
    const size_t need = pair_scratch_layout(sizeof(Rec), Op::NACC, TB, nt, ns, kMaxSplit, true).total;
    char *buf = reinterpret_cast<char *>(o.scratch);
    const bool own = !(buf && o.scratch_bytes >= need);
    if (own) PTROM_TRY(scratch_alloc((void **)&buf, need, stream));
    cudaEvent_t ev[2];
    PTROM_CUDA(cudaEventCreate(&ev[0]));
    PTROM_CUDA(cudaEventCreate(&ev[1]));
    float best_ms = -1.f;
    int bS = 1;
    cudaError_t e = cudaSuccess;
    for (int S : cands) {
        if (S > 1 && nchunks < 8 * S) break;  // every warp keeps a step of 32 records
        float tmin = -1.f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(ev[0], stream);
            if (e == cudaSuccess) e = launch_pairs_on<Op>(args, nt, ns, stream, o, S, true, buf);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (rep > 0 && (tmin < 0.f || ms < tmin)) tmin = ms;
        }
        if (e != cudaSuccess) break;
        if (best_ms < 0.f || tmin < best_ms) {
            best_ms = tmin;
            bS = S;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    const int s2 = own ? scratch_free(buf, stream) : PTROM_OK;
    if (e != cudaSuccess) return check_cuda(e, "pair split autotuning");
    PTROM_TRY(s2);
    store_tuned_split(reinterpret_cast<const void *>(pair_kernel<Op>), nt, ns, bS);
    *best = bS;
    return PTROM_OK;
}

template <class Op>
int launch_pairs(const typename Op::Args &args, int nt, int ns, cudaStream_t stream, const LaunchOpts &o = {}) {
    using Rec = typename Op::Rec;
    constexpr int NACC = Op::NACC;
    constexpr int TB = op_tb<Op>();
    const int nchunks = (ns + kChunk - 1) / kChunk;
    const int forced = o.split > 0 ? o.split : g_source_split.load();
    const int mode = g_split_mode.load();
    bool global = mode != 1;
    int S = forced;
    if (S <= 0) {
        S = kAutoSplit;
        while (S > 1 && nchunks < S * kWarps) --S;
        if (global) {
            const int t = tuned_split(reinterpret_cast<const void *>(pair_kernel<Op>), nt, ns);
            if (t > 0) {
                S = t;
            } else if ((o.tune || g_autotune.load()) && !o.skip) {
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
                    PTROM_TRY(tune_split<Op>(args, nt, ns, stream, o, &S));
            }
        }
    }
    if (global && o.scratch && pair_scratch_layout(sizeof(Rec), NACC, TB, nt, ns, S, true).total > o.scratch_bytes) {
        if (mode == 2) return set_error(PTROM_ENOMEM, "pair launch: scratch too small for the global combine");
        global = false;  // the caller's scratch holds the records only
    }
    if (!global && S > kMaxCluster)
        return set_error(PTROM_EINVAL, "pair launch: cluster split %d > %d", S, kMaxCluster);
    if (S < 1 || S > kMaxSplit) return set_error(PTROM_EINVAL, "bad source split %d", S);
    const PairScratchLayout L = pair_scratch_layout(sizeof(Rec), NACC, TB, nt, ns, S, global);
    char *buf = reinterpret_cast<char *>(o.scratch);
    const bool own = buf == nullptr;
    if (own) PTROM_TRY(scratch_alloc((void **)&buf, L.total, stream));
    const cudaError_t e = launch_pairs_on<Op>(args, nt, ns, stream, o, S, global, buf);
    if (own) {
        const int s2 = scratch_free(buf, stream);
        if (e == cudaSuccess && s2 != PTROM_OK) return s2;
    }
    if (e != cudaSuccess) return check_cuda(e, "pair_kernel launch");
    return PTROM_OK;
}

// Batched launch over B instances: args[b], nt[b] targets, ns[b] sources.
// One pack launch and one cluster launch (split S for every instance).
template <class Op>
int launch_pairs_batched(const typename Op::Args *args, const int *nt, const int *ns, int B, cudaStream_t stream,
                         int S) {
    using Rec = typename Op::Rec;
    if (B < 1) return PTROM_OK;
    if (S < 1 || S > kMaxCluster) return set_error(PTROM_EINVAL, "bad source split %d", S);
    std::vector<BatchItem<Op>> items(B);
    std::vector<int> prefix(B + 1, 0), rprefix(B + 1, 0);
    for (int b = 0; b < B; ++b) {
        const int nchunks = (ns[b] + kChunk - 1) / kChunk;
        items[b].args = args[b];
        items[b].nchunks = nchunks;
        prefix[b + 1] = prefix[b] + (nt[b] + op_tb<Op>() - 1) / op_tb<Op>();
        rprefix[b + 1] = rprefix[b] + nchunks * kChunk;
    }
    const size_t head = ((sizeof(BatchItem<Op>) * B + 2 * sizeof(int) * (B + 1)) + 255) & ~size_t(255);
    char *buf = nullptr;
    PTROM_TRY(scratch_alloc((void **)&buf, head + sizeof(Rec) * (size_t)rprefix[B], stream));
    Rec *packed = reinterpret_cast<Rec *>(buf + head);
    for (int b = 0; b < B; ++b) items[b].packed = packed + rprefix[b];
    BatchItem<Op> *ditems = reinterpret_cast<BatchItem<Op> *>(buf);
    int *dprefix = reinterpret_cast<int *>(buf + sizeof(BatchItem<Op>) * B);
    int *drprefix = dprefix + (B + 1);
    std::vector<char> hostbuf(head);
    memcpy(hostbuf.data(), items.data(), sizeof(BatchItem<Op>) * B);
    memcpy(hostbuf.data() + sizeof(BatchItem<Op>) * B, prefix.data(), sizeof(int) * (B + 1));
    memcpy(hostbuf.data() + sizeof(BatchItem<Op>) * B + sizeof(int) * (B + 1), rprefix.data(), sizeof(int) * (B + 1));
    cudaError_t e = cudaMemcpyAsync(buf, hostbuf.data(), head, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        int pgrid = (rprefix[B] + 255) / 256;
        if (pgrid > 8 * device_sm_count()) pgrid = 8 * device_sm_count();
        pack_kernel_batched<Op><<<pgrid, 256, 0, stream>>>(ditems, drprefix, B, packed);
        count_launch();
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(prefix[B], S, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = S;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const int slot = timing_begin(Op::kKind, stream);
        e = cudaLaunchKernelEx(&cfg, pair_kernel_batched<Op>, (const BatchItem<Op> *)ditems, (const int *)dprefix, B);
        timing_end(slot, stream);
        if (e == cudaSuccess) count_launch();
    }
    const int s2 = scratch_free(buf, stream);
    if (e != cudaSuccess) return check_cuda(e, "pair_kernel_batched launch");
    return s2;
}

// Bytes of scratch one launch over nt targets and ns sources needs with the
// global combine at any split up to kMaxSplit (upper bound over all ops:
// records of at most 96 bytes (FP64), at most kMaxNacc sums per target; the
// partials of a split take NACC doubles per target, rounded up to whole target
// blocks of at most kTB * kMaxSets targets).
inline size_t pack_scratch_bytes_impl(int nt, int ns) {
    return pair_scratch_layout(96, kMaxNacc, kTB * kMaxSets, nt, ns, kMaxSplit, true).total;
}

}  // namespace ptrom

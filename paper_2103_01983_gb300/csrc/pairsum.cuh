// All-pairs Biot-Savart sums on sm_103a: the tiled target x source skeleton
// shared by the velocity, J v and J^T w kernels.
//
// Geometry (one launch):
//   * a CTA owns kTB = 64 targets; lane l of every warp holds targets
//     tbase + l and tbase + 32 + l packed in one 2-wide register pair, so the
//     FP32 path runs on the packed FADD2/FMUL2/FFMA2 instructions;
//   * a pack kernel first converts every source once into an FP32 record laid
//     out the way the inner loop reads it (positions relative to a common
//     origin, negated and duplicated for the packed instructions, gamma =
//     Gamma/(2 pi)); FP64 arithmetic, slow on GB300, thus never runs per pair
//     or per staged chunk;
//   * the CTA's source range is cut into chunks of 32 records dealt
//     round-robin to its 8 warps; each warp stages its chunk in its own
//     shared-memory double buffer (coalesced 16-byte loads of the next chunk are
//     in flight while the current one is consumed), so no CTA-wide barrier
//     sits in the loop;
//   * gridDim.y (default 4) splits the sources further; the gridDim.y CTAs
//     of one target block form a thread-block cluster and reduce their partial sums through
//     distributed shared memory in a fixed order (deterministic, no atomics,
//     no global scratch).
// Accumulation: FP32 pair terms summed plainly inside a chunk, then folded
// into a TwoSum-compensated (hi, lo) pair once per chunk; the FP64 variant
// accumulates in FP64 directly.
#pragma once

#include <cooperative_groups.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ptrom {
namespace cg = cooperative_groups;

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kChunk = 32;
constexpr int kTB = 64;
constexpr int kMaxCluster = 8;
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
template <class Op>
__global__ void __launch_bounds__(256)
pack_kernel(const typename Op::Args args, typename Op::Rec *__restrict__ out, int ns_pad, const int *skip) {
    if (skip && *skip) return;
    const typename Op::Origin org = Op::origin(args);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns_pad; j += gridDim.x * blockDim.x)
        out[j] = Op::pack(args, j, org);
}

// One CTA's work: targets tbase .. tbase+63 against the sources of this
// CTA's split (gridDim.y) of `nchunks` packed chunks.
template <class Op>
__device__ __forceinline__ void pair_block(const typename Op::Args &args, const typename Op::Rec *__restrict__ packed,
                                           int nchunks, int tbase) {
    using R = typename Op::Real;
    using V = typename VT<R>::V;
    using Rec = typename Op::Rec;
    constexpr int NACC = Op::NACC;
    struct Chunk { Rec r[kChunk]; };

    // the staging buffers and the cross-warp reduction buffer share storage
    constexpr size_t kStageBytes = sizeof(Chunk) * kWarps * 2;
    constexpr size_t kRedBytes = sizeof(double) * kWarps * NACC * kTB;
    __shared__ __align__(16) unsigned char smraw[kStageBytes > kRedBytes ? kStageBytes : kRedBytes];
    __shared__ double fin[NACC][kTB];
    auto &stage = *reinterpret_cast<Chunk(*)[kWarps][2]>(smraw);
    auto &red = *reinterpret_cast<double(*)[kWarps][NACC][kTB]>(smraw);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    const typename Op::Origin org = Op::origin(args);
    typename Op::Tgt tgt;
    Op::load_tgt(args, tbase + lane, tbase + 32 + lane, org, tgt);

    Acc<R> acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k].zero();

    const int c_begin = (int)(((long long)blockIdx.y * nchunks) / gridDim.y);
    const int c_end = (int)(((long long)(blockIdx.y + 1) * nchunks) / gridDim.y);

    Rec reg;
    int c = c_begin + warp;
    if (c < c_end) reg = packed[c * kChunk + lane];
    int b = 0;
    for (; c < c_end; c += kWarps) {
        stage[warp][b].r[lane] = reg;
        __syncwarp();
        const int cn = c + kWarps;
        if (cn < c_end) reg = packed[cn * kChunk + lane];
        V part[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) part[k] = VT<R>::mk(0, 0);
#pragma unroll kPairUnroll
        for (int k = 0; k < kChunk; ++k) Op::pair(stage[warp][b].r[k], tgt, part);
#pragma unroll
        for (int k = 0; k < NACC; ++k) acc[k].add(part[k]);
        b ^= 1;
    }

    // reduce the 8 warps (fixed order); the staging storage is reused
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
        red[warp][k][lane] = acc[k].x();
        red[warp][k][32 + lane] = acc[k].y();
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NACC * kTB; e += kThreads) {
        const int k = e / kTB, t = e % kTB;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += red[w][k][t];
        fin[k][t] = s;
    }

    const int S = gridDim.y;
    if (S == 1) {
        __syncthreads();
        if (threadIdx.x < kTB) {
            const int t = tbase + threadIdx.x;
            if (t < Op::num_targets(args)) {
                double s[NACC];
#pragma unroll
                for (int k = 0; k < NACC; ++k) s[k] = fin[k][threadIdx.x];
                Op::finalize(args, t, s);
            }
        }
        return;
    }
    // cluster of S CTAs along y: rank r finalises targets t with t % S == r
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    const int rank = (int)cluster.block_rank();
    for (int tl = rank + (int)threadIdx.x * S; tl < kTB; tl += kThreads * S) {
        double s[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) s[k] = 0.0;
        for (int r = 0; r < S; ++r) {
            const double *peer = cluster.map_shared_rank(&fin[0][0], r);
#pragma unroll
            for (int k = 0; k < NACC; ++k) s[k] += peer[k * kTB + tl];
        }
        const int t = tbase + tl;
        if (t < Op::num_targets(args)) Op::finalize(args, t, s);
    }
    cluster.sync();
}

template <class Op>
__global__ void __launch_bounds__(kThreads, Op::kMinBlocks)
pair_kernel(const typename Op::Args args, const typename Op::Rec *__restrict__ packed, int nchunks, const int *skip) {
    if (skip && *skip) return;  // uniform over the grid: no CTA reaches a cluster barrier
    pair_block<Op>(args, packed, nchunks, blockIdx.x * kTB);
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
    pair_block<Op>(it.args, it.packed, it.nchunks, ((int)blockIdx.x - prefix[lo]) * kTB);
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

// Launch helper: packs the sources (into `scratch` when given, else into a
// stream-ordered allocation freed right after), picks the cluster split S
// (1..8) and launches the pair kernel.
template <class Op>
int launch_pairs(const typename Op::Args &args, int nt, int ns, cudaStream_t stream, const LaunchOpts &o = {}) {
    const int force_split = o.split;
    void *scratch = o.scratch;
    using Rec = typename Op::Rec;
    const int tblocks = (nt + kTB - 1) / kTB;
    const int nchunks = (ns + kChunk - 1) / kChunk;
    const int ns_pad = nchunks * kChunk;
    int S = 1;
    const int forced = force_split > 0 ? force_split : g_source_split.load();
    if (forced > 0) {
        S = forced;
    } else {
        // kAutoSplit CTAs per target block, fewer when the warps would run out
        // of chunks: measured on GB300 at N = 4096 .. 65536, a split of 4 is
        // within a few per cent of the best split for every op, while larger
        // splits (more, shorter CTAs that fill the last wave) lose more to the
        // per-CTA prologue and cluster reduction than they gain.
        S = kAutoSplit;
        while (S > 1 && nchunks < S * kWarps) --S;
    }
    if (S < 1 || S > kMaxCluster) return set_error(PTROM_EINVAL, "bad source split %d", S);
    Rec *packed = reinterpret_cast<Rec *>(scratch);
    const bool own = packed == nullptr;
    if (own) PTROM_TRY(scratch_alloc((void **)&packed, sizeof(Rec) * (size_t)ns_pad, stream));
    int pgrid = (ns_pad + 255) / 256;
    if (pgrid > 4 * device_sm_count()) pgrid = 4 * device_sm_count();
    const int pslot = timing_begin(PTROM_K_PACK, stream);
    pack_kernel<Op><<<pgrid, 256, 0, stream>>>(args, packed, ns_pad, o.skip);
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
    attr[0].val.clusterDim.y = S;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int slot = timing_begin(Op::kKind, stream);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, pair_kernel<Op>, args, (const Rec *)packed, nchunks, o.skip);
    timing_end(slot, stream);
    if (o.slots) o.slots->add(slot);
    if (own) {
        const int s2 = scratch_free(packed, stream);
        if (e == cudaSuccess && s2 != PTROM_OK) return s2;
    }
    if (e != cudaSuccess) return check_cuda(e, "pair_kernel launch");
    count_launch();
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
        prefix[b + 1] = prefix[b] + (nt[b] + kTB - 1) / kTB;
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

// Bytes of packed-source scratch one launch over ns sources needs (upper
// bound over all ops: 48-byte FP32 records, 96-byte FP64 records).
inline size_t pack_scratch_bytes_impl(int ns) {
    const size_t pad = ((size_t)ns + kChunk - 1) / kChunk * kChunk;
    return pad * 96;
}

}  // namespace ptrom

// bs_jphi: the kernel Jacobian applied to every column of a basis,
//     (J Phi)_i = sum_{j != i} gamma_j A(x_i - x_j) (Phi_i - Phi_j)
// (the J Phi of the LSPG Gauss-Newton problem, Sec. 3.2, with J = d f/d x).
//
// One thread per target, 12 basis columns per grid.y slice: the 2x2 pair block
// gamma_j A is generated once per pair on the FP32 pipes and applied to the 12
// columns' row differences with packed FFMA2 (two columns per instruction).
// Sources are packed once (positions relative to a common origin, gamma, and
// their 12 negated Phi rows per slice) and staged 32 at a time in shared
// memory.  Accumulation: the 32 pair terms of a staged round are summed in
// plain FP32, then folded into a TwoSum-compensated (hi, lo) pair per output.
// gridDim.z splits the sources; each split writes its FP64 partial to
// scratch and a second kernel adds the splits in split order, so results are
// the same run to run.  An FP64 variant (one thread per target and column)
// serves checking.
#include <algorithm>

#include "common.cuh"
#include "scratch.h"
#include "internal.h"

namespace ptrom {
// J Phi on the tensor cores with FP16 operands (jphi_tc.cu; delta = 0 falls
// back to TF32); split as jphi.
int jphi_tc_f16(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out,
                cudaStream_t st, int split);
namespace {

constexpr int kJT = 128;  // targets per CTA
// basis columns per slice: 12 (measured on GB300 against 8 and 16 with the
// compensated sums: 16 needs 190 registers per thread, 8 repeats the pair
// block's generation too often; at N = 65536, M = 60: 6.2e10, 6.7e10 and
// 6.0e10 pairs/s for 8, 12 and 16)
constexpr int kMC = 12;
constexpr int kJS = 32;   // sources per shared-memory round

struct __align__(16) JRec {
    float nx, ny, g, pad;
    float2 nc[kMC / 2];  // -Phi rows, chi component, column pairs
    float2 np[kMC / 2];  // -Phi rows, psi component
};

__global__ void k_jphi_pack(int n, const double *x, const double *G, const double *phi, int M, int nslices,
                            int ns_pad, JRec *out) {
    const double ox = x[0], oy = x[n];
    const int total = nslices * ns_pad;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int slice = e / ns_pad, j = e % ns_pad;
        JRec r;
        const bool in = j < n;
        r.nx = in ? (float)(-(x[j] - ox)) : 0.f;
        r.ny = in ? (float)(-(x[n + j] - oy)) : 0.f;
        r.g = in ? (float)(G[j] * kInv2Pi) : 0.f;
        r.pad = 0.f;
        for (int k = 0; k < kMC / 2; ++k) {
            float c[2], p[2];
            for (int h = 0; h < 2; ++h) {
                const int m = slice * kMC + 2 * k + h;
                const bool ok = in && m < M;
                c[h] = ok ? (float)(-phi[(size_t)m * 2 * n + j]) : 0.f;
                p[h] = ok ? (float)(-phi[(size_t)m * 2 * n + n + j]) : 0.f;
            }
            r.nc[k] = make_float2(c[0], c[1]);
            r.np[k] = make_float2(p[0], p[1]);
        }
        out[e] = r;
    }
}

template <bool MASK>
__global__ void __launch_bounds__(kJT)
k_jphi(int n, const double *x, const double *phi, int M, float delta, const JRec *__restrict__ packed, int ns_pad,
       int nchunks, double *out, double *part) {
    __shared__ JRec src[kJS];
    const int i = blockIdx.x * kJT + threadIdx.x;
    const int slice = blockIdx.y;
    const bool active = i < n;
    const double ox = x[0], oy = x[n];
    const float tx = active ? (float)(x[i] - ox) : 0.f, ty = active ? (float)(x[n + i] - oy) : 0.f;
    float2 pc[kMC / 2], pp[kMC / 2];
    CSum2 ac[kMC / 2], ap[kMC / 2];  // compensated sums over rounds
#pragma unroll
    for (int k = 0; k < kMC / 2; ++k) {
        float c[2], p[2];
        for (int h = 0; h < 2; ++h) {
            const int m = slice * kMC + 2 * k + h;
            const bool ok = active && m < M;
            c[h] = ok ? (float)phi[(size_t)m * 2 * n + i] : 0.f;
            p[h] = ok ? (float)phi[(size_t)m * 2 * n + n + i] : 0.f;
        }
        pc[k] = make_float2(c[0], c[1]);
        pp[k] = make_float2(p[0], p[1]);
        ac[k].zero();
        ap[k].zero();
    }
    const JRec *base = packed + (size_t)slice * ns_pad;
    const int c_begin = (int)(((long long)blockIdx.z * nchunks) / gridDim.z);
    const int c_end = (int)(((long long)(blockIdx.z + 1) * nchunks) / gridDim.z);
    for (int c = c_begin; c < c_end; ++c) {
        __syncthreads();
        for (int e = threadIdx.x; e < kJS * (int)(sizeof(JRec) / 16); e += kJT)
            reinterpret_cast<float4 *>(src)[e] = __ldg(reinterpret_cast<const float4 *>(base + (size_t)c * kJS) + e);
        __syncthreads();
        float2 tc[kMC / 2], tq[kMC / 2];  // this round's plain FP32 sums
#pragma unroll
        for (int k = 0; k < kMC / 2; ++k) {
            tc[k] = make_float2(0.f, 0.f);
            tq[k] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int s = 0; s < kJS; ++s) {
            const JRec &r = src[s];
            const float a = tx + r.nx, b = ty + r.ny;
            const float d2 = fmaf(a, a, b * b);
            float rr = rcp_approx(d2 + delta);
            if (MASK) rr = d2 == 0.f ? 0.f : rr;
            const float q = r.g * rr;
            const float p2 = 2.f * q * rr;
            const float pa = p2 * a, pb = p2 * b;
            const float a00 = pa * b, a01 = fmaf(pb, b, -q), a10 = fmaf(-pa, a, q);
            const float2 A00 = make_float2(a00, a00), A01 = make_float2(a01, a01), A10 = make_float2(a10, a10),
                         N00 = make_float2(-a00, -a00);
#pragma unroll
            for (int k = 0; k < kMC / 2; ++k) {
                const float2 dc = __fadd2_rn(pc[k], r.nc[k]);
                const float2 dp = __fadd2_rn(pp[k], r.np[k]);
                tc[k] = __ffma2_rn(A00, dc, tc[k]);
                tc[k] = __ffma2_rn(A01, dp, tc[k]);
                tq[k] = __ffma2_rn(A10, dc, tq[k]);
                tq[k] = __ffma2_rn(N00, dp, tq[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kMC / 2; ++k) {
            ac[k].add(tc[k]);
            ap[k].add(tq[k]);
        }
    }
    if (!active) return;
    // one split: the output itself; several: this split's slab of the partials
    double *dst = gridDim.z > 1 ? part + (size_t)blockIdx.z * 2 * n * M : out;
#pragma unroll
    for (int k = 0; k < kMC / 2; ++k) {
        const double vc[2] = {ac[k].x(), ac[k].y()}, vp[2] = {ap[k].x(), ap[k].y()};
        for (int h = 0; h < 2; ++h) {
            const int m = slice * kMC + 2 * k + h;
            if (m >= M) continue;
            dst[(size_t)m * 2 * n + i] = vc[h];
            dst[(size_t)m * 2 * n + n + i] = vp[h];
        }
    }
}

// out = sum over the S splits' partials, in split order.
__global__ void k_jphi_sum(size_t len, int S, const double *__restrict__ part, double *__restrict__ out) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < S; ++s) v += part[(size_t)s * len + e];
        out[e] = v;
    }
}

// FP64 variant: one thread per (target, column), plain double loops.
__global__ void k_jphi64(int n, const double *x, const double *G, double delta, const double *phi, int M,
                         double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (i >= n) return;
    const double *col = phi + (size_t)m * 2 * n;
    const double pci = col[i], ppi = col[n + i];
    double sc = 0.0, sp = 0.0;
    for (int j = 0; j < n; ++j) {
        const double a = x[i] - x[j], b = x[n + i] - x[n + j];
        const double d2 = a * a + b * b;
        if (d2 == 0.0) continue;
        const double rr = 1.0 / (d2 + delta);
        const double q = G[j] * kInv2Pi * rr, p2 = 2.0 * q * rr;
        const double a00 = p2 * a * b, a01 = p2 * b * b - q, a10 = q - p2 * a * a;
        const double dc = pci - col[j], dp = ppi - col[n + j];
        sc += a00 * dc + a01 * dp;
        sp += a10 * dc - a00 * dp;
    }
    out[(size_t)m * 2 * n + i] = sc;
    out[(size_t)m * 2 * n + n + i] = sp;
}

}  // namespace

int jphi(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out, int prec,
         cudaStream_t st, int split) {
    if (prec == PTROM_TF32X3) return jphi_tc(n, x, G, delta, phi, M, out, st, split);
    if (prec == PTROM_F16X3) return jphi_tc_f16(n, x, G, delta, phi, M, out, st, split);
    if (prec == PTROM_FP64) {
        dim3 grid((n + 127) / 128, M);
        const int slot = timing_begin(PTROM_K_JPHI, st);
        k_jphi64<<<grid, 128, 0, st>>>(n, x, G, delta, phi, M, out);
        timing_end(slot, st);
        PTROM_CUDA(cudaGetLastError());
        count_launch();
        return PTROM_OK;
    }
    const int nslices = (M + kMC - 1) / kMC;
    const int nchunks = (n + kJS - 1) / kJS;
    const int ns_pad = nchunks * kJS;
    const int tblocks = (n + kJT - 1) / kJT;
    int S = split;
    if (S <= 0) {  // fill about 4 waves of 8 CTAs per SM
        const long long want = 4LL * 8 * device_sm_count();
        S = 1;
        while ((long long)tblocks * nslices * S * 2 <= want && (S * 2) * 4 <= nchunks) S *= 2;
    }
    JRec *packed = nullptr;
    double *part = nullptr;
    const size_t len = 2 * (size_t)n * M;
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&packed, sizeof(JRec) * (size_t)nslices * ns_pad));
    if (S > 1) PTROM_TRY(sc.alloc(&part, sizeof(double) * len * S));
    int pgrid = (nslices * ns_pad + 255) / 256;
    if (pgrid > 8 * device_sm_count()) pgrid = 8 * device_sm_count();
    k_jphi_pack<<<pgrid, 256, 0, st>>>(n, x, G, phi, M, nslices, ns_pad, packed);
    count_launch();
    dim3 grid(tblocks, nslices, S);
    const int slot = timing_begin(PTROM_K_JPHI, st);
    if (delta == 0.0)
        k_jphi<true><<<grid, kJT, 0, st>>>(n, x, phi, M, (float)delta, packed, ns_pad, nchunks, out, part);
    else
        k_jphi<false><<<grid, kJT, 0, st>>>(n, x, phi, M, (float)delta, packed, ns_pad, nchunks, out, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && S > 1) {
        int rgrid = (int)std::min<size_t>((len + 255) / 256, (size_t)8 * device_sm_count());
        k_jphi_sum<<<rgrid, 256, 0, st>>>(len, S, part, out);
        e = cudaGetLastError();
        count_launch();
    }
    timing_end(slot, st);
    PTROM_TRY(sc.release());
    if (e != cudaSuccess) return check_cuda(e, "k_jphi launch");
    count_launch();
    return PTROM_OK;
}

}  // namespace ptrom

using namespace ptrom;

extern "C" int bs_jphi(int n, const double *x, const double *Gamma, double delta, const double *phi, int M,
                       double *out, int prec, ptrom_stream_t stream) {
    if (n < 2 || M < 1) return set_error(PTROM_EINVAL, "bs_jphi: need n >= 2 and M >= 1 (n=%d M=%d)", n, M);
    if (!(delta >= 0.0)) return set_error(PTROM_EINVAL, "bs_jphi: delta must be >= 0");
    if (prec != PTROM_FP32C && prec != PTROM_FP64 && prec != PTROM_TF32X3 && prec != PTROM_F16X3)
        return set_error(PTROM_EINVAL, "bs_jphi: bad prec %d", prec);
    if (!x || !Gamma || !phi || !out) return set_error(PTROM_EINVAL, "bs_jphi: NULL array");
    return jphi(n, x, Gamma, delta, phi, M, out, prec, (cudaStream_t)stream, g_source_split.load());
}

// Online PTROM: Gauss-Newton (Alg. 4) over the hyper-reduced pairwise
// interaction (Alg. 5) -- ptrom_model_create / ptrom_set_param / ptrom_step.
//
// One CTA (512 threads) per parameter instance runs whole time steps with all
// per-iteration data resident in shared memory:
//   1. cluster gather         x^QT = x0_c + Phi_c xhat (FP32)
//   2. HyperPair + residual   warp per sampled body: x~_i = x0_s + Phi_s xhat,
//                             its CSR cluster list -> f~_i and the 2x2 block D~_i
//                             (inexact Jacobian, Sec. 2), and
//                             r_i = Phi_s,i (xhat - xhat^{n-1}) - dt/2 (f~_i + f~^{n-1}_i)
//   4. A C and A r            C = J Phi_s, J = I - dt/2 blockdiag(D~), generated
//                             32 dofs at a time in shared memory, 4x4 register
//                             tiles per thread (FP32)
//   5. eps numerator          || (A C)^T (A r) || (gradient of the minimised
//                             objective; the printed Phi^T J^T r does not vanish
//                             at the minimiser when M_r > M)
//   6. least squares          Householder QR of [A C | A r] (FP32, or FP64 on
//                             request), back substitution, xhat += dxhat (FP64,
//                             alpha = 1)
// On GB300 every warp-wide FP64 instruction (conversions included) costs ~16
// SM cycles, so FP64 is confined to the reduced state and the optional QR.
// A batch of instances (one model or many, uneven sizes) is one launch; there
// are no inter-CTA waits.  Positions are kept relative to a per-model origin
// before FP32 rounding.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "scratch.h"
#include "internal.h"
#include "ptrom_model.h"

namespace ptrom {

struct DevStats {
    unsigned long long gn_iters, steps;
    int noconv, max_iters;
};

// ------------------------------------------------------------------ layout
struct SmemLayout {
    size_t xh, xp, dx, xhf, df, red, f, fp, r, D, xq, gq, Bf, Bd, Ct, Ats, phiS, At, idx, total;
};

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

// rows / idx: also reserve the staged Phi_s and A^T rows / the 16-bit cluster
// lists (nlist entries), constant for the whole launch and read every
// Gauss-Newton iteration.
// xqg: x^QT and Gamma~ stay in global memory (no shared-memory room for them).
__host__ __device__ inline SmemLayout smem_layout(int ns, int M, int Mr, int Nc, int Mp, int Mrp, int qr64,
                                                  int rows = 0, int idx = 0, int nlist = 0, int xqg = 0) {
    SmemLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += al16(bytes); return at; };
    L.xh = take(8 * (size_t)M);
    L.xp = take(8 * (size_t)M);
    L.dx = take(8 * (size_t)Mp);
    L.xhf = take(4 * (size_t)Mp);
    L.df = take(4 * (size_t)Mp);
    L.red = take(4 * 64);
    L.f = take(4 * 2 * (size_t)ns);
    L.fp = take(4 * 2 * (size_t)ns);
    L.r = take(4 * 2 * (size_t)ns);
    L.D = take(4 * 3 * (size_t)ns);
    L.xq = take(xqg ? 0 : 4 * 2 * (size_t)Nc);
    L.gq = take(xqg ? 0 : 4 * (size_t)Nc);
    // [A C | A r], column-major, ld = Mrp, column M = rhs: FP64 for the FP64
    // QR (assembled in place), else FP32
    L.Bf = take(qr64 ? 0 : 4 * (size_t)Mrp * (M + 1));
    L.Bd = take(qr64 ? 8 * (size_t)Mrp * (M + 1) : 0);
    L.Ct = take(4 * 2 * kTileB * (size_t)Mp);
    L.Ats = take(4 * 2 * kTileB * (size_t)Mrp);
    L.phiS = take(rows ? 4 * 2 * (size_t)ns * Mp : 0);
    L.At = take(rows ? 4 * 2 * (size_t)ns * Mrp : 0);
    L.idx = take(idx ? 2 * (size_t)nlist : 0);
    L.total = o;
    return L;
}

__device__ __forceinline__ float warp_allsum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP32 sum (all threads get the result).
__device__ float block_allsum(float v, float *red) {
    v = warp_allsum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kPT / 32; ++w) s += red[w];
    return s;
}

// ------------------------------------------------------------------ pieces
// Phase A: xhat and its increment in FP32, then x^QT = x0_c + Phi_c xhat.
__device__ void gather_clusters(const DevModel &m, const double *xh, const double *xp, float *xhf, float *df,
                                float *xq) {
    for (int k = threadIdx.x; k < m.Mp; k += kPT) {
        xhf[k] = k < m.M ? (float)xh[k] : 0.f;
        df[k] = k < m.M ? (float)(xh[k] - xp[k]) : 0.f;
    }
    __syncthreads();
    // two rows per thread per round, so twice the L2 loads are in flight
    const int rows = 2 * m.Nc;
    for (int row = threadIdx.x; row < rows; row += 2 * kPT) {
        const int row2 = row + kPT;
        const bool two = row2 < rows;
        const float *ph = m.phiT + (size_t)row * m.Mp, *ph2 = m.phiT + (size_t)(two ? row2 : row) * m.Mp;
        float acc = m.x0T[row], acc2 = two ? m.x0T[row2] : 0.f;
#pragma unroll 4
        for (int k = 0; k < m.Mp; k += 4) {
            const float4 p = __ldg(reinterpret_cast<const float4 *>(ph + k));
            const float4 p2 = __ldg(reinterpret_cast<const float4 *>(ph2 + k));
            acc = fmaf(p.x, xhf[k], acc);
            acc = fmaf(p.y, xhf[k + 1], acc);
            acc = fmaf(p.z, xhf[k + 2], acc);
            acc = fmaf(p.w, xhf[k + 3], acc);
            acc2 = fmaf(p2.x, xhf[k], acc2);
            acc2 = fmaf(p2.y, xhf[k + 1], acc2);
            acc2 = fmaf(p2.z, xhf[k + 2], acc2);
            acc2 = fmaf(p2.w, xhf[k + 3], acc2);
        }
        xq[row] = acc;
        if (two) xq[row2] = acc2;
    }
    __syncthreads();
}

// dot of a Phi_s row with a shared-memory vector, lanes over the modes.
__device__ __forceinline__ float row_dot(const float *row, const float *vec, int Mp, int lane) {
    float s = 0.f;
    for (int k = lane; k < Mp; k += 32) s = fmaf(row[k], vec[k], s);
    return warp_allsum(s);
}

// Phase B, warp per sampled body i: x~_i, the HyperPair sums f~_i and D~_i
// over its clusters, and the residual r_i = Phi_s,i dxhat - h (f~_i + f~^{n-1}_i)
// - dt u_i (u: the superimposed inflow of Sec. 6.3, stored as dt u).
// phiB: the Phi_s rows (shared or global memory); idx16: the cluster lists in
// shared memory as 16-bit indices, or nullptr to read m.idx.
__device__ void hyperpair_residual(const DevModel &m, const float *phiB, const unsigned short *idx16,
                                   const float *xhf, const float *df, const float *xq, const float *gq,
                                   const float *fp, float *f, float *D, float *r) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float dd = (float)m.delta, h = (float)(0.5 * m.dt);
    for (int i = warp; i < m.ns; i += kPT / 32) {
        const float *rc = phiB + (size_t)i * m.Mp, *rp = phiB + (size_t)(m.ns + i) * m.Mp;
        const float tx = m.x0B[i] + row_dot(rc, xhf, m.Mp, lane);
        const float ty = m.x0B[m.ns + i] + row_dot(rp, xhf, m.Mp, lane);
        const float gx = row_dot(rc, df, m.Mp, lane), gy = row_dot(rp, df, m.Mp, lane);
        float u = 0.f, v = 0.f, d00 = 0.f, d01 = 0.f, d10n = 0.f;
        const int e_end = m.off[i + 1];
#pragma unroll 4
        for (int e = m.off[i] + lane; e < e_end; e += 32) {
            const int c = idx16 ? (int)idx16[e] : __ldg(m.idx + e);
            const float a = tx - xq[c], b = ty - xq[m.Nc + c];
            const float d2 = fmaf(a, a, b * b);
            float rr = rcp_approx(d2 + dd);  // MUFU reciprocal, ~1 ulp (as in the all-pairs kernels)
            rr = (d2 == 0.f) ? 0.f : rr;
            const float q = gq[c] * rr;
            u = fmaf(q, b, u);
            v = fmaf(q, a, v);
            const float p2 = 2.f * q * rr;
            d00 = fmaf(p2 * a, b, d00);
            d01 += fmaf(p2 * b, b, -q);
            d10n += fmaf(p2 * a, a, -q);
        }
        u = warp_allsum(u);
        v = warp_allsum(v);
        d00 = warp_allsum(d00);
        d01 = warp_allsum(d01);
        d10n = warp_allsum(d10n);
        if (lane == 0) {
            const float fx = -u, fy = v;
            f[i] = fx;
            f[m.ns + i] = fy;
            D[i] = d00;
            D[m.ns + i] = d01;
            D[2 * m.ns + i] = -d10n;
            r[i] = gx - h * (fx + fp[i]) - m.uB[i];
            r[m.ns + i] = gy - h * (fy + fp[m.ns + i]) - m.uB[m.ns + i];
        }
    }
    __syncthreads();
}

// Phase C: B[:, 0..M-1] = A C (C = J Phi_s), B[:, M] = A r; B column-major
// (ld Mrp), FP32 products, each tile's sums added to B in TB (FP32 or FP64).  Each tile of 16 bodies (32 dofs) stages its rows of A^T
// and of C in shared memory with one cooperative round of loads; threads own
// 4x4 blocks of B (several each for large M, M_r) and add each tile's
// contribution to them in shared memory.
template <typename TB>
__device__ void assemble_lsq(const DevModel &m, const float *phiB, const float *At, const float *D, const float *r,
                             float *Ct, float *Ats, TB *B) {
    const float h = (float)(0.5 * m.dt);
    const int tilesM = m.Mp / 4, tilesR = m.Mrp / 4, nblk = tilesM * tilesR;
    for (int e = threadIdx.x; e < m.Mrp * (m.M + 1); e += kPT) B[e] = TB(0);
    for (int i0 = 0; i0 < m.ns; i0 += kTileB) {
        const int nbt = min(kTileB, m.ns - i0);
        // stage the tile's A^T rows (slot 2j = chi dof of body i0+j, 2j+1 = psi dof)
        for (int e = threadIdx.x; e < 2 * kTileB * (m.Mrp / 4); e += kPT) {
            const int slot = e / (m.Mrp / 4), c4 = e % (m.Mrp / 4), j = slot >> 1;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < nbt) {
                const int dof = (slot & 1) ? m.ns + i0 + j : i0 + j;
                v = reinterpret_cast<const float4 *>(At + (size_t)dof * m.Mrp)[c4];
            }
            reinterpret_cast<float4 *>(Ats + (size_t)slot * m.Mrp)[c4] = v;
        }
        // the tile's C rows
        for (int e = threadIdx.x; e < 2 * kTileB * m.Mp; e += kPT) {
            const int slot = e / m.Mp, k = e % m.Mp, j = slot >> 1;
            float val = 0.f;
            if (j < nbt) {
                const int i = i0 + j;
                const float pc = phiB[(size_t)i * m.Mp + k], pp = phiB[(size_t)(m.ns + i) * m.Mp + k];
                const float d00 = D[i], d01 = D[m.ns + i], d10 = D[2 * m.ns + i];
                val = (slot & 1) ? pp - h * (d10 * pc - d00 * pp) : pc - h * (d00 * pc + d01 * pp);
            }
            Ct[slot * m.Mp + k] = val;
        }
        __syncthreads();
        for (int blk = threadIdx.x; blk < nblk; blk += kPT) {
            const int r0 = 4 * (blk / tilesM), m0 = 4 * (blk % tilesM);
            float acc[4][4] = {};
            float bacc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int j = 0; j < nbt; ++j) {
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int dof = half ? m.ns + i0 + j : i0 + j;
                    const float4 a = *reinterpret_cast<const float4 *>(Ats + (size_t)(2 * j + half) * m.Mrp + r0);
                    const float4 c = *reinterpret_cast<const float4 *>(Ct + (2 * j + half) * m.Mp + m0);
                    const float av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], cv[y], acc[x][y]);
                    if (m0 == 0) {
                        const float rv = r[dof];
#pragma unroll
                        for (int x = 0; x < 4; ++x) bacc[x] = fmaf(av[x], rv, bacc[x]);
                    }
                }
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                if (r0 + x >= m.Mr) continue;
#pragma unroll
                for (int y = 0; y < 4; ++y)
                    if (m0 + y < m.M) B[(size_t)(m0 + y) * m.Mrp + r0 + x] += (TB)acc[x][y];
                if (m0 == 0) B[(size_t)m.M * m.Mrp + r0 + x] += (TB)bacc[x];
            }
        }
        __syncthreads();
    }
}

// eps numerator: || (A C)^T (A r) || from B = [A C | A r] (before the QR).
template <typename TB>
__device__ float lsq_gradient(const DevModel &m, const TB *B, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TB *b = B + (size_t)m.M * m.Mrp;
    float g2 = 0.f;
    for (int k = warp; k < m.M; k += kPT / 32) {
        float s = 0.f;
        for (int i = lane; i < m.Mr; i += 32) s = fmaf((float)B[(size_t)k * m.Mrp + i], (float)b[i], s);
        s = warp_allsum(s);
        if (lane == 0) g2 += s * s;
    }
    return sqrtf(block_allsum(g2, red));
}

// Householder QR of B (Mr x M, column-major, rhs in column M) in T arithmetic,
// then dx = -R^{-1} (Q^T b)[0..M-1].  One CTA barrier per column: warps
// update the later columns in parallel (in FP64 four per warp: warp w takes
// j+1+4w .. j+4+4w, then the next 64; in FP32 one: j+1+w, then the next 16),
// and the warp that owns column j+1 (warp 0) derives that column's reflector
// as soon as its own update of it is done, before the barrier.  The reflector's
// square root and division thus run once per column, not in every warp: in
// FP64 a warp-wide instruction holds a sub-partition's FP64 unit for ~64
// cycles whatever its active lanes, so sixteen redundant copies would cost
// more than the rest of the column.
template <typename T>
__device__ __forceinline__ T warp_allsum_t(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sqrt and reciprocal: exact in FP64; MUFU (~1 ulp) in FP32, since the FP32
// solve's IEEE sequences sit on a chain of 20 dependent steps per column loop
// and the Gauss-Newton fixed point is set by the residual, not by the solve
__device__ __forceinline__ double ls_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ double ls_rcp(double v) { return 1.0 / v; }
__device__ __forceinline__ float ls_sqrt(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }
__device__ __forceinline__ float ls_rcp(float v) { return rcp_approx(v); }

// Reflector of column j (called by one whole warp; the values are warp-
// uniform): v = (x0 - alpha, c_j[j+1..]), H = I - tau v v^T, with
// alpha = -sign(x0) |c_j[j..]|.  The squared norm comes from the downdated
// s_rem unless half of it is gone (each downdate errs by ~eps |c_j|^2 <=
// eps s_ref, so the value is good to ~40 eps while half remains), in which
// case it is summed again.  Writes alpha, v0 and tau to slot j & 1.
template <typename T>
__device__ __forceinline__ void reflector(const T *cj, int j, int Mr, int lane, const T *s_rem, const T *s_ref,
                                          T *s_alpha, T (*s_scal)[2]) {
    T s = s_rem[j];
    if (!(s >= (T)0.5 * s_ref[j])) {
        s = 0;
        for (int i = j + lane; i < Mr; i += 32) s += cj[i] * cj[i];
        s = warp_allsum_t(s);
    }
    const T x0 = cj[j];
    const T nrm = ls_sqrt(s);
    const T alpha = x0 >= 0 ? -nrm : nrm;
    const T v0 = x0 - alpha;
    const T vn2 = s - x0 * x0 + v0 * v0;
    const T tau = vn2 > 0 ? (T)2 * ls_rcp(vn2) : (T)0;
    if (lane == 0) {
        s_alpha[j] = alpha;
        s_scal[j & 1][0] = v0;
        s_scal[j & 1][1] = tau;
    }
}

template <typename T>
__device__ void lsq_solve(const DevModel &m, T *B, double *dx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Mr = m.Mr, M = m.M, ld = m.Mrp;
    __shared__ T s_alpha[kMaxM], s_y[kMaxM], s_rem[kMaxM], s_ref[kMaxM];
    __shared__ T s_scal[2][2];  // (v0, tau) of column j in slot j & 1
    const int ncols = min(M, Mr);
    // remaining squared norm of every column over the rows not yet reduced
    // (downdated after each reflection: |c_k[j..]|^2 = |c_k[j-1..]|^2 - R_{j-1,k}^2,
    // as in QR with column pivoting), so a column's reflector needs no reduction
    for (int k = warp; k < ncols; k += kPT / 32) {
        const T *ck = B + (size_t)k * ld;
        T s = 0;
        for (int i = lane; i < Mr; i += 32) s += ck[i] * ck[i];
        s = warp_allsum_t(s);
        if (lane == 0) s_rem[k] = s_ref[k] = s;
    }
    __syncthreads();
    if (warp == 0 && ncols > 0) reflector(B, 0, Mr, lane, s_rem, s_ref, s_alpha, s_scal);
    __syncthreads();
    // FP64: each warp updates kCols = 4 columns at once, kG = 8 lanes per
    // column, so a warp instruction carries four columns' work on the scarce
    // FP64 unit (and the dot products need three shuffle levels instead of
    // five).  FP32 is latency-bound instead: one column per warp, 32 lanes.
    constexpr int kG = sizeof(T) == 8 ? 8 : 32, kCols = 32 / kG;
    const int sub = lane / kG, gl = lane % kG;
    for (int j = 0; j < ncols; ++j) {
        const T *cj = B + (size_t)j * ld;
        const T v0 = s_scal[j & 1][0], tau = s_scal[j & 1][1];
        for (int kb = j + 1 + warp * kCols; kb <= M; kb += (kPT / 32) * kCols) {
            const int k = kb + sub;
            const bool act = k <= M;  // uniform within each group of kG lanes
            T *ck = B + (size_t)k * ld;
            T w = 0;
            if (act)
                for (int i = j + gl; i < Mr; i += kG) w += (i == j ? v0 : cj[i]) * ck[i];
            for (int o = kG / 2; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            w *= tau;
            if (act)
                for (int i = j + gl; i < Mr; i += kG) {
                    const T c = ck[i] - w * (i == j ? v0 : cj[i]);
                    ck[i] = c;
                    if (i == j && k < ncols) s_rem[k] -= c * c;  // row j of column k is now R_jk
                }
            if (kb == j + 1 && kb < ncols) {  // warp 0: column j+1 is final for step j+1
                __syncwarp();
                reflector(B + (size_t)kb * ld, kb, Mr, lane, s_rem, s_ref, s_alpha, s_scal);
            }
        }
        __syncthreads();  // the updated columns and the next reflector are read by every warp next
    }
    // 1 / R_jj for every column at once (s_rem is free now), off the
    // back substitution's dependent chain
    for (int j = threadIdx.x; j < ncols; j += kPT) s_rem[j] = s_alpha[j] != 0 ? ls_rcp(s_alpha[j]) : (T)0;
    __syncthreads();
    // back substitution R y = -c (warp 0, in T), column by column: lane l
    // holds the right-hand sides of rows l, l + 32, ...; each step broadcasts
    // y_j from its row's lane and updates the rows above it (R_ij is column
    // j's row i), one shuffle and one multiply-add per step; the row blocks
    // entirely below j are skipped (warp-uniform), since even lanes switched
    // off by a predicate occupy the FP64 unit
    if (warp == 0) {
        const T *rhs = B + (size_t)M * ld;
        constexpr int kQ = kMaxM / 32;  // rows per lane
        T c[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) c[q] = lane + 32 * q < ncols ? -rhs[lane + 32 * q] : (T)0;
        for (int j = ncols - 1; j >= 0; --j) {
            T own = c[0];
#pragma unroll
            for (int q = 1; q < kQ; ++q) own = (j >> 5) == q ? c[q] : own;
            const T cj = __shfl_sync(0xffffffffu, own, j & 31);
            const T yj = cj * s_rem[j];
            if (lane == (j & 31)) s_y[j] = yj;
            const T *cjc = B + (size_t)j * ld;
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                if (32 * q < j && lane + 32 * q < j) c[q] -= cjc[lane + 32 * q] * yj;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += kPT) dx[j] = j < ncols ? (double)s_y[j] : 0.0;
    __syncthreads();
}

__global__ void __launch_bounds__(kPT, 1)
k_ptrom(const InstArgs *__restrict__ insts, int nsteps, DevStats *stats) {
    extern __shared__ __align__(16) unsigned char sm[];
    const InstArgs &I = insts[blockIdx.x];
    const DevModel m = I.m;
    const SmemLayout L =
        smem_layout(m.ns, m.M, m.Mr, m.Nc, m.Mp, m.Mrp, m.qr64, m.cache_rows, m.cache_idx, m.nlist, m.xq_global);
    double *xh = (double *)(sm + L.xh), *xp = (double *)(sm + L.xp), *dx = (double *)(sm + L.dx);
    float *xhf = (float *)(sm + L.xhf), *df = (float *)(sm + L.df), *red = (float *)(sm + L.red);
    float *f = (float *)(sm + L.f), *fp = (float *)(sm + L.fp), *r = (float *)(sm + L.r), *D = (float *)(sm + L.D);
    // x^QT in shared memory, or (large N_c) in this instance's state buffer; Gamma~ staged, or read in place
    float *xq = m.xq_global ? (float *)((char *)I.state + state_base_bytes(m.M, m.ns)) : (float *)(sm + L.xq);
    float *gqs = (float *)(sm + L.gq), *Bf = (float *)(sm + L.Bf);
    const float *gq = m.xq_global ? m.gT : gqs;
    double *Bd = (double *)(sm + L.Bd);
    float *Ct = (float *)(sm + L.Ct), *Ats = (float *)(sm + L.Ats);

    double *st_x = I.state, *st_f = I.state + m.M, *st_flag = I.state + m.M + 2 * m.ns;
    for (int k = threadIdx.x; k < m.M; k += kPT) {
        xh[k] = st_x[k];
        xp[k] = st_x[k];
    }
    if (!m.xq_global)
        for (int c = threadIdx.x; c < m.Nc; c += kPT) gqs[c] = m.gT[c];
    // constant model rows and lists, read every Gauss-Newton iteration: staged once
    const float *phiB = m.phiB, *At = m.At;
    const unsigned short *idx16 = nullptr;
    if (m.cache_rows) {
        float *ps = (float *)(sm + L.phiS), *as = (float *)(sm + L.At);
        for (int e = threadIdx.x; e < 2 * m.ns * m.Mp; e += kPT) ps[e] = m.phiB[e];
        for (int e = threadIdx.x; e < 2 * m.ns * m.Mrp; e += kPT) as[e] = m.At[e];
        phiB = ps;
        At = as;
    }
    if (m.cache_idx) {
        unsigned short *is = (unsigned short *)(sm + L.idx);
        for (int e = threadIdx.x; e < m.nlist; e += kPT) is[e] = (unsigned short)m.idx[e];
        idx16 = is;
    }
    const bool have_f = st_flag[0] != 0.0;
    for (int d = threadIdx.x; d < 2 * m.ns; d += kPT) fp[d] = have_f ? (float)st_f[d] : 0.f;
    __syncthreads();
    if (!have_f) {  // f~ at the initial coordinates (R11)
        gather_clusters(m, xh, xp, xhf, df, xq);
        hyperpair_residual(m, phiB, idx16, xhf, df, xq, gq, fp, f, D, r);
        for (int d = threadIdx.x; d < 2 * m.ns; d += kPT) fp[d] = f[d];
        __syncthreads();
    }
    int local_iters = 0, local_noconv = 0, local_max = 0;
    for (int step = 0; step < nsteps; ++step) {
        for (int k = threadIdx.x; k < m.M; k += kPT) xp[k] = xh[k];
        __syncthreads();
        float first = -1.f;
        int kk = 0;
        while (true) {
            gather_clusters(m, xh, xp, xhf, df, xq);
            hyperpair_residual(m, phiB, idx16, xhf, df, xq, gq, fp, f, D, r);
            float g;
            if (m.qr64) {
                assemble_lsq(m, phiB, At, D, r, Ct, Ats, Bd);
                g = lsq_gradient(m, Bd, red);
                lsq_solve<double>(m, Bd, dx);
            } else {
                assemble_lsq(m, phiB, At, D, r, Ct, Ats, Bf);
                g = lsq_gradient(m, Bf, red);
                lsq_solve<float>(m, Bf, dx);
            }
            for (int k = threadIdx.x; k < m.M; k += kPT) xh[k] += dx[k];
            __syncthreads();
            if (first < 0.f) first = g;
            ++kk;
            const float eps = first > 0.f ? g / first : 0.f;
            const bool conv = kk > 1 && eps <= (float)m.tol;
            if (conv || first == 0.f || kk >= m.max_gn || !isfinite(g)) {
                if (!conv && first != 0.f) ++local_noconv;
                break;
            }
        }
        local_iters += kk;
        local_max = max(local_max, kk);
        for (int d = threadIdx.x; d < 2 * m.ns; d += kPT) fp[d] = f[d];  // R11: last HyperPair velocity
        if (I.hist)
            for (int k = threadIdx.x; k < m.M; k += kPT) I.hist[(size_t)step * m.M + k] = xh[k];
        __syncthreads();
    }
    for (int k = threadIdx.x; k < m.M; k += kPT) {
        st_x[k] = xh[k];
        if (I.xhat) I.xhat[k] = xh[k];
    }
    for (int d = threadIdx.x; d < 2 * m.ns; d += kPT) st_f[d] = (double)fp[d];
    if (threadIdx.x == 0) {
        st_flag[0] = 1.0;
        if (stats) {
            atomicAdd(&stats->gn_iters, (unsigned long long)local_iters);
            atomicAdd(&stats->steps, (unsigned long long)nsteps);
            atomicAdd(&stats->noconv, local_noconv);
            atomicMax(&stats->max_iters, local_max);
        }
    }
}

}  // namespace ptrom

// ------------------------------------------------------------------ host side
using namespace ptrom;

static int upload(ptrom_model *m, const void *host, size_t bytes, void **out) {
    void *p = nullptr;
    PTROM_CUDA(cudaMalloc(&p, bytes ? bytes : 16));
    m->bufs.push_back(p);
    if (bytes && host) PTROM_CUDA(cudaMemcpy(p, host, bytes, cudaMemcpyHostToDevice));
    *out = p;
    return PTROM_OK;
}

// Row-major FP64 [rows][cols] -> FP32 [rows][ld], zero padded.
static std::vector<float> to_f32_rows(const double *a, int rows, int cols, int ld) {
    std::vector<float> o((size_t)rows * ld, 0.f);
    for (int i = 0; i < rows; ++i)
        for (int k = 0; k < cols; ++k) o[(size_t)i * ld + k] = (float)a[(size_t)i * cols + k];
    return o;
}

int ptrom::model_fill_param(ptrom_model *m, const double *x0_s, const double *phi_c, const double *x0_c,
                      const double *gamma_c) {
    DevModel &d = m->d;
    if (x0_s) m->h_x0_s.assign(x0_s, x0_s + 2 * (size_t)d.ns);
    if (phi_c) m->h_phi_c.assign(phi_c, phi_c + 2 * (size_t)d.Nc * d.M);
    if (x0_c) m->h_x0_c.assign(x0_c, x0_c + 2 * (size_t)d.Nc);
    if (gamma_c) m->h_gamma_c.assign(gamma_c, gamma_c + (size_t)d.Nc);
    if (x0_s) {
        std::vector<float> v(2 * (size_t)d.ns);
        for (int i = 0; i < d.ns; ++i) {
            v[i] = (float)(x0_s[i] - m->ox);
            v[d.ns + i] = (float)(x0_s[d.ns + i] - m->oy);
        }
        PTROM_CUDA(cudaMemcpy((void *)d.x0B, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    }
    if (phi_c) {
        std::vector<float> v = to_f32_rows(phi_c, 2 * d.Nc, d.M, d.Mp);
        PTROM_CUDA(cudaMemcpy((void *)d.phiT, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    }
    if (x0_c) {
        std::vector<float> v(2 * (size_t)d.Nc);
        for (int c = 0; c < d.Nc; ++c) {
            v[c] = (float)(x0_c[c] - m->ox);
            v[d.Nc + c] = (float)(x0_c[d.Nc + c] - m->oy);
        }
        PTROM_CUDA(cudaMemcpy((void *)d.x0T, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    }
    if (gamma_c) {
        std::vector<float> v(d.Nc);
        for (int c = 0; c < d.Nc; ++c) v[c] = (float)(gamma_c[c] * kInv2Pi);
        PTROM_CUDA(cudaMemcpy((void *)d.gT, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    }
    return PTROM_OK;
}

int ptrom::model_fill_inflow(ptrom_model *m, const double *u_s) {
    const DevModel &d = m->d;
    std::vector<float> v(2 * (size_t)d.ns, 0.f);
    if (u_s) {
        m->h_u_s.assign(u_s, u_s + 2 * (size_t)d.ns);
        for (int e = 0; e < 2 * d.ns; ++e) v[e] = (float)(d.dt * u_s[e]);
    } else {
        m->h_u_s.clear();
    }
    PTROM_CUDA(cudaMemcpy((void *)d.uB, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
    return PTROM_OK;
}

extern "C" int ptrom_model_create(const ptrom_model_desc *desc, ptrom_model **out) {
    if (!desc || !out) return set_error(PTROM_EINVAL, "ptrom_model_create: NULL argument");
    const ptrom_model_desc &s = *desc;
    if (s.n_s < 1 || s.n_s > kMaxNs || s.M < 1 || s.M > kMaxM || s.M_r < 1 || s.M_r > kMaxMr || s.N_c < 1 ||
        s.N_c > kMaxNc)
        return set_error(PTROM_EINVAL, "ptrom_model_create: sizes out of range (n_s=%d M=%d M_r=%d N_c=%d)", s.n_s,
                         s.M, s.M_r, s.N_c);
    if (!(s.dt > 0) || !(s.delta >= 0) || !(s.tol >= 0) || s.max_gn < 1 ||
        (s.qr_prec != PTROM_FP64 && s.qr_prec != PTROM_FP32C))
        return set_error(PTROM_EINVAL, "ptrom_model_create: bad dt/delta/tol/max_gn/qr_prec");
    if (!s.phi_s || !s.x0_s || !s.phi_c || !s.x0_c || !s.gamma_c || !s.A || !s.off || !s.idx)
        return set_error(PTROM_EINVAL, "ptrom_model_create: NULL array");
    if (s.off[0] != 0) return set_error(PTROM_EINVAL, "ptrom_model_create: off[0] must be 0");
    for (int i = 0; i < s.n_s; ++i)
        if (s.off[i + 1] < s.off[i]) return set_error(PTROM_EINVAL, "ptrom_model_create: off not monotone");
    const int L = s.off[s.n_s];
    for (int e = 0; e < L; ++e)
        if (s.idx[e] < 0 || s.idx[e] >= s.N_c)
            return set_error(PTROM_EINVAL, "ptrom_model_create: idx[%d]=%d out of [0,%d)", e, s.idx[e], s.N_c);
    ptrom_model *m = new ptrom_model();
    PTROM_CUDA(cudaGetDevice(&m->device));
    DevModel &d = m->d;
    d.ns = s.n_s;
    d.M = s.M;
    d.Mr = s.M_r;
    d.Nc = s.N_c;
    d.Mp = (s.M + 3) & ~3;
    d.Mrp = (s.M_r + 3) & ~3;
    d.dt = s.dt;
    d.delta = s.delta;
    d.tol = s.tol;
    d.max_gn = s.max_gn;
    d.qr64 = s.qr_prec == PTROM_FP64;
    m->qr_prec = s.qr_prec;
    m->h_phi_s.assign(s.phi_s, s.phi_s + 2 * (size_t)s.n_s * s.M);
    m->h_A.assign(s.A, s.A + (size_t)s.M_r * 2 * s.n_s);
    m->h_off.assign(s.off, s.off + s.n_s + 1);
    m->h_idx.assign(s.idx, s.idx + L);
    m->ox = s.x0_s[0];
    m->oy = s.x0_s[s.n_s];
    d.nlist = L;
    constexpr size_t kSmemCap = 220 * 1024;
    // x^QT and Gamma~ in shared memory when they fit, else in global memory
    d.xq_global = smem_layout(d.ns, d.M, d.Mr, d.Nc, d.Mp, d.Mrp, d.qr64).total > kSmemCap ? 1 : 0;
    const int xg = d.xq_global;
    const SmemLayout lay = smem_layout(d.ns, d.M, d.Mr, d.Nc, d.Mp, d.Mrp, d.qr64, 0, 0, 0, xg);
    m->smem = lay.total;
    // stage constant rows / lists in shared memory when they fit
    if (smem_layout(d.ns, d.M, d.Mr, d.Nc, d.Mp, d.Mrp, d.qr64, 1, 0, L, xg).total <= kSmemCap) {
        d.cache_rows = 1;
        m->smem = smem_layout(d.ns, d.M, d.Mr, d.Nc, d.Mp, d.Mrp, d.qr64, 1, 0, L, xg).total;
    }
    if (d.Nc <= 65535 &&
        smem_layout(d.ns, d.M, d.Mr, d.Nc, d.Mp, d.Mrp, d.qr64, d.cache_rows, 1, L, xg).total <= kSmemCap) {
        d.cache_idx = 1;
        m->smem = smem_layout(d.ns, d.M, d.Mr, d.Nc, d.Mp, d.Mrp, d.qr64, d.cache_rows, 1, L, xg).total;
    }
    if (m->smem > kSmemCap) {
        delete m;
        return set_error(PTROM_EINVAL, "ptrom_model_create: model needs %zu bytes of shared memory", lay.total);
    }
    int st = PTROM_OK;
    void *p;
    auto fail = [&](int code) {
        ptrom_free(m);
        return code;
    };
    {
        std::vector<float> v = to_f32_rows(s.phi_s, 2 * d.ns, d.M, d.Mp);
        if ((st = upload(m, v.data(), v.size() * 4, &p))) return fail(st);
        d.phiB = (const float *)p;
    }
    if ((st = upload(m, nullptr, 2 * (size_t)d.ns * 4, &p))) return fail(st);
    d.x0B = (const float *)p;
    if ((st = upload(m, nullptr, 2 * (size_t)d.Nc * d.Mp * 4, &p))) return fail(st);
    d.phiT = (const float *)p;
    if ((st = upload(m, nullptr, 2 * (size_t)d.Nc * 4, &p))) return fail(st);
    d.x0T = (const float *)p;
    if ((st = upload(m, nullptr, (size_t)d.Nc * 4, &p))) return fail(st);
    d.gT = (const float *)p;
    if ((st = upload(m, nullptr, 2 * (size_t)d.ns * 4, &p))) return fail(st);
    d.uB = (const float *)p;
    if ((st = upload(m, s.off, (size_t)(d.ns + 1) * 4, &p))) return fail(st);
    d.off = (const int *)p;
    if ((st = upload(m, s.idx, (size_t)L * 4, &p))) return fail(st);
    d.idx = (const int *)p;
    {
        std::vector<float> At((size_t)2 * d.ns * d.Mrp, 0.f);
        for (int r = 0; r < d.Mr; ++r)
            for (int dof = 0; dof < 2 * d.ns; ++dof) At[(size_t)dof * d.Mrp + r] = (float)s.A[(size_t)r * 2 * d.ns + dof];
        if ((st = upload(m, At.data(), At.size() * 4, &p))) return fail(st);
        d.At = (const float *)p;
    }
    if ((st = model_fill_param(m, s.x0_s, s.phi_c, s.x0_c, s.gamma_c))) return fail(st);
    if ((st = model_fill_inflow(m, s.u_s))) return fail(st);
    *out = m;
    return PTROM_OK;
}

extern "C" void ptrom_free(ptrom_model *m) {
    if (!m) return;
    for (void *p : m->bufs) cudaFree(p);
    delete m;
}

extern "C" int ptrom_set_param(ptrom_model *m, const double *x0_s, const double *phi_c, const double *x0_c,
                               const double *gamma_c) {
    if (!m) return set_error(PTROM_EINVAL, "ptrom_set_param: NULL model");
    return model_fill_param(m, x0_s, phi_c, x0_c, gamma_c);
}

extern "C" int ptrom_set_inflow(ptrom_model *m, const double *u_s) {
    if (!m) return set_error(PTROM_EINVAL, "ptrom_set_inflow: NULL model");
    return model_fill_inflow(m, u_s);
}

extern "C" size_t ptrom_state_bytes(const ptrom_model *m) {
    if (!m) return 0;
    const size_t base = state_base_bytes(m->d.M, m->d.ns);
    return m->d.xq_global ? base + ((sizeof(float) * 2 * (size_t)m->d.Nc + 255) & ~size_t(255)) : base;
}

extern "C" int ptrom_step(ptrom_model *const *models, int batch, void *const *state, double *const *xhat,
                          double *const *hist, int nsteps, ptrom_stats *stats, ptrom_stream_t stream) {
    if (!models || !state || batch < 1 || nsteps < 0)
        return set_error(PTROM_EINVAL, "ptrom_step: bad arguments (batch=%d nsteps=%d)", batch, nsteps);
    if (nsteps == 0) return PTROM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<InstArgs> host(batch);
    size_t smem = 0;
    for (int b = 0; b < batch; ++b) {
        if (!models[b] || !state[b]) return set_error(PTROM_EINVAL, "ptrom_step: NULL model/state at %d", b);
        if (((uintptr_t)state[b]) & 255) return set_error(PTROM_EINVAL, "ptrom_step: state %d not 256-byte aligned", b);
        host[b].m = models[b]->d;
        host[b].state = (double *)state[b];
        host[b].xhat = xhat ? xhat[b] : nullptr;
        host[b].hist = hist ? hist[b] : nullptr;
        smem = std::max(smem, models[b]->smem);
    }
    void *dev = nullptr;
    const size_t bytes = sizeof(InstArgs) * batch + sizeof(DevStats);
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&dev, bytes));
    InstArgs *dinst = (InstArgs *)dev;
    DevStats *dstats = (DevStats *)((char *)dev + sizeof(InstArgs) * batch);
    PTROM_CUDA(cudaMemcpyAsync(dinst, host.data(), sizeof(InstArgs) * batch, cudaMemcpyHostToDevice, st));
    PTROM_CUDA(cudaMemsetAsync(dstats, 0, sizeof(DevStats), st));
    PTROM_CUDA(cudaFuncSetAttribute(k_ptrom, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int slot = timing_begin(PTROM_K_PTROM_STEP, st);
    k_ptrom<<<batch, kPT, smem, st>>>(dinst, nsteps, dstats);
    timing_end(slot, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return check_cuda(e, "k_ptrom launch");
    count_launch();
    if (stats) {
        DevStats hs{};
        PTROM_CUDA(cudaMemcpyAsync(&hs, dstats, sizeof hs, cudaMemcpyDeviceToHost, st));
        PTROM_CUDA(cudaStreamSynchronize(st));
        stats->gn_iters = (long long)hs.gn_iters;
        stats->steps = (long long)hs.steps;
        stats->noconv = hs.noconv;
        stats->max_iters = hs.max_iters;
    }
    return sc.release();
}

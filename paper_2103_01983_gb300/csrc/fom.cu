// Full-order model: one implicit trapezoid step solved by Newton (Sec. 2,
// Eq. linKstep) -- the C-ABI entry fom_step and its device kernels.
//
// Host-driven Newton loop; every heavy product (velocity, self blocks, J v)
// runs in the all-pairs kernels of bs_pair.cu, every vector operation and
// reduction in the kernels below (FP64 state, deterministic fixed-order
// reductions: per-block partials, the last block to finish sums them in
// block order).  Linear solves:
//   block-diagonal : per-body 2x2 solve with (I - dt/2 D_i)
//   JFNK           : restarted right-preconditioned GMRES with classical
//                    Gram-Schmidt applied twice (CGS2) on the device; the
//                    (m+1) x m Hessenberg least-squares (Givens) on the host.
//                    One Arnoldi step is three launches and one host read:
//                    normalise + precondition, the J v pair kernel with the
//                    (I - dt/2 J) epilogue, and CGS2 as one cooperative
//                    kernel (three grid barriers); the correction
//                    d = M^{-1} V y is one more launch per cycle.
//   dense          : FP64 assembly of I - dt/2 J, LU with partial pivoting in
//                    one cooperative kernel (one grid barrier per column),
//                    forward/back substitution in one CTA.
#include <cooperative_groups.h>

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "scratch.h"
#include "internal.h"

namespace ptrom {
namespace cg = cooperative_groups;

constexpr int kRedThreads = 256;
constexpr int kMaxRestart = 64;
constexpr int kMaxDots = kMaxRestart + 2;
constexpr int kDenseMaxN = 4096;

// ---------------------------------------------------------------- reductions
struct Red {
    double *partials;        // [gridDim.x][nk]
    unsigned int *counter;   // zero between launches (reset by the last block)
    double *out;             // [nk]
};

// Sum `v` over the block; thread 0 returns the total.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    return s;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// After every block has written its nk partials: the last block sums them
// into red.out (warp w takes k = w, w + nwarps, ...; lanes stride the blocks;
// fixed order, so the result is deterministic) and resets the counter.
// Returns true in the last block, after a barrier (red.out readable by all
// of its threads).
__device__ __forceinline__ bool finish_reduction(const Red &red, int nk) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(red.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < nk; k += nw) {
        double s = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s += red.partials[(size_t)b * nk + k];
        s = warp_sum(s);
        if (lane == 0) red.out[k] = s;
    }
    if (threadIdx.x == 0) *red.counter = 0u;
    __syncthreads();
    return true;
}

// r = xi - xprev - hdt (fxi + fprev) [- dt u];   out = {||r||^2, ||xi||^2}.
// u: the optional superimposed inflow (Sec. 6.3), constant per dof; the
// trapezoid rule averages it with itself, so it enters as dt u = 2 hdt u.
// The last block also takes the Newton decision (converged when
// ||r|| <= tol max(1, ||xi||)): st = {stop, ||r||, ||xi||} with stop 0 = go on,
// 1 = converged, 2 = non-finite residual, 3 = iteration limit (limit set);
// flags[0] = (stop != 0) lets queued Newton-update kernels skip themselves.
__global__ void k_residual(int n2, const double *xi, const double *xprev, const double *fxi,
                           const double *fprev, const double *u, double hdt, double *r, Red red, double tol,
                           int limit, int *flags, double *st) {
    __shared__ double sh[32];
    double s0 = 0.0, s1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
        double v = xi[i] - xprev[i] - hdt * (fxi[i] + fprev[i]);
        if (u) v -= (2.0 * hdt) * u[i];
        r[i] = v;
        s0 += v * v;
        s1 += xi[i] * xi[i];
    }
    double t0 = block_sum(s0, sh);
    double t1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        red.partials[blockIdx.x * 2 + 0] = t0;
        red.partials[blockIdx.x * 2 + 1] = t1;
    }
    if (finish_reduction(red, 2) && threadIdx.x == 0) {
        const double rn = sqrt(red.out[0]), xn = sqrt(red.out[1]);
        const bool conv = rn <= tol * (xn > 1.0 ? xn : 1.0);
        const int stop = !isfinite(rn) ? 2 : (conv ? 1 : (limit ? 3 : 0));
        flags[0] = stop != 0;
        st[0] = stop;
        st[1] = rn;
        st[2] = xn;
    }
}

// out[k] = <V_k, w> for k < K (V: K rows of length n2); with V == nullptr,
// out[0] = <w, w>.  One pass: each thread keeps its w entries in registers
// (at most kMaxPer per thread), warps reduce every dot by shuffles, one CTA
// barrier combines the warps.
constexpr int kMaxPer = 8;
constexpr int kMaxB = kMaxPer / 2;  // bodies per thread in the cooperative FOM kernels (at most)
// Cooperative grid for n bodies: one block per SM at least.  These kernels
// are bound by FP64 issue (on GB300 one warp-wide FP64 instruction occupies
// an SM sub-partition's FP64 unit for ~64 cycles), so the work is spread over
// every SM; more blocks only when kMaxB bodies per thread do not cover n.
static int coop_grid(int n) {
    const int need = (n + kRedThreads * kMaxB - 1) / (kRedThreads * kMaxB);
    const int sms = device_sm_count();
    return need > sms ? need : sms;
}
__global__ void k_multidot(int n2, int K, const double *V, const double *w, Red red, const int *skip = nullptr) {
    if (skip && *skip) return;
    __shared__ double sh[kRedThreads / 32][kMaxDots];
    const int stride = gridDim.x * blockDim.x;
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    double wl[kMaxPer];
#pragma unroll
    for (int e = 0; e < kMaxPer; ++e) {
        const int i = i0 + e * stride;
        wl[e] = i < n2 ? w[i] : 0.0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < K; ++k) {
        const double *vk = V ? V + (size_t)k * n2 : w;
        double s = 0.0;
#pragma unroll
        for (int e = 0; e < kMaxPer; ++e) {
            const int i = i0 + e * stride;
            if (i < n2) s += vk[i] * wl[e];
        }
        s = warp_sum(s);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int wq = 0; wq < kRedThreads / 32; ++wq) s += sh[wq][k];
        red.partials[(size_t)blockIdx.x * K + k] = s;
    }
    finish_reduction(red, K);
}

// w -= sum_k h[k] V_k;  out[0] = ||w||^2
__global__ void k_orth_update(int n2, int K, const double *V, const double *h, double *w, Red red,
                              const int *skip = nullptr) {
    if (skip && *skip) return;
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
        double v = w[i];
        for (int k = 0; k < K; ++k) v -= h[k] * V[(size_t)k * n2 + i];
        w[i] = v;
        s += v * v;
    }
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) red.partials[blockIdx.x] = t;
    finish_reduction(red, 1);
}

// Per-body 2x2 solve (I - hdt D_i)^{-1} (r0, r1) (transposed block when
// transpose is set); D = [D00 | D01 | D10], D11 = -D00.
__device__ __forceinline__ void bd_solve(const double *D, int n, int i, double hdt, int transpose, double r0,
                                         double r1, double scale, double &z0, double &z1) {
    const double d00 = D[i], d11 = -d00;
    const double d01 = transpose ? D[2 * n + i] : D[n + i], d10 = transpose ? D[n + i] : D[2 * n + i];
    const double m00 = 1.0 - hdt * d00, m01 = -hdt * d01, m10 = -hdt * d10, m11 = 1.0 - hdt * d11;
    const double det = m00 * m11 - m01 * m10;
    z0 = scale * (m11 * r0 - m01 * r1) / det;
    z1 = scale * (m00 * r1 - m10 * r0) / det;
}

// The preconditioner as stored inverse blocks: Mi = [a | b | c | d] (4 n
// doubles), M_i^{-1} = [[a, b], [c, d]] = (I - hdt D_i)^{-1}, built once per
// refresh of D so that applying it is four multiply-adds (FP64 division is
// slow on GB300 and sat on the latency path of every small FOM kernel).
__device__ __forceinline__ void minv_fill(const double *D, double *Mi, int n, int i, double hdt) {
    const double d00 = D[i], d01 = D[n + i], d10 = D[2 * n + i], d11 = -d00;
    const double m00 = 1.0 - hdt * d00, m01 = -hdt * d01, m10 = -hdt * d10, m11 = 1.0 - hdt * d11;
    const double inv = 1.0 / (m00 * m11 - m01 * m10);
    Mi[i] = m11 * inv;
    Mi[n + i] = -m01 * inv;
    Mi[2 * (size_t)n + i] = -m10 * inv;
    Mi[3 * (size_t)n + i] = m00 * inv;
}
// z = M_i^{-1} r (M_i^{-T} r when transpose is set), in arithmetic type A
template <typename A>
__device__ __forceinline__ void minv_apply(const double *Mi, int n, int i, int transpose, A r0, A r1, A &z0, A &z1) {
    const A a = (A)Mi[i], b = (A)Mi[n + i], c = (A)Mi[2 * (size_t)n + i], d = (A)Mi[3 * (size_t)n + i];
    if (transpose) {
        z0 = a * r0 + c * r1;
        z1 = b * r0 + d * r1;
    } else {
        z0 = a * r0 + b * r1;
        z1 = c * r0 + d * r1;
    }
}
__global__ void k_minv(int n, const double *D, double hdt, double *Mi) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) minv_fill(D, Mi, n, i, hdt);
}

// Block-diagonal solve: z_i = scale * (I - hdt D_i)^{-1} v_i, added to z
// when accumulate is set.
__global__ void k_blockdiag(int n, const double *D, const double *v, double hdt, double scale,
                            double *z, int accumulate, int transpose) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double z0, z1;
        bd_solve(D, n, i, hdt, transpose, v[i], v[n + i], scale, z0, z1);
        if (accumulate) {
            z[i] += z0;
            z[n + i] += z1;
        } else {
            z[i] = z0;
            z[n + i] = z1;
        }
    }
}

// Next Arnoldi vector and its preconditioned image in one pass:
//   v = scale * src / (|scale| sqrt(*nrm2))  -> V_out,   z = M^{-1} v
// (*nrm2 = ||src||^2 on the device, so the host need not read it first).
__global__ void k_norm_precond(int n, const double *src, double scale, const double *nrm2, const double *Mi,
                               int transpose, double *V_out, double *z, const int *skip) {
    if (skip && *skip) return;
    const double inv = 1.0 / (fabs(scale) * sqrt(*nrm2));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v0 = inv * (scale * src[i]), v1 = inv * (scale * src[n + i]);
        V_out[i] = v0;
        V_out[n + i] = v1;
        double z0, z1;
        minv_apply<double>(Mi, n, i, transpose, v0, v1, z0, z1);
        z[i] = z0;
        z[n + i] = z1;
    }
}

// GMRES least-squares state of one cycle on the device: the rotated
// Hessenberg matrix H [(m+1) x m] (row-major, leading dimension m), the Givens
// cosines and sines, the rotated right-hand side g [m+1], and
// scal = {||b|| (first cycle), this cycle's initial residual norm}.
struct GmDev {
    double *H, *cs, *sn, *g, *scal;
};

// One Arnoldi column into the least squares (the host-side Givens update of
// GMRES moved to the device): column j of H from the two CGS passes (h1 + h2)
// and ||w|| (nrm2 = ||w||^2), the previous rotations applied, a new one
// chosen, g rotated.  beta2: device address of the cycle's initial squared
// norm (scaled by beta_scale^2).  Writes st = {stop, ||w||, |g_{j+1}|,
// ||b||} with stop 0 = go on, 1 = converged (|g_{j+1}| <= rtol ||b||), at the
// iteration limit or breakdown (||w|| = 0), 2 = non-finite; flags[0] = stop != 0.
// The arithmetic is done in type A (FP32 when the Krylov solve is in FP32,
// see Ctx::krylov32); the state is stored in FP64.
template <typename A>
__device__ void givens_column(GmDev gm, int m, int j, const A *h1, const A *h2, A nrm2, const double *beta2,
                              double beta_scale, int first_cycle, double rtol, int total, int max_iter, int *flags,
                              double *st) {
    double *H = gm.H;
    if (j == 0) {
        const A beta = (A)fabs(beta_scale) * sqrt((A)*beta2);
        gm.g[0] = beta;
        gm.scal[1] = beta;
        if (first_cycle) gm.scal[0] = beta;
    }
    A col[kMaxRestart + 1];
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    const A hn = sqrt(nrm2);
    col[j + 1] = hn;
    int stop = 0;
    A gj1 = 0;
    if (!isfinite(hn)) {
        stop = 2;
    } else {
        for (int i = 0; i < j; ++i) {
            const A ci = (A)gm.cs[i], si = (A)gm.sn[i];
            const A a = col[i], b2 = col[i + 1];
            col[i] = ci * a + si * b2;
            col[i + 1] = -si * a + ci * b2;
        }
        const A a = col[j], b2 = col[j + 1];
        // the entries are O(1) (unit Krylov vectors, I - hdt J near I), so the
        // plain norm neither overflows nor underflows; one division
        const A rr = sqrt(a * a + b2 * b2);
        const A irr = rr > 0 ? (A)1 / rr : (A)0;
        const A cj = rr > 0 ? a * irr : (A)1, sj = rr > 0 ? b2 * irr : (A)0;
        gm.cs[j] = cj;
        gm.sn[j] = sj;
        col[j] = rr;
        col[j + 1] = 0;
        const A gj = (A)gm.g[j];
        gj1 = -sj * gj;
        gm.g[j + 1] = gj1;
        gm.g[j] = cj * gj;
        if (fabs(gj1) <= (A)rtol * (A)gm.scal[0] || total >= max_iter || hn == 0) stop = 1;
    }
    for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = col[i];
    flags[0] = stop != 0;
    st[0] = stop;
    st[1] = hn;
    st[2] = fabs(gj1);
    st[3] = gm.scal[0];
}

// GMRES correction of one cycle of K steps: y = R^{-1} g (R = the leading
// K x K block of the rotated H; each block solves it, warp 0, in shared
// memory), then d += M^{-1} (sum_k y_k V_k); with x given, also x += d (the
// Newton update after the last cycle).
template <typename A>
__global__ void k_combine_precond(int n, int K, int m, const double *V, GmDev gm, const double *Mi, int transpose,
                                  double *d, double *x) {
    __shared__ A y[kMaxRestart];
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int i = K - 1; i >= 0; --i) {
            A s = 0;
            for (int k = i + 1 + lane; k < K; k += 32) s += (A)gm.H[(size_t)i * m + k] * y[k];
            s = warp_sum(s);
            if (lane == 0) {
                const A hii = (A)gm.H[(size_t)i * m + i];
                y[i] = hii != 0 ? ((A)gm.g[i] - s) / hii : (A)0;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    const size_t n2 = 2 * (size_t)n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        A u0 = 0, u1 = 0;
        for (int k = 0; k < K; ++k) {
            u0 += y[k] * (A)V[k * n2 + i];
            u1 += y[k] * (A)V[k * n2 + n + i];
        }
        A z0, z1;
        minv_apply<A>(Mi, n, i, transpose, u0, u1, z0, z1);
        const double d0 = d[i] + z0, d1 = d[n + i] + z1;
        d[i] = d0;
        d[n + i] = d1;
        if (x) {
            x[i] += d0;
            x[n + i] += d1;
        }
    }
}

// r0 = scale * rhs - a   (a = (I - hdt J) d)
__global__ void k_restart_res(int n2, const double *rhs, double scale, const double *a, double *r0) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x)
        r0[i] = scale * rhs[i] - a[i];
}

// Arguments of givens_column for one Arnoldi step.
struct GivensArgs {
    GmDev gm;
    int m;
    const double *beta2;
    double beta_scale;
    int first_cycle;
    double rtol;
    int total, max_iter;
    int *flags;
    double *st;
};

// Classical Gram-Schmidt applied twice to w against V_0..V_{K-1}, as one
// cooperative kernel over bodies: each thread keeps both components of its
// (at most kMaxB) bodies of w in registers throughout.  Per pass: block
// partial dots -> grid barrier -> every block sums the partials in the same
// fixed order (all blocks hold identical coefficients) -> w -= sum_k h_k V_k.
// The second pass also sums ||w||^2 before its update, so the final norm is
// ||w||^2 - sum_k h2_k^2 (Pythagoras, V orthonormal) without a third
// reduction; when that subtraction loses more than half of ||w||^2 the norm is
// summed again exactly (a uniform branch: every block sees the same values).
// Outputs: out[0..K) first-pass h, out[kMaxDots..) second-pass h,
// out[2 kMaxDots] = ||w||^2; block 0 adds the column to the least squares
// (givens_column).  Finally every block writes the next Arnoldi vector
// v = w / ||w|| (Vnext) and its preconditioned image z = M^{-1} v.
// partials: 2 * gridDim.x * kMaxDots + gridDim.x doubles.
template <typename A>
__global__ void __launch_bounds__(kRedThreads)
k_cgs2(int n, int K, const double *V, const double *w, double *partials, double *out, GivensArgs ga,
       const double *Mi, int transpose, double *Vnext, double *z, const int *skip) {
    if (*skip) return;  // uniform over the grid: no block reaches a grid barrier
    cg::grid_group grid = cg::this_grid();
    __shared__ A sh[kRedThreads / 32][kMaxDots];
    __shared__ A h1s[kMaxDots], hs[kMaxDots];
    __shared__ A nrm2_s;
    const int G = gridDim.x;
    const int stride = G * blockDim.x;
    const int b0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const size_t n2 = 2 * (size_t)n;
    // bodies b0 + e * stride; `we` = how many of the e slots this warp uses
    // (a warp-uniform count, so empty slots issue no FP64 instructions: a
    // predicated-off FP64 instruction still occupies the slow FP64 pipe)
    const int wbase = blockIdx.x * blockDim.x + warp * 32;
    int we = 0;
    while (we < kMaxB && wbase + we * stride < n) ++we;
    A w0[kMaxB], w1[kMaxB];
#pragma unroll
    for (int e = 0; e < kMaxB; ++e) {
        const int i = b0 + e * stride;
        w0[e] = (e < we && i < n) ? (A)w[i] : (A)0;
        w1[e] = (e < we && i < n) ? (A)w[n + i] : (A)0;
    }
    for (int pass = 0; pass < 2; ++pass) {
        const int nk = pass == 0 ? K : K + 1;  // pass 2 also sums ||w||^2
        A *P = reinterpret_cast<A *>(partials + (size_t)pass * G * kMaxDots);
        for (int k = 0; k < nk; ++k) {
            A s = 0;
            if (we > 0) {
                if (k < K) {
                    const double *vk = V + (size_t)k * n2;
#pragma unroll
                    for (int e = 0; e < kMaxB; ++e) {
                        if (e >= we) break;
                        const int i = b0 + e * stride;
                        if (i < n) s += (A)vk[i] * w0[e] + (A)vk[n + i] * w1[e];
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < kMaxB; ++e) {
                        if (e >= we) break;
                        s += w0[e] * w0[e] + w1[e] * w1[e];
                    }
                }
                s = warp_sum(s);
            }
            if (lane == 0) sh[warp][k] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            A s = 0;
            for (int q = 0; q < nw; ++q) s += sh[q][k];
            P[(size_t)blockIdx.x * nk + k] = s;
        }
        grid.sync();
        for (int k = warp; k < nk; k += nw) {
            A s = 0;
            for (int b = lane; b < G; b += 32) s += P[(size_t)b * nk + k];
            s = warp_sum(s);
            if (lane == 0) {
                hs[k] = s;
                if (pass == 0) h1s[k] = s;
            }
        }
        __syncthreads();
        if (blockIdx.x == 0)
            for (int k = threadIdx.x; k < K; k += blockDim.x) out[pass * kMaxDots + k] = hs[k];
#pragma unroll
        for (int e = 0; e < kMaxB; ++e) {
            if (e >= we) break;
            const int i = b0 + e * stride;
            if (i < n) {
                A v0 = w0[e], v1 = w1[e];
                for (int k = 0; k < K; ++k) {
                    v0 -= hs[k] * (A)V[(size_t)k * n2 + i];
                    v1 -= hs[k] * (A)V[(size_t)k * n2 + n + i];
                }
                w0[e] = v0;
                w1[e] = v1;
            }
        }
        __syncthreads();  // sh and hs are rewritten by the next pass
    }
    if (threadIdx.x == 0) {
        A t = hs[K];  // ||w||^2 before the second update
        for (int k = 0; k < K; ++k) t -= hs[k] * hs[k];
        nrm2_s = t;
    }
    __syncthreads();
    if (!(nrm2_s >= (A)0.5 * hs[K])) {  // cancellation (or NaN): sum ||w||^2 again
        A s = 0;
        if (we > 0) {
#pragma unroll
            for (int e = 0; e < kMaxB; ++e) {
                if (e >= we) break;
                s += w0[e] * w0[e] + w1[e] * w1[e];
            }
            s = warp_sum(s);
        }
        __syncthreads();
        if (lane == 0) sh[warp][0] = s;
        __syncthreads();
        A *Pn = reinterpret_cast<A *>(partials + (size_t)2 * G * kMaxDots);
        if (threadIdx.x == 0) {
            A t = 0;
            for (int q = 0; q < nw; ++q) t += sh[q][0];
            Pn[blockIdx.x] = t;
        }
        grid.sync();
        if (warp == 0) {
            A t = 0;
            for (int b = lane; b < G; b += 32) t += Pn[b];
            t = warp_sum(t);
            if (lane == 0) nrm2_s = t;
        }
        __syncthreads();
    }
    const A nrm2 = nrm2_s;
    __shared__ A inv_s;
    if (threadIdx.x == 0) inv_s = (A)1 / sqrt(nrm2);  // once per block
    __syncthreads();
    const A inv = inv_s;
#pragma unroll
    for (int e = 0; e < kMaxB; ++e) {
        if (e >= we) break;
        const int i = b0 + e * stride;
        if (i < n) {
            const A v0 = inv * w0[e], v1 = inv * w1[e];
            Vnext[i] = v0;
            Vnext[n + i] = v1;
            A z0, z1;
            minv_apply<A>(Mi, n, i, transpose, v0, v1, z0, z1);
            z[i] = z0;
            z[n + i] = z1;
        }
    }
    // block 0, one thread: the column into the least squares (after its own
    // share of the vector writes, which the other blocks do meanwhile)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[2 * kMaxDots] = nrm2;
        givens_column<A>(ga.gm, ga.m, K - 1, h1s, hs, nrm2, ga.beta2, ga.beta_scale, ga.first_cycle, ga.rtol, ga.total,
                      ga.max_iter, ga.flags, ga.st);
    }
}

// Newton residual of the trapezoid step in one cooperative kernel over
// bodies: r = x - xprev - hdt (f(x) + fprev) [- dt u], ||r||^2 and ||x||^2 reduced in a
// fixed order that every block repeats, the Newton test (converged when
// ||r|| <= tol max(1, ||x||)) taken identically in every block.  Block 0 writes
// st = {stop, ||r||, ||x||} (stop 0 go on, 1 converged, 2 non-finite, 3 at
// the iteration limit), flags[0] = stop != 0 and redout[0..1] = the squared
// norms.  With refresh set the preconditioner blocks M_i^{-1} are first
// rebuilt from D.  When the iteration goes on, mode 1 applies the
// block-diagonal Newton update x += M^{-1}(-r); mode 2 writes the first
// Arnoldi vector v_0 = -r / ||r|| and z = M^{-1} v_0 for GMRES.
struct NewtonArgs {
    int n;
    double *x, *xprev;
    const double *fxi, *fprev;
    const double *u;  // superimposed inflow [2n] or nullptr
    double hdt;
    double *r, *partials, *redout;
    double tol;
    int limit;
    int *flags;
    double *st;
    int refresh;
    const double *D;
    double *Mi;
    int mode;
    double *V0, *z;
    int first;              // k = 0: xprev := x (x^{n-1}) and counter := 0
    double *f_out;          // f(x) -> f_out when the iteration stops (converged or at the limit)
    double *d;              // mode 2: d := 0 (the GMRES correction)
    unsigned int *counter;  // the non-cooperative reductions' arrival counter
    const int *skip;        // optional: nonzero at launch -> the kernel does nothing
    double *iters;          // optional: incremented once per iteration that runs
};
__global__ void __launch_bounds__(kRedThreads) k_newton(NewtonArgs a) {
    // every block reads the flag before the grid barrier, and block 0 writes
    // it only after it, so all blocks take the same branch here
    if (a.skip && *a.skip) return;
    cg::grid_group grid = cg::this_grid();
    __shared__ double sh[2][kRedThreads / 32];
    __shared__ double tot[2];
    const int n = a.n, G = gridDim.x, stride = G * blockDim.x;
    const int b0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int wbase = blockIdx.x * blockDim.x + warp * 32;  // warp-uniform body slots, as in k_cgs2
    int we = 0;
    while (we < kMaxB && wbase + we * stride < n) ++we;
    double r0[kMaxB], r1[kMaxB];
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int e = 0; e < kMaxB; ++e) {
        const int i = b0 + e * stride;
        r0[e] = 0.0;
        r1[e] = 0.0;
        if (e < we && i < n) {
            if (a.refresh) minv_fill(a.D, a.Mi, n, i, a.hdt);
            const double x0 = a.x[i], x1 = a.x[n + i];
            double xp0, xp1;
            if (a.first) {
                xp0 = x0;
                xp1 = x1;
                a.xprev[i] = x0;
                a.xprev[n + i] = x1;
            } else {
                xp0 = a.xprev[i];
                xp1 = a.xprev[n + i];
            }
            double v0 = x0 - xp0 - a.hdt * (a.fxi[i] + a.fprev[i]);
            double v1 = x1 - xp1 - a.hdt * (a.fxi[n + i] + a.fprev[n + i]);
            if (a.u) {
                v0 -= (2.0 * a.hdt) * a.u[i];
                v1 -= (2.0 * a.hdt) * a.u[n + i];
            }
            a.r[i] = v0;
            a.r[n + i] = v1;
            r0[e] = v0;
            r1[e] = v1;
            s0 += v0 * v0 + v1 * v1;
            s1 += x0 * x0 + x1 * x1;
        }
    }
    if (we > 0) {
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
    }
    if (lane == 0) {
        sh[0][warp] = s0;
        sh[1][warp] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += sh[threadIdx.x][q];
        a.partials[(size_t)blockIdx.x * 2 + threadIdx.x] = t;
    }
    grid.sync();
    if (warp < 2) {
        double t = 0.0;
        for (int b = lane; b < G; b += 32) t += a.partials[(size_t)b * 2 + warp];
        t = warp_sum(t);
        if (lane == 0) tot[warp] = t;
    }
    __syncthreads();
    // the Newton test once per block (identical in every block), broadcast
    __shared__ int stop_s;
    __shared__ double rn_s, xn_s, inv_s;
    if (threadIdx.x == 0) {
        const double rn = sqrt(tot[0]), xn = sqrt(tot[1]);
        const bool conv = rn <= a.tol * (xn > 1.0 ? xn : 1.0);
        stop_s = !isfinite(rn) ? 2 : (conv ? 1 : (a.limit ? 3 : 0));
        rn_s = rn;
        xn_s = xn;
        inv_s = 1.0 / rn;
    }
    __syncthreads();
    const int stop = stop_s;
    const double rn = rn_s, xn = xn_s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.iters) *a.iters += 1.0;
        a.flags[0] = stop != 0;
        a.st[0] = stop;
        a.st[1] = rn;
        a.st[2] = xn;
        a.redout[0] = tot[0];
        a.redout[1] = tot[1];
        if (a.first) *a.counter = 0u;
    }
    if (stop == 1 || stop == 3) {  // the step ends here: f(x^n) into f
#pragma unroll
        for (int e = 0; e < kMaxB; ++e) {
            const int i = b0 + e * stride;
            if (e < we && i < n) {
                a.f_out[i] = a.fxi[i];
                a.f_out[n + i] = a.fxi[n + i];
            }
        }
    }
    if (stop != 0 || a.mode == 0) return;
    const double inv = inv_s;
#pragma unroll
    for (int e = 0; e < kMaxB; ++e) {
        const int i = b0 + e * stride;
        if (e >= we || i >= n) continue;
        if (a.mode == 1) {
            double z0, z1;
            minv_apply(a.Mi, n, i, 0, -r0[e], -r1[e], z0, z1);
            a.x[i] += z0;
            a.x[n + i] += z1;
        } else {
            const double v0 = inv * -r0[e], v1 = inv * -r1[e];
            a.V0[i] = v0;
            a.V0[n + i] = v1;
            a.d[i] = 0.0;
            a.d[n + i] = 0.0;
            double z0, z1;
            minv_apply(a.Mi, n, i, 0, v0, v1, z0, z1);
            a.z[i] = z0;
            a.z[n + i] = z1;
        }
    }
}

// The same least-squares update after the four-launch CGS2 (grids too large
// to be co-resident): one thread.
__global__ void k_givens(int K, const double *out, GivensArgs ga, const int *skip) {
    if (*skip) return;
    givens_column<double>(ga.gm, ga.m, K - 1, out, out + kMaxDots, out[2 * kMaxDots], ga.beta2, ga.beta_scale,
                  ga.first_cycle, ga.rtol, ga.total, ga.max_iter, ga.flags, ga.st);
}

// y += a * x
__global__ void k_axpy(int n2, double a, const double *x, double *y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) y[i] += a * x[i];
}

// ---------------------------------------------------------------- dense path
// M = I - hdt J (row-major m x m, m = 2n); J's diagonal blocks are the self
// blocks D, the off-diagonal block (i, j) is -gamma_j A(x_i - x_j).
__global__ void k_dense_assemble(int n, const double *x, const double *G, double delta, const double *D,
                                 double hdt, double *M) {
    const int m = 2 * n;
    const long long total = (long long)m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(e / m), col = (int)(e % m);
        const int i = row % n, ci = row / n, j = col % n, cj = col / n;
        double Jij;
        if (i == j) {
            const double d00 = D[i], d01 = D[n + i], d10 = D[2 * n + i];
            Jij = ci == 0 ? (cj == 0 ? d00 : d01) : (cj == 0 ? d10 : -d00);
        } else {
            const double a = x[i] - x[j], b = x[n + i] - x[n + j];
            if (a == 0.0 && b == 0.0) {
                Jij = 0.0;
            } else {
                const double s = a * a + b * b + delta, s2 = s * s;
                double A;
                if (ci == 0) A = cj == 0 ? 2.0 * a * b / s2 : -1.0 / s + 2.0 * b * b / s2;
                else A = cj == 0 ? 1.0 / s - 2.0 * a * a / s2 : -2.0 * a * b / s2;
                Jij = -(G[j] * kInv2Pi) * A;
            }
        }
        M[e] = (row == col ? 1.0 : 0.0) - hdt * Jij;
    }
}

// In-place LU with partial pivoting; rows are permuted logically (perm[l] is
// the physical row holding logical row l).  Every CTA finds the pivot itself
// (same data, same order -> same choice), so one grid barrier per column.
__global__ void k_lu_coop(int m, double *A, int *perm, int *status) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ int sperm[];
    __shared__ double bval[32];
    __shared__ int bidx[32];
    __shared__ int piv_s;
    for (int i = threadIdx.x; i < m; i += blockDim.x) sperm[i] = i;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int gwarp = blockIdx.x * nwarps + warp, gwarps = gridDim.x * nwarps;
    for (int k = 0; k < m; ++k) {
        // pivot search over logical rows k..m-1 (max |a|, ties -> lowest row)
        double best = -1.0;
        int bi = m;
        for (int l = k + threadIdx.x; l < m; l += blockDim.x) {
            const double v = fabs(A[(size_t)sperm[l] * m + k]);
            if (v > best || (v == best && l < bi)) { best = v; bi = l; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { bval[warp] = best; bidx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bb = -1.0;
            int ii = m;
            for (int w = 0; w < nwarps; ++w)
                if (bval[w] > bb || (bval[w] == bb && bidx[w] < ii)) { bb = bval[w]; ii = bidx[w]; }
            const int t = sperm[k];
            sperm[k] = sperm[ii];
            sperm[ii] = t;
            piv_s = (bb > 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (!piv_s) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *status = 1 + k;  // singular at column k
            break;  // every CTA sees the same zero pivot and leaves together
        }
        const double *prow = A + (size_t)sperm[k] * m;
        const double pkk = prow[k];
        for (int l = k + 1 + gwarp; l < m; l += gwarps) {
            double *row = A + (size_t)sperm[l] * m;
            const double lk = row[k] / pkk;
            for (int c = k + 1 + lane; c < m; c += 32) row[c] -= lk * prow[c];
            __syncwarp();
            if (lane == 0) row[k] = lk;
        }
        grid.sync();
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) perm[i] = sperm[i];
    }
}

// Solve (LU) d = rhs * scale with the factors of k_lu_coop (one CTA).
__global__ void k_lu_solve(int m, const double *A, const int *perm, const double *rhs, double scale, double *y) {
    for (int l = threadIdx.x; l < m; l += blockDim.x) y[l] = scale * rhs[perm[l]];
    __syncthreads();
    // forward: unit lower
    for (int k = 0; k < m; ++k) {
        const double yk = y[k];
        for (int l = k + 1 + threadIdx.x; l < m; l += blockDim.x) y[l] -= A[(size_t)perm[l] * m + k] * yk;
        __syncthreads();
    }
    // backward: upper
    for (int k = m - 1; k >= 0; --k) {
        if (threadIdx.x == 0) y[k] = y[k] / A[(size_t)perm[k] * m + k];
        __syncthreads();
        const double yk = y[k];
        for (int l = threadIdx.x; l < k; l += blockDim.x) y[l] -= A[(size_t)perm[l] * m + k] * yk;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- workspace
// Status records copied to the host: slot 0 the Newton residual
// {stop, ||r||, ||x||}, slot 1 + j Arnoldi step j {stop, ||w||, |g_{j+1}|, ||b||}.
constexpr int kStatDoubles = 4;
constexpr int kStatSlots = kMaxRestart + 1;

struct Work {
    double *xprev, *fprev, *fxi, *r, *D, *d, *jz, *w, *z, *b, *V, *partials, *redout, *M;
    double *stat;  // [kStatSlots][kStatDoubles]
    double *Mi;    // [4][n] preconditioner blocks (M_i^{-1})
    GmDev gm;
    void *pack;
    size_t pack_bytes;
    unsigned int *counter;
    int *flags;    // flags[0]: skip the queued Newton-update kernels
    int *perm, *status;
    size_t bytes;
};

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

static int red_grid(int n2) {
    int g = (n2 + kRedThreads - 1) / kRedThreads;
    const int cap = 2 * device_sm_count();
    g = g < 1 ? 1 : (g > cap ? cap : g);
    // k_multidot keeps at most kMaxPer entries of w per thread
    const int need = (n2 + kRedThreads * kMaxPer - 1) / (kRedThreads * kMaxPer);
    return g < need ? need : g;
}

static Work layout(const ptrom_fom_params *p, int n, char *base) {
    Work W{};
    size_t off = 0;
    const size_t n2 = 2 * (size_t)n;
    auto take = [&](size_t bytes) {
        char *ptr = base ? base + off : nullptr;
        off += align256(bytes);
        return ptr;
    };
    W.xprev = (double *)take(n2 * 8);
    W.fprev = (double *)take(n2 * 8);
    W.fxi = (double *)take(n2 * 8);
    W.r = (double *)take(n2 * 8);
    W.D = (double *)take(3 * (size_t)n * 8);
    W.Mi = (double *)take(4 * (size_t)n * 8);
    W.d = (double *)take(n2 * 8);
    W.jz = (double *)take(n2 * 8);
    W.w = (double *)take(n2 * 8);
    W.z = (double *)take(n2 * 8);
    W.b = (double *)take(n2 * 8);
    const int m = (p->jac_mode == PTROM_JAC_JFNK) ? p->gmres_restart : 0;
    W.V = (double *)take((size_t)(m + 1) * n2 * 8);
    // reductions: per-block partials, 2 passes of dots + 1 norm (k_cgs2)
    const int rg = std::max(std::max(red_grid((int)n2), 2 * device_sm_count()), coop_grid(n));
    W.partials = (double *)take(((size_t)2 * rg * kMaxDots + rg) * 8);
    W.redout = (double *)take(4 * kMaxDots * 8);
    W.counter = (unsigned int *)take(64);
    W.flags = (int *)take(64);
    W.stat = (double *)take(sizeof(double) * kStatSlots * kStatDoubles);
    W.gm.H = (double *)take(sizeof(double) * (kMaxRestart + 1) * kMaxRestart);
    W.gm.cs = (double *)take(sizeof(double) * kMaxRestart);
    W.gm.sn = (double *)take(sizeof(double) * kMaxRestart);
    W.gm.g = (double *)take(sizeof(double) * (kMaxRestart + 1));
    W.gm.scal = (double *)take(sizeof(double) * 2);
    W.pack_bytes = pack_scratch_bytes(n, n);
    W.pack = take(W.pack_bytes);
    if (p->jac_mode == PTROM_JAC_DENSE) {
        W.M = (double *)take(n2 * n2 * 8);
        W.perm = (int *)take(n2 * 4);
        W.status = (int *)take(64);
    }
    W.bytes = off;
    return W;
}

static int validate(const ptrom_fom_params *p, int n) {
    if (!p) return set_error(PTROM_EINVAL, "fom: NULL params");
    if (n < 2) return set_error(PTROM_EINVAL, "fom: n must be >= 2");
    if (!(p->dt > 0.0)) return set_error(PTROM_EINVAL, "fom: dt must be > 0");
    if (!(p->delta >= 0.0)) return set_error(PTROM_EINVAL, "fom: delta must be >= 0");
    if (!(p->tol >= 0.0)) return set_error(PTROM_EINVAL, "fom: tol must be >= 0");
    if (p->max_iter < 1) return set_error(PTROM_EINVAL, "fom: max_iter must be >= 1");
    if (p->p_it < 1) return set_error(PTROM_EINVAL, "fom: p_it must be >= 1");
    if (p->prec != PTROM_FP32C && p->prec != PTROM_FP64) return set_error(PTROM_EINVAL, "fom: bad prec");
    if (p->jac_mode == PTROM_JAC_JFNK) {
        if (p->gmres_restart < 1 || p->gmres_restart > kMaxRestart)
            return set_error(PTROM_EINVAL, "fom: gmres_restart must be in [1, %d]", kMaxRestart);
        if (p->gmres_max_iter < 1) return set_error(PTROM_EINVAL, "fom: gmres_max_iter must be >= 1");
        if (!(p->gmres_rtol > 0.0)) return set_error(PTROM_EINVAL, "fom: gmres_rtol must be > 0");
    } else if (p->jac_mode == PTROM_JAC_DENSE) {
        if (n > kDenseMaxN) return set_error(PTROM_EINVAL, "fom: dense Jacobian limited to n <= %d", kDenseMaxN);
    } else if (p->jac_mode != PTROM_JAC_BLOCKDIAG) {
        return set_error(PTROM_EINVAL, "fom: bad jac_mode %d", p->jac_mode);
    }
    return PTROM_OK;
}

// ---------------------------------------------------------------- solvers
struct Ctx {
    int transpose = 0;  // GMRES on (I - hdt J)^T (adjoint solves) instead of (I - hdt J)
    const ptrom_fom_params *p;
    int n, n2;
    const double *G;
    const double *xi;
    double hdt;
    cudaStream_t st;
    Work W;
    int grid, rgrid;
    int cgrid = 1;      // blocks of the cooperative kernels
    bool coop = false;  // cooperative CGS2 / Newton kernels (cgrid blocks co-resident)
    // Krylov arithmetic (CGS2, least squares, correction) in FP32: when the
    // pair sums are FP32 and the GMRES tolerance is loose (>= 1e-5) the solve
    // needs no FP64, and on GB300 every dependent FP64 operation costs
    // hundreds of cycles (the reductions and the scalar chain of one Arnoldi
    // step are latency-bound).  Vectors stay FP64 in memory either way.
    bool krylov32 = false;
    ptrom_fom_stats *stats;
    double *mb = nullptr;        // pinned status mailbox [kStatSlots][kStatDoubles]
    cudaEvent_t *ev = nullptr;   // one event per mailbox slot
};

// Whether `blocks` CTAs of the cooperative FOM kernels (k_cgs2, k_newton) fit
// on the device at once and cover n bodies with kMaxB bodies per thread.
static bool coop_fits(int blocks, int n) {
    static int per_sm = -1;
    if (per_sm < 0) {
        int v1 = 0, v2 = 0;
        int v3 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v1, k_cgs2<double>, kRedThreads, 0) != cudaSuccess) v1 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v3, k_cgs2<float>, kRedThreads, 0) != cudaSuccess) v3 = 0;
        v1 = v1 < v3 ? v1 : v3;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v2, k_newton, kRedThreads, 0) != cudaSuccess) v2 = 0;
        per_sm = v1 < v2 ? v1 : v2;
    }
    return blocks <= per_sm * device_sm_count() && (long long)blocks * kRedThreads * kMaxB >= n;
}

static Red mkred(const Work &W, int slot) { return Red{W.partials, W.counter, W.redout + slot * kMaxDots}; }

// A launch timed under `kind` (ptrom_timing_*); its slot goes to *slots when given.
#define PTROM_TIMED(kind, stream, slots, ...)             \
    do {                                                  \
        const int _slot = timing_begin((kind), (stream)); \
        __VA_ARGS__;                                      \
        timing_end(_slot, (stream));                      \
        if (slots) (slots)->add(_slot);                   \
    } while (0)
static void discard(Slots &s) {
    for (int i = 0; i < s.n; ++i) timing_discard(s.s[i]);
    s.n = 0;
}

static int fetch(const Ctx &c, const double *dev, double *host, int count) {
    PTROM_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, c.st));
    PTROM_CUDA(cudaStreamSynchronize(c.st));
    return PTROM_OK;
}

// Queue the copy of status slot k to the pinned mailbox and its event.
static int post(Ctx &c, int k) {
    PTROM_CUDA(cudaMemcpyAsync(c.mb + k * kStatDoubles, c.W.stat + k * kStatDoubles, sizeof(double) * kStatDoubles,
                               cudaMemcpyDeviceToHost, c.st));
    PTROM_CUDA(cudaEventRecord(c.ev[k], c.st));
    return PTROM_OK;
}

// Wait for status slot k (the stream may hold later work) and return it.
static const double *wait_post(Ctx &c, int k) {
    if (cudaEventSynchronize(c.ev[k]) != cudaSuccess) return nullptr;
    return c.mb + k * kStatDoubles;
}

// out = J v, or with lin set out = (I - hdt J) v, through the all-pairs
// J v kernel (J^T w for the adjoint solves).
static int apply_jvp(Ctx &c, const double *v, double *out, bool lin, const int *skip = nullptr,
                     Slots *slots = nullptr) {
    LaunchOpts o;
    o.scratch = c.W.pack;
    o.scratch_bytes = c.W.pack_bytes;
    o.skip = skip;
    o.slots = slots;
    if (lin) {
        o.lin.z = v;
        o.lin.hdt = c.hdt;
    }
    if (c.transpose) {
        PTROM_TRY(vjp(c.n, c.xi, c.G, c.p->delta, v, out, nullptr, c.p->prec, c.st, o));
    } else {
        PTROM_TRY(jvp(c.n, c.xi, c.G, c.p->delta, v, out, c.p->prec, c.st, o));
    }
    return PTROM_OK;
}

// One GMRES cycle's fixed launch arguments.
struct Cycle {
    const double *r0;       // cycle start vector (times r0_scale)
    double r0_scale;
    const double *r0_nrm2;  // device ||r0||^2
    int first;              // first cycle (defines ||b||)
    int total;              // Arnoldi steps taken in earlier cycles
};

// Queue Arnoldi step j of a cycle; every kernel of it skips itself when
// flags[0] is set (an earlier step or the Newton test already stopped), so a
// step may be queued before the previous one's outcome is known.
static int queue_step(Ctx &c, const Cycle &cy, int j, Slots *slots) {
    Work &W = c.W;
    const int n2 = c.n2, m = c.p->gmres_restart;
    const int *skip = W.flags;
    double *vj = W.V + (size_t)j * n2;
    // v_j = previous Krylov vector / its norm (read on the device); z = M^{-1} v_j.
    // The cooperative path has these from the kernel that ended step j - 1
    // (or from k_newton / the cycle set-up for j = 0).
    if (!c.coop) {
        const double *src = j == 0 ? cy.r0 : W.w;
        const double *nrm2 = j == 0 ? cy.r0_nrm2 : W.redout + 3 * kMaxDots;
        const double sc = j == 0 ? cy.r0_scale : 1.0;
        PTROM_TIMED(PTROM_K_FOM_VEC, c.st, slots,
                    k_norm_precond<<<c.grid, 256, 0, c.st>>>(c.n, src, sc, nrm2, W.Mi, c.transpose, vj, W.z, skip));
        count_launch();
    }
    PTROM_TRY(apply_jvp(c, W.z, W.w, true, skip, slots));  // w = (I - hdt J) z
    GivensArgs ga{W.gm, m, cy.r0_nrm2, cy.r0_scale, cy.first, c.p->gmres_rtol, cy.total + j + 1,
                  c.p->gmres_max_iter, W.flags, W.stat + (1 + j) * kStatDoubles};
    int K = j + 1;
    if (c.coop) {
        const double *V = W.V, *Mi = W.Mi;
        const double *w = W.w;
        double *P = W.partials, *out = W.redout + kMaxDots, *Vn = W.V + (size_t)(j + 1) * n2, *z = W.z;
        int nv = c.n, tr = c.transpose;
        void *args[] = {&nv, &K, &V, &w, &P, &out, &ga, &Mi, &tr, &Vn, &z, &skip};
        cudaError_t e = cudaSuccess;
        PTROM_TIMED(PTROM_K_FOM_ORTH, c.st, slots,
                    e = cudaLaunchCooperativeKernel(c.krylov32 ? (void *)k_cgs2<float> : (void *)k_cgs2<double>,
                                                    dim3(c.cgrid), dim3(kRedThreads), args, 0, c.st));
        PTROM_CUDA(e);
        count_launch();
    } else {
        PTROM_TIMED(PTROM_K_FOM_ORTH, c.st, slots,
                    k_multidot<<<c.rgrid, kRedThreads, 0, c.st>>>(n2, K, W.V, W.w, mkred(W, 1), skip);
                    k_orth_update<<<c.rgrid, kRedThreads, 0, c.st>>>(n2, K, W.V, W.redout + kMaxDots, W.w,
                                                                      mkred(W, 3), skip);
                    k_multidot<<<c.rgrid, kRedThreads, 0, c.st>>>(n2, K, W.V, W.w, mkred(W, 2), skip);
                    k_orth_update<<<c.rgrid, kRedThreads, 0, c.st>>>(n2, K, W.V, W.redout + 2 * kMaxDots, W.w,
                                                                      mkred(W, 3), skip);
                    k_givens<<<1, 1, 0, c.st>>>(K, W.redout + kMaxDots, ga, skip));
        count_launch(5);
    }
    PTROM_CUDA(cudaGetLastError());
    return post(c, 1 + j);
}

// Solve (I - hdt J) d = rhs_scale * rhs with right-preconditioned GMRES(m),
// M = blockdiag(I - hdt D_i); d starts at 0.  rhs_nrm2: device ||rhs||^2.
// With x_upd given, x_upd += d at the end (the Newton update).
// queued: Arnoldi steps of the first cycle the caller has already queued
// (0 or 1, with their timing slots in *first); the caller then has also
// written v_0 and z = M^{-1} v_0 (k_newton).
//
// Pipelining: step j + 1 is queued before the host waits for step j's status,
// so the GPU never waits for the host inside a cycle; when step j stops the
// cycle, the queued step j + 1 runs as empty kernels and its timing slot is
// dropped.
static int gmres(Ctx &c, const double *rhs, double rhs_scale, double *d, double *x_upd, const double *rhs_nrm2,
                 int queued = 0, const Slots *first = nullptr) {
    const int n2 = c.n2, m = c.p->gmres_restart;
    Work &W = c.W;
    std::vector<Slots> tslot(m + 1);
    if (queued && first) tslot[0] = *first;
    Cycle cy{rhs, rhs_scale, rhs_nrm2, 1, 0};
    double bnorm = 0.0;
    while (true) {
        int next = queued;
        if (next == 0) {
            if (c.coop) {  // v_0 and z for the cooperative path
                PTROM_TIMED(PTROM_K_FOM_VEC, c.st, (Slots *)nullptr,
                            k_norm_precond<<<c.grid, 256, 0, c.st>>>(c.n, cy.r0, cy.r0_scale, cy.r0_nrm2, W.Mi,
                                                                     c.transpose, W.V, W.z, nullptr));
                count_launch();
            }
            PTROM_TRY(queue_step(c, cy, next++, &tslot[0]));
        }
        int K = m;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            if (next == j + 1 && next < m) {
                PTROM_TRY(queue_step(c, cy, next, &tslot[next]));
                ++next;
            }
            const double *st = wait_post(c, 1 + j);
            if (!st) return set_error(PTROM_ECUDA, "fom: waiting for GMRES step %d failed", j);
            if (c.stats) {
                c.stats->jvp_evals++;
                c.stats->linear_iters++;
            }
            bnorm = st[3];
            if (st[0] == 2.0) return set_error(PTROM_ENAN, "fom: non-finite Krylov vector");
            if (st[0] != 0.0) {
                K = j + 1;
                done = true;
                break;
            }
        }
        for (int j = K; j < next; ++j) discard(tslot[j]);  // queued steps that did nothing
        for (auto &t : tslot) t.n = 0;
        queued = 0;
        double *xu = done ? x_upd : nullptr;
        if (c.krylov32)
            PTROM_TIMED(PTROM_K_FOM_VEC, c.st, (Slots *)nullptr,
                        k_combine_precond<float><<<c.grid, 256, 0, c.st>>>(c.n, K, m, W.V, W.gm, W.Mi, c.transpose,
                                                                           d, xu));
        else
            PTROM_TIMED(PTROM_K_FOM_VEC, c.st, (Slots *)nullptr,
                        k_combine_precond<double><<<c.grid, 256, 0, c.st>>>(c.n, K, m, W.V, W.gm, W.Mi, c.transpose,
                                                                            d, xu));
        count_launch();
        PTROM_CUDA(cudaGetLastError());
        if (done) break;
        // restart: r0 = b - (I - hdt J) d
        PTROM_TRY(apply_jvp(c, d, W.jz, true));
        if (c.stats) c.stats->jvp_evals++;
        PTROM_TIMED(PTROM_K_FOM_VEC, c.st, (Slots *)nullptr,
                    k_restart_res<<<c.grid, 256, 0, c.st>>>(n2, rhs, rhs_scale, W.jz, W.b);
                    k_multidot<<<c.rgrid, kRedThreads, 0, c.st>>>(n2, 1, nullptr, W.b, mkred(W, 0)));
        count_launch(2);
        double r2 = 0.0;
        PTROM_TRY(fetch(c, W.redout, &r2, 1));
        if (sqrt(r2) <= c.p->gmres_rtol * bnorm) {
            if (x_upd) {
                k_axpy<<<c.grid, 256, 0, c.st>>>(n2, 1.0, d, x_upd);
                count_launch();
            }
            break;
        }
        cy = Cycle{W.b, 1.0, W.redout, 0, cy.total + m};
        PTROM_CUDA(cudaMemsetAsync(W.flags, 0, sizeof(int), c.st));
    }
    return PTROM_OK;
}

static int dense_factor(Ctx &c) {
    const int m = c.n2;
    Work &W = c.W;
    const long long total = (long long)m * m;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8 * device_sm_count()) blocks = 8 * device_sm_count();
    k_dense_assemble<<<blocks, 256, 0, c.st>>>(c.n, c.xi, c.G, c.p->delta, W.D, c.hdt, W.M);
    count_launch();
    PTROM_CUDA(cudaGetLastError());
    PTROM_CUDA(cudaMemsetAsync(W.status, 0, sizeof(int), c.st));
    const int threads = 512;
    const size_t smem = sizeof(int) * (size_t)m;
    int per_sm = 0;
    PTROM_CUDA(cudaFuncSetAttribute(k_lu_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PTROM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_coop, threads, smem));
    if (per_sm < 1) return set_error(PTROM_ECUDA, "fom: LU kernel cannot be resident");
    int grid = per_sm * device_sm_count();        // co-resident by construction
    const int need = (m + threads / 32 - 1) / (threads / 32);  // one warp per row at k = 0
    if (grid > need) grid = need;
    int mm = m;
    double *A = W.M;
    int *perm = W.perm, *status = W.status;
    void *args[] = {&mm, &A, &perm, &status};
    PTROM_CUDA(cudaLaunchCooperativeKernel((void *)k_lu_coop, dim3(grid), dim3(threads), args, smem, c.st));
    count_launch();
    int st = 0;
    PTROM_CUDA(cudaMemcpyAsync(&st, W.status, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    PTROM_CUDA(cudaStreamSynchronize(c.st));
    if (st != 0) return set_error(PTROM_ENAN, "fom: dense Jacobian singular at column %d", st - 1);
    return PTROM_OK;
}

bool timing_active();  // status.cu: launches are being event-timed

// Rollout bookkeeping of fom_steps: flags[0] is the skip flag of the step's
// kernels, flags[1] halts the rest of the rollout.  At a step's start its
// kernels run unless an earlier step halted; at its end the step's status
// (stop, |r|, iterations that ran) goes to log[step] and a step that did not
// converge halts the rest.
__global__ void k_roll_begin(int *flags, double *iters) {
    flags[0] = flags[1];
    *iters = 0.0;
}
__global__ void k_roll_end(int *flags, const double *st, const double *iters, double *log, int *step) {
    if (flags[1]) return;
    const int s = *step;
    log[3 * s] = st[0];
    log[3 * s + 1] = st[1];
    log[3 * s + 2] = *iters;
    *step = s + 1;
    if (st[0] != 1.0) flags[1] = 1;
}

}  // namespace ptrom

using namespace ptrom;

extern "C" size_t fom_workspace_bytes(const ptrom_fom_params *p, int n) {
    if (validate(p, n) != PTROM_OK) return 0;
    return layout(p, n, nullptr).bytes;
}

// The solver context of one call (fom_step, fom_steps).
static int init_ctx(Ctx &c, const char *fn, const ptrom_fom_params *p, int n, const double *Gamma, double *x,
                    double *f, void *work, size_t work_bytes, ptrom_stream_t stream) {
    PTROM_TRY(validate(p, n));
    if (!Gamma || !x || !f || !work) return set_error(PTROM_EINVAL, "%s: NULL pointer", fn);
    if (((uintptr_t)work) & 255) return set_error(PTROM_EINVAL, "%s: work must be 256-byte aligned", fn);
    c.p = p;
    c.n = n;
    c.n2 = 2 * n;
    c.G = Gamma;
    c.xi = x;
    c.hdt = 0.5 * p->dt;
    c.st = (cudaStream_t)stream;
    c.W = layout(p, n, (char *)work);
    if (work_bytes < c.W.bytes)
        return set_error(PTROM_EINVAL, "%s: work has %zu bytes, needs %zu", fn, work_bytes, c.W.bytes);
    c.grid = (c.n2 + 255) / 256;
    if (c.grid > 4 * device_sm_count()) c.grid = 4 * device_sm_count();
    c.rgrid = red_grid(c.n2);
    c.cgrid = coop_grid(n);
    c.coop = coop_fits(c.cgrid, n);
    c.krylov32 = c.coop && p->prec == PTROM_FP32C && p->gmres_rtol >= 1e-5;
    return host_mailbox(kStatSlots * kStatDoubles, kStatSlots, &c.mb, &c.ev);
}

extern "C" int fom_step(const ptrom_fom_params *p, int n, const double *Gamma, double *x, double *f,
                        void *work, size_t work_bytes, ptrom_fom_stats *stats, ptrom_stream_t stream) {
    Ctx c{};
    PTROM_TRY(init_ctx(c, "fom_step", p, n, Gamma, x, f, work, work_bytes, stream));
    ptrom_fom_stats local{};
    c.stats = stats ? stats : &local;
    memset(c.stats, 0, sizeof(*c.stats));
    Work &W = c.W;
    // f keeps f(x^{n-1}) until the step's last residual, so it serves as fprev;
    // the cooperative Newton kernel copies x^{n-1} and zeroes the reduction
    // counter itself at k = 0
    if (!c.coop) {
        PTROM_CUDA(cudaMemsetAsync(W.counter, 0, 64, c.st));
        PTROM_CUDA(cudaMemcpyAsync(W.xprev, x, sizeof(double) * c.n2, cudaMemcpyDeviceToDevice, c.st));
    }
    bool have_jac = false;
    for (int k = 0; k <= p->max_iter; ++k) {
        const bool refresh = (k % p->p_it == 0) || !have_jac;
        LaunchOpts vo;
        vo.scratch = W.pack;
        vo.scratch_bytes = W.pack_bytes;
        PTROM_TRY(velocity(n, x, n, x, Gamma, p->delta, W.fxi, refresh ? W.D : nullptr, p->prec, c.st, vo));
        c.stats->velocity_evals++;
        const bool jfnk = p->jac_mode == PTROM_JAC_JFNK;
        if (c.coop) {
            // residual, norms, Newton test, M^{-1} refresh and (block-diagonal)
            // the Newton update or (JFNK) v_0 and z in one cooperative launch
            NewtonArgs na{n, x, W.xprev, W.fxi, f, p->u_inf, c.hdt, W.r, W.partials, W.redout, p->tol,
                          k == p->max_iter, W.flags, W.stat, refresh ? 1 : 0, W.D, W.Mi,
                          p->jac_mode == PTROM_JAC_BLOCKDIAG ? 1 : (jfnk ? 2 : 0), W.V, W.z,
                          k == 0 ? 1 : 0, f, W.d, W.counter};
            void *args[] = {&na};
            cudaError_t e = cudaSuccess;
            PTROM_TIMED(PTROM_K_FOM_VEC, c.st, (Slots *)nullptr,
                        e = cudaLaunchCooperativeKernel((void *)k_newton, dim3(c.cgrid), dim3(kRedThreads), args, 0,
                                                        c.st));
            PTROM_CUDA(e);
            count_launch();
        } else {
            if (refresh) {
                k_minv<<<c.grid, 256, 0, c.st>>>(n, W.D, c.hdt, W.Mi);
                count_launch();
            }
            PTROM_TIMED(PTROM_K_FOM_VEC, c.st, (Slots *)nullptr,
                        k_residual<<<c.rgrid, kRedThreads, 0, c.st>>>(c.n2, x, W.xprev, W.fxi, f, p->u_inf, c.hdt, W.r,
                                                                     mkred(W, 0), p->tol, k == p->max_iter, W.flags,
                                                                     W.stat));
            count_launch();
        }
        PTROM_CUDA(cudaGetLastError());
        PTROM_TRY(post(c, 0));
        // JFNK: queue the first Arnoldi step before reading the Newton test
        // (it skips itself if the test stops the iteration)
        Slots slot0;
        if (jfnk) {
            if (!c.coop) PTROM_CUDA(cudaMemsetAsync(W.d, 0, sizeof(double) * c.n2, c.st));
            const Cycle cy{W.r, -1.0, W.redout, 1, 0};
            PTROM_TRY(queue_step(c, cy, 0, &slot0));
        }
        const double *st = wait_post(c, 0);
        if (!st) return set_error(PTROM_ECUDA, "fom_step: waiting for the residual failed");
        const int stop = (int)st[0];
        const double rn = st[1];
        if (k == 0) c.stats->res_norm0 = rn;
        c.stats->res_norm = rn;
        if (stop != 0) {
            discard(slot0);
            if (stop == 2) return set_error(PTROM_ENAN, "fom_step: non-finite residual at iteration %d", k);
            if (!c.coop)  // (the cooperative Newton kernel has copied f(x^n) into f)
                PTROM_CUDA(cudaMemcpyAsync(f, W.fxi, sizeof(double) * c.n2, cudaMemcpyDeviceToDevice, c.st));
            if (stop == 3) return set_error(PTROM_ENOCONV, "fom_step: %d Newton iterations, |r| = %.3e", k, rn);
            return PTROM_OK;
        }
        c.stats->newton_iters++;
        if (p->jac_mode == PTROM_JAC_BLOCKDIAG) {
            if (!c.coop) {  // (the cooperative residual kernel already applied it)
                k_blockdiag<<<c.grid, 256, 0, c.st>>>(n, W.D, W.r, c.hdt, -1.0, x, 1, 0);
                count_launch();
            }
        } else if (jfnk) {
            // solve (I - hdt J) d = -r; x += d (slot 0 of redout holds ||r||^2)
            PTROM_TRY(gmres(c, W.r, -1.0, W.d, x, W.redout, 1, &slot0));
        } else {
            if (refresh) PTROM_TRY(dense_factor(c));
            k_lu_solve<<<1, 1024, 0, c.st>>>(c.n2, W.M, W.perm, W.r, -1.0, W.d);
            count_launch();
            k_axpy<<<c.grid, 256, 0, c.st>>>(c.n2, 1.0, W.d, x);
            count_launch();
        }
        PTROM_CUDA(cudaGetLastError());
        have_jac = true;
    }
    return PTROM_OK;
}


namespace ptrom {
// ---------------------------------------------------------------- adjoint step
// Reverse-mode derivative of one trapezoid step (implicit function theorem on
// r(x^n, x^{n-1}, Gamma) = 0):
//   mu          = (I - dt/2 J(x^n))^{-T} lambda          (GMRES on J^T w)
//   lambda_prev = mu + dt/2 J(x^{n-1})^T mu
//   gGamma     += dt/2 (F(x^n) + F(x^{n-1}))^T mu,   F = d f / d Gamma.
__global__ void k_add(int n, const double *a, double *y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] += a[i];
}
__global__ void k_axpby(int n, double a, const double *x, double b, const double *y, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a * x[i] + b * y[i];
}

}  // namespace ptrom

extern "C" size_t fom_adjoint_workspace_bytes(const ptrom_fom_params *p, int n) {
    if (!p) return 0;
    ptrom_fom_params q = *p;
    q.jac_mode = PTROM_JAC_JFNK;
    if (validate(&q, n) != PTROM_OK) return 0;
    return layout(&q, n, nullptr).bytes + ((size_t)n * 8 + 255) / 256 * 256;
}

extern "C" int fom_adjoint_step(const ptrom_fom_params *p, int n, const double *Gamma, const double *x_n,
                                const double *x_prev, double *lambda, double *gGamma, void *work,
                                size_t work_bytes, ptrom_fom_stats *stats, ptrom_stream_t stream) {
    using namespace ptrom;
    if (!p) return set_error(PTROM_EINVAL, "fom_adjoint_step: NULL params");
    ptrom_fom_params q = *p;
    q.jac_mode = PTROM_JAC_JFNK;
    PTROM_TRY(validate(&q, n));
    if (!Gamma || !x_n || !x_prev || !lambda || !gGamma || !work)
        return set_error(PTROM_EINVAL, "fom_adjoint_step: NULL pointer");
    if (((uintptr_t)work) & 255) return set_error(PTROM_EINVAL, "fom_adjoint_step: work must be 256-byte aligned");
    Ctx c{};
    c.transpose = 1;
    c.p = &q;
    c.n = n;
    c.n2 = 2 * n;
    c.G = Gamma;
    c.xi = x_n;
    c.hdt = 0.5 * q.dt;
    c.st = (cudaStream_t)stream;
    c.W = layout(&q, n, (char *)work);
    const size_t need = c.W.bytes + ((size_t)n * 8 + 255) / 256 * 256;
    if (work_bytes < need)
        return set_error(PTROM_EINVAL, "fom_adjoint_step: work has %zu bytes, needs %zu", work_bytes, need);
    double *gtmp = (double *)((char *)work + c.W.bytes);
    c.grid = (c.n2 + 255) / 256;
    if (c.grid > 4 * device_sm_count()) c.grid = 4 * device_sm_count();
    c.rgrid = red_grid(c.n2);
    c.cgrid = coop_grid(n);
    c.coop = coop_fits(c.cgrid, n);
    PTROM_TRY(host_mailbox(kStatSlots * kStatDoubles, kStatSlots, &c.mb, &c.ev));
    ptrom_fom_stats local{};
    c.stats = stats ? stats : &local;
    memset(c.stats, 0, sizeof(*c.stats));
    Work &W = c.W;
    PTROM_CUDA(cudaMemsetAsync(W.counter, 0, 64, c.st));
    PTROM_CUDA(cudaMemsetAsync(W.flags, 0, 64, c.st));
    // self blocks at x^n for the (transposed) preconditioner
    LaunchOpts po;
    po.scratch = W.pack;
    po.scratch_bytes = W.pack_bytes;
    PTROM_TRY(velocity(n, x_n, n, x_n, Gamma, q.delta, W.fxi, W.D, q.prec, c.st, po));
    c.stats->velocity_evals++;
    k_minv<<<c.grid, 256, 0, c.st>>>(n, W.D, c.hdt, W.Mi);
    count_launch();
    // mu = (I - h J_n)^{-T} lambda  (mu = 0 when lambda = 0)
    PTROM_CUDA(cudaMemsetAsync(W.d, 0, sizeof(double) * c.n2, c.st));
    k_multidot<<<c.rgrid, kRedThreads, 0, c.st>>>(c.n2, 1, nullptr, lambda, mkred(W, 0));
    count_launch();
    double l2 = 0.0;
    PTROM_TRY(fetch(c, W.redout, &l2, 1));
    if (l2 > 0.0) PTROM_TRY(gmres(c, lambda, 1.0, W.d, nullptr, W.redout));
    // gGamma += h F_n^T mu
    PTROM_TRY(vjp(n, x_n, Gamma, q.delta, W.d, nullptr, gtmp, q.prec, c.st, po));
    k_axpy<<<c.grid, 256, 0, c.st>>>(n, c.hdt, gtmp, gGamma);
    count_launch();
    // lambda_prev = mu + h J_{n-1}^T mu ;  gGamma += h F_{n-1}^T mu
    PTROM_TRY(vjp(n, x_prev, Gamma, q.delta, W.d, W.jz, gtmp, q.prec, c.st, po));
    c.stats->jvp_evals += 2;
    k_axpby<<<c.grid, 256, 0, c.st>>>(c.n2, 1.0, W.d, c.hdt, W.jz, lambda);
    k_axpy<<<c.grid, 256, 0, c.st>>>(n, c.hdt, gtmp, gGamma);
    count_launch(2);
    PTROM_CUDA(cudaGetLastError());
    return PTROM_OK;
}


// ---------------------------------------------------------------- batched FOM
namespace ptrom {
struct BInst {
    int n;
    double *x, *xprev, *fxi, *fprev, *r, *D;
    Red red;
    double *norm_out;  // [2]
};

__global__ void k_residual_batched(const BInst *__restrict__ I, double hdt) {
    const BInst b = I[blockIdx.y];
    __shared__ double sh[32];
    const int n2 = 2 * b.n;
    double s0 = 0.0, s1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
        const double v = b.x[i] - b.xprev[i] - hdt * (b.fxi[i] + b.fprev[i]);
        b.r[i] = v;
        s0 += v * v;
        s1 += b.x[i] * b.x[i];
    }
    const double t0 = block_sum(s0, sh);
    const double t1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        b.red.partials[blockIdx.x * 2 + 0] = t0;
        b.red.partials[blockIdx.x * 2 + 1] = t1;
    }
    Red rr = b.red;
    rr.out = b.norm_out;
    finish_reduction(rr, 2);
}

__global__ void k_blockdiag_batched(const BInst *__restrict__ I, double hdt) {
    const BInst b = I[blockIdx.y];
    const int n = b.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d00 = b.D[i], d01 = b.D[n + i], d10 = b.D[2 * n + i], d11 = -d00;
        const double m00 = 1.0 - hdt * d00, m01 = -hdt * d01, m10 = -hdt * d10, m11 = 1.0 - hdt * d11;
        const double det = m00 * m11 - m01 * m10;
        const double r0 = b.r[i], r1 = b.r[n + i];
        b.x[i] -= (m11 * r0 - m01 * r1) / det;
        b.x[n + i] -= (m00 * r1 - m10 * r0) / det;
    }
}
}  // namespace ptrom

extern "C" int fom_step_batched(const ptrom_fom_params *p, int B, const int *n, const double *const *Gamma,
                                double *const *x, double *const *f, void *const *work, const size_t *work_bytes,
                                ptrom_fom_stats *stats, ptrom_stream_t stream) {
    using namespace ptrom;
    if (!p || B < 1 || !n || !Gamma || !x || !f || !work || !work_bytes)
        return set_error(PTROM_EINVAL, "fom_step_batched: bad arguments");
    if (p->jac_mode != PTROM_JAC_BLOCKDIAG)
        return set_error(PTROM_EINVAL, "fom_step_batched: only the block-diagonal (inexact) Jacobian is batched");
    if (p->u_inf) return set_error(PTROM_EINVAL, "fom_step_batched: u_inf must be NULL (one inflow per instance)");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<Work> W(B);
    for (int b = 0; b < B; ++b) {
        PTROM_TRY(validate(p, n[b]));
        if (!Gamma[b] || !x[b] || !f[b] || !work[b] || (((uintptr_t)work[b]) & 255))
            return set_error(PTROM_EINVAL, "fom_step_batched: bad instance %d", b);
        W[b] = layout(p, n[b], (char *)work[b]);
        if (work_bytes[b] < W[b].bytes) return set_error(PTROM_EINVAL, "fom_step_batched: work %d too small", b);
        PTROM_CUDA(cudaMemsetAsync(W[b].counter, 0, 64, st));
        PTROM_CUDA(cudaMemcpyAsync(W[b].xprev, x[b], sizeof(double) * 2 * n[b], cudaMemcpyDeviceToDevice, st));
        PTROM_CUDA(cudaMemcpyAsync(W[b].fprev, f[b], sizeof(double) * 2 * n[b], cudaMemcpyDeviceToDevice, st));
        if (stats) memset(&stats[b], 0, sizeof(ptrom_fom_stats));
    }
    const double hdt = 0.5 * p->dt;
    int maxn = 0;
    for (int b = 0; b < B; ++b) maxn = std::max(maxn, n[b]);
    const int rg = std::min(red_grid(2 * maxn), 2 * device_sm_count());
    BInst *dinst = nullptr;
    double *dnorm = nullptr;
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&dinst, sizeof(BInst) * B));
    PTROM_TRY(sc.alloc(&dnorm, sizeof(double) * 2 * B));
    std::vector<int> active(B);
    for (int b = 0; b < B; ++b) active[b] = b;
    std::vector<double> norms(2 * B);
    int status = PTROM_OK;
    for (int k = 0; k <= p->max_iter && !active.empty(); ++k) {
        const int A = (int)active.size();
        std::vector<int> an(A);
        std::vector<const double *> ax(A), aG(A);
        std::vector<double> ad(A);
        std::vector<double *> af(A), aD(A);
        std::vector<BInst> hi(A);
        for (int a = 0; a < A; ++a) {
            const int b = active[a];
            an[a] = n[b];
            ax[a] = x[b];
            aG[a] = Gamma[b];
            ad[a] = p->delta;
            af[a] = W[b].fxi;
            aD[a] = W[b].D;
            hi[a] = BInst{n[b], x[b], W[b].xprev, W[b].fxi, W[b].fprev, W[b].r, W[b].D,
                          Red{W[b].partials, W[b].counter, W[b].redout}, dnorm + 2 * a};
            if (stats) stats[b].velocity_evals++;
        }
        PTROM_TRY(velocity_batched(A, an.data(), ax.data(), aG.data(), ad.data(), af.data(), aD.data(), p->prec, st, 2));
        PTROM_CUDA(cudaMemcpyAsync(dinst, hi.data(), sizeof(BInst) * A, cudaMemcpyHostToDevice, st));
        k_residual_batched<<<dim3(rg, A), kRedThreads, 0, st>>>(dinst, hdt);
        count_launch();
        PTROM_CUDA(cudaMemcpyAsync(norms.data(), dnorm, sizeof(double) * 2 * A, cudaMemcpyDeviceToHost, st));
        PTROM_CUDA(cudaStreamSynchronize(st));
        std::vector<int> next;
        std::vector<BInst> upd;
        for (int a = 0; a < A; ++a) {
            const int b = active[a];
            const double rn = sqrt(norms[2 * a]), xn = sqrt(norms[2 * a + 1]);
            if (stats) {
                if (k == 0) stats[b].res_norm0 = rn;
                stats[b].res_norm = rn;
            }
            if (!isfinite(rn)) {
                status = set_error(PTROM_ENAN, "fom_step_batched: non-finite residual in instance %d", b);
                PTROM_CUDA(cudaMemcpyAsync(f[b], W[b].fxi, sizeof(double) * 2 * n[b], cudaMemcpyDeviceToDevice, st));
                continue;
            }
            const bool conv = rn <= p->tol * (xn > 1.0 ? xn : 1.0);
            if (conv || k == p->max_iter) {
                PTROM_CUDA(cudaMemcpyAsync(f[b], W[b].fxi, sizeof(double) * 2 * n[b], cudaMemcpyDeviceToDevice, st));
                if (!conv && status == PTROM_OK)
                    status = set_error(PTROM_ENOCONV, "fom_step_batched: instance %d did not converge", b);
                continue;
            }
            if (stats) stats[b].newton_iters++;
            next.push_back(b);
            upd.push_back(hi[a]);
        }
        if (!upd.empty()) {
            PTROM_CUDA(cudaMemcpyAsync(dinst, upd.data(), sizeof(BInst) * upd.size(), cudaMemcpyHostToDevice, st));
            k_blockdiag_batched<<<dim3(std::min(4 * device_sm_count(), (maxn + 255) / 256), (int)upd.size()), 256, 0, st>>>(
                dinst, hdt);
            count_launch();
            PTROM_CUDA(cudaGetLastError());
        }
        active.swap(next);
    }
    PTROM_TRY(sc.release());
    PTROM_CUDA(cudaStreamSynchronize(st));
    return status;
}

extern "C" int fom_steps(const ptrom_fom_params *p, int n, const double *Gamma, double *x, double *f, void *work,
                         size_t work_bytes, int nsteps, int iters, ptrom_fom_stats *stats, int *steps_done,
                         ptrom_stream_t stream) {
    if (steps_done) *steps_done = 0;
    if (!p) return set_error(PTROM_EINVAL, "fom_steps: NULL params");
    if (p->jac_mode != PTROM_JAC_BLOCKDIAG)
        return set_error(PTROM_EINVAL, "fom_steps: graph-captured steps take the block-diagonal Newton only");
    if (nsteps < 1 || iters < 0 || iters > p->max_iter + 1)
        return set_error(PTROM_EINVAL, "fom_steps: nsteps=%d must be >= 1 and iters=%d in [0, max_iter + 1]", nsteps,
                         iters);
    Ctx c{};
    PTROM_TRY(init_ctx(c, "fom_steps", p, n, Gamma, x, f, work, work_bytes, stream));
    ptrom_fom_stats total{}, one{};
    int done = 0;
    // iters = 0: the first step, host-driven, tells how many iterations a step takes
    if (iters == 0) {
        PTROM_TRY(fom_step(p, n, Gamma, x, f, work, work_bytes, &one, stream));
        total = one;
        done = 1;
        iters = std::min(one.velocity_evals + 2, p->max_iter + 1);
    }
    if (done < nsteps && (!c.coop || timing_active())) {
        // no cooperative Newton kernel at this size, or launches being timed: step by step
        for (; done < nsteps; ++done) {
            const int e = fom_step(p, n, Gamma, x, f, work, work_bytes, &one, stream);
            total.newton_iters += one.newton_iters;
            total.velocity_evals += one.velocity_evals;
            total.res_norm = one.res_norm;
            if (e != PTROM_OK) {
                if (stats) *stats = total;
                if (steps_done) *steps_done = done;
                return e;
            }
        }
    }
    if (done < nsteps) {
        Work &W = c.W;
        const int todo = nsteps - done;
        char *rb = nullptr;
        ScratchScope sc(c.st);
        PTROM_TRY(sc.alloc(&rb, 256 + sizeof(double) * 3 * (size_t)todo));
        double *itersp = (double *)rb, *log = (double *)(rb + 256);
        int *stepp = (int *)(rb + 8);
        PTROM_CUDA(cudaMemsetAsync(rb, 0, 256, c.st));
        PTROM_CUDA(cudaMemsetAsync(W.flags, 0, 64, c.st));
        // capture one step on a private stream (the caller's may be the legacy
        // default stream, which cannot be captured) and replay it on theirs
        cudaStream_t cs = nullptr;
        PTROM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        int kernels = 2;
        int status = PTROM_OK;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            Ctx cc = c;
            cc.st = cs;
            k_roll_begin<<<1, 1, 0, cs>>>(W.flags, itersp);
            for (int k = 0; k < iters && status == PTROM_OK; ++k) {
                const bool refresh = k % p->p_it == 0;
                LaunchOpts vo;
                vo.scratch = W.pack;
                vo.scratch_bytes = W.pack_bytes;
                vo.skip = W.flags;
                status = velocity(n, x, n, x, Gamma, p->delta, W.fxi, refresh ? W.D : nullptr, p->prec, cs, vo);
                NewtonArgs na{n, x, W.xprev, W.fxi, f, p->u_inf, cc.hdt, W.r, W.partials, W.redout, p->tol,
                              k == p->max_iter, W.flags, W.stat, refresh ? 1 : 0, W.D, W.Mi, 1, W.V, W.z,
                              k == 0 ? 1 : 0, f, W.d, W.counter, W.flags, itersp};
                void *args[] = {&na};
                if (status == PTROM_OK) {
                    const cudaError_t el = cudaLaunchCooperativeKernel((void *)k_newton, dim3(cc.cgrid),
                                                                      dim3(kRedThreads), args, 0, cs);
                    if (el != cudaSuccess) status = check_cuda(el, "fom_steps: Newton kernel capture");
                }
                kernels += 3;
            }
            k_roll_end<<<1, 1, 0, cs>>>(W.flags, W.stat, itersp, log, stepp);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess && status == PTROM_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        for (int s2 = 0; e == cudaSuccess && status == PTROM_OK && s2 < todo; ++s2) e = cudaGraphLaunch(exec, c.st);
        if (e == cudaSuccess && status == PTROM_OK) count_launch(kernels * todo);
        std::vector<double> hlog(3 * (size_t)todo);
        int nd = 0;
        if (e == cudaSuccess && status == PTROM_OK) e = cudaMemcpyAsync(&nd, stepp, sizeof(int), cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess && status == PTROM_OK)
            e = cudaMemcpyAsync(hlog.data(), log, sizeof(double) * hlog.size(), cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess && status == PTROM_OK) e = cudaStreamSynchronize(c.st);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (status != PTROM_OK) return status;
        if (e != cudaSuccess) return check_cuda(e, "fom_steps: graph");
        PTROM_TRY(sc.release());
        for (int s2 = 0; s2 < nd; ++s2) {
            const int it = (int)hlog[3 * s2 + 2];
            total.velocity_evals += it;
            total.newton_iters += hlog[3 * s2] == 1.0 ? it - 1 : it;
            total.res_norm = hlog[3 * s2 + 1];
        }
        const int ok = (nd > 0 && hlog[3 * (nd - 1)] != 1.0) ? nd - 1 : nd;
        done += ok;
        if (stats) *stats = total;
        if (steps_done) *steps_done = done;
        if (ok < todo) {
            const double stop = nd > 0 ? hlog[3 * (nd - 1)] : 0.0;
            if (stop == 2.0) return set_error(PTROM_ENAN, "fom_steps: non-finite residual in step %d", done);
            return set_error(PTROM_ENOCONV, "fom_steps: step %d did not converge in %d captured Newton iterations "
                                            "(|r| = %.3e)", done, iters, total.res_norm);
        }
        return PTROM_OK;
    }
    if (stats) *stats = total;
    if (steps_done) *steps_done = done;
    return PTROM_OK;
}

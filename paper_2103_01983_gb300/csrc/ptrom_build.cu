// Offline PTROM training (Sec. 5.1, Stages 1-4) -- ptrom_build,
// ptrom_set_param_full, ptrom_reconstruct, ptrom_model_query.
//
// GPU: FOM training runs (fom_step), the FP64 snapshot Gram matrix and basis
// products, and Tier-II LSPG over all bodies (cluster gather, warp-per-body
// pair sums with the residual, normal equations of the Gauss-Newton least
// squares), the symmetric eigen-solve of the Gram or covariance matrix
// (cuSOLVER syevd).  Host C++: the quadtree over the weighted POD space with WeightedMean,
// FindClusters/checkPrune and UniqueSearch (Alg. 2/3), the greedy sampling
// (Alg. 1) and the gappy pseudo-inverse; their sizes are O(N) or tiny.
#include <math.h>
#include <string.h>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <random>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "ptrom_model.h"
#include "scratch.h"

namespace ptrom {
namespace {

using Clock = std::chrono::steady_clock;
double secs(Clock::time_point a) { return std::chrono::duration<double>(Clock::now() - a).count(); }


// ------------------------------------------------------------------ host dense algebra
// Eigen-decomposition of a symmetric n x n matrix (row-major) by cyclic
// Jacobi rotations; eigenvalues descending, eigenvectors as columns of V.
void jacobi_eig(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double total = 0.0;
    for (double v : A) total += v * v;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-30 * total || off == 0.0) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
    std::vector<double> V2((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[(size_t)ord[j] * n + ord[j]];
        for (int k = 0; k < n; ++k) V2[(size_t)k * n + j] = V[(size_t)k * n + ord[j]];
    }
    V.swap(V2);
}

// Least squares X = argmin ||A X - B|| by Householder QR (A: m x n col-major,
// m >= n, full column rank; B: m x k col-major); X: n x k col-major.
bool lstsq_qr(int m, int n, std::vector<double> A, std::vector<double> B, int k, std::vector<double> &X) {
    if (m < n) return false;
    std::vector<double> diag(n);
    for (int j = 0; j < n; ++j) {
        double *cj = &A[(size_t)j * m];
        double s = 0.0;
        for (int i = j; i < m; ++i) s += cj[i] * cj[i];
        const double nrm = sqrt(s);
        if (nrm == 0.0) return false;
        const double alpha = cj[j] >= 0 ? -nrm : nrm;
        const double v0 = cj[j] - alpha;
        const double vn2 = s - cj[j] * cj[j] + v0 * v0;
        cj[j] = v0;
        const double tau = vn2 > 0 ? 2.0 / vn2 : 0.0;
        for (int c = j + 1; c < n + k; ++c) {
            double *col = c < n ? &A[(size_t)c * m] : &B[(size_t)(c - n) * m];
            double w = 0.0;
            for (int i = j; i < m; ++i) w += cj[i] * col[i];
            w *= tau;
            for (int i = j; i < m; ++i) col[i] -= w * cj[i];
        }
        diag[j] = alpha;
    }
    X.assign((size_t)n * k, 0.0);
    for (int c = 0; c < k; ++c) {
        for (int j = n - 1; j >= 0; --j) {
            double s = B[(size_t)c * m + j];
            for (int q = j + 1; q < n; ++q) s -= A[(size_t)q * m + j] * X[(size_t)c * n + q];
            X[(size_t)c * n + j] = s / diag[j];
        }
    }
    return true;
}

// Minimum-norm least squares X = argmin ||X|| over argmin ||A X - B|| (the
// Moore-Penrose solution A^+ B) for any shape and rank (A: m x n col-major,
// B: m x k col-major; X: n x k col-major).  A well-conditioned full-column-rank
// A (m >= n) takes the Householder QR above, whose solution is then the unique
// one; otherwise A's SVD is formed by one-sided Jacobi rotations (Hestenes:
// rotate pairs of columns of A V until they are orthogonal, so A V = U Sigma),
// and X = V Sigma^+ U^T B keeps the singular values above
// max(m, n) * eps * sigma_max, the rank threshold of LAPACK-style least
// squares drivers.
void lstsq_minnorm(int m, int n, const std::vector<double> &A, const std::vector<double> &B, int k,
                   std::vector<double> &X) {
    if (m >= n) {
        // QR fast path, taken only when the diagonal of R shows a well-conditioned A
        bool ok = true;
        double dmax = 0.0, dmin = INFINITY;
        {
            std::vector<double> T = A;
            for (int j = 0; j < n && ok; ++j) {
                double *cj = &T[(size_t)j * m];
                double s2 = 0.0;
                for (int i = j; i < m; ++i) s2 += cj[i] * cj[i];
                const double nrm = sqrt(s2);
                dmax = std::max(dmax, nrm);
                dmin = std::min(dmin, nrm);
                if (nrm == 0.0) {
                    ok = false;
                    break;
                }
                const double alpha = cj[j] >= 0 ? -nrm : nrm;
                const double v0 = cj[j] - alpha;
                const double vn2 = s2 - cj[j] * cj[j] + v0 * v0;
                cj[j] = v0;
                const double tau = vn2 > 0 ? 2.0 / vn2 : 0.0;
                for (int c = j + 1; c < n; ++c) {
                    double *col = &T[(size_t)c * m];
                    double w = 0.0;
                    for (int i = j; i < m; ++i) w += cj[i] * col[i];
                    w *= tau;
                    for (int i = j; i < m; ++i) col[i] -= w * cj[i];
                }
            }
        }
        if (ok && dmin > 1e-7 * dmax && lstsq_qr(m, n, A, B, k, X)) return;
    }
    // one-sided Jacobi SVD of A (m x n): columns of U S in Us, V (n x n)
    std::vector<double> Us = A, V((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = 1.0;
    const double eps = 2.220446049250313e-16;
    for (int sweep = 0; sweep < 60; ++sweep) {
        bool rotated = false;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *up = &Us[(size_t)p * m], *uq = &Us[(size_t)q * m];
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < m; ++i) {
                    alpha += up[i] * up[i];
                    beta += uq[i] * uq[i];
                    gamma += up[i] * uq[i];
                }
                if (gamma == 0.0 || fabs(gamma) <= eps * sqrt(alpha * beta)) continue;
                rotated = true;
                const double zeta = (beta - alpha) / (2.0 * gamma);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < m; ++i) {
                    const double a = up[i], b = uq[i];
                    up[i] = c * a - s * b;
                    uq[i] = s * a + c * b;
                }
                double *vp = &V[(size_t)p * n], *vq = &V[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    const double a = vp[i], b = vq[i];
                    vp[i] = c * a - s * b;
                    vq[i] = s * a + c * b;
                }
            }
        }
        if (!rotated) break;
    }
    std::vector<double> sv(n);
    double smax = 0.0;
    for (int j = 0; j < n; ++j) {
        double s2 = 0.0;
        for (int i = 0; i < m; ++i) s2 += Us[(size_t)j * m + i] * Us[(size_t)j * m + i];
        sv[j] = sqrt(s2);
        smax = std::max(smax, sv[j]);
    }
    const double cut = (double)std::max(m, n) * eps * smax;
    X.assign((size_t)n * k, 0.0);
    for (int j = 0; j < n; ++j) {
        if (!(sv[j] > cut)) continue;
        const double inv2 = 1.0 / (sv[j] * sv[j]);  // (U S)_j^T b / s_j^2 = U_j^T b / s_j
        for (int c = 0; c < k; ++c) {
            double w = 0.0;
            for (int i = 0; i < m; ++i) w += Us[(size_t)j * m + i] * B[(size_t)c * m + i];
            w *= inv2;
            for (int i = 0; i < n; ++i) X[(size_t)c * n + i] += w * V[(size_t)j * n + i];
        }
    }
}

// Cholesky solve of G x = b (G n x n row-major, SPD); b is overwritten by x.
bool chol_solve(int n, std::vector<double> G, std::vector<double> &b) {
    for (int j = 0; j < n; ++j) {
        double d = G[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= G[(size_t)j * n + k] * G[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        d = sqrt(d);
        G[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = G[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= G[(size_t)i * n + k] * G[(size_t)j * n + k];
            G[(size_t)i * n + j] = s / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= G[(size_t)i * n + k] * b[k];
        b[i] = s / G[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= G[(size_t)k * n + i] * b[k];
        b[i] = s / G[(size_t)i * n + i];
    }
    return true;
}

// ------------------------------------------------------------------ GPU kernels
// G = S^T S (K x K) for S (nd x K, column-major), FP64; 32 x 32 output tile per block.
__global__ void k_gram(int nd, int K, const double *__restrict__ S, double *__restrict__ G) {
    __shared__ double ta[32][33], tb[32][33];
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
    if (b0 < a0) return;  // upper triangle only (mirrored on the host)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    double acc[4] = {0, 0, 0, 0};
    for (int r0 = 0; r0 < nd; r0 += 32) {
        for (int q = ty; q < 32; q += 8) {
            const int row = r0 + tx;
            ta[q][tx] = (row < nd && a0 + q < K) ? S[(size_t)(a0 + q) * nd + row] : 0.0;
            tb[q][tx] = (row < nd && b0 + q < K) ? S[(size_t)(b0 + q) * nd + row] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            const double bv = tb[tx][rr];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += ta[ty + 8 * u][rr] * bv;
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u) {
        const int a = a0 + ty + 8 * u, b = b0 + tx;
        if (a < K && b < K) G[(size_t)a * K + b] = acc[u];
    }
}

// Phi[d][m] = sum_k S[d][k] W[k][m]   (S nd x K column-major, W K x M row-major)
__global__ void k_combine(int nd, int K, int M, const double *__restrict__ S, const double *__restrict__ W,
                          double *__restrict__ Phi) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    for (int m = 0; m < M; ++m) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += S[(size_t)k * nd + d] * W[(size_t)k * M + m];
        Phi[(size_t)d * M + m] = s;
    }
}

// one snapshot column: the state x^n itself (Sec. 3.1)
__global__ void k_snapshot(int nd, const double *x, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x) out[i] = x[i];
}

struct T2 {
    int n, Nc, M, Mp;
    float h, delta;
    const float *phi;   // [2n][Mp]   all bodies
    const float *x0;    // [2n]       relative to origin
    const float *phic;  // [2Nc][Mp]
    const float *x0c;   // [2Nc]
    const float *gc;    // [Nc]
    const int *off, *idx;
    const float *u;     // [2n]       dt times the superimposed inflow (Sec. 6.3), zeros for none
};

// rows < 2n: xt = x0 + Phi xh and pd = Phi dxh; rows >= 2n: xq = x0c + Phic xh
__global__ void k_t2_gather(T2 t, const float *xh, const float *dxh, float *xt, float *pd, float *xq) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int nb = 2 * t.n;
    if (row >= nb + 2 * t.Nc) return;
    if (row < nb) {
        const float *ph = t.phi + (size_t)row * t.Mp;
        float a = t.x0[row], b = 0.f;
        for (int k = 0; k < t.M; ++k) {
            a = fmaf(ph[k], xh[k], a);
            b = fmaf(ph[k], dxh[k], b);
        }
        xt[row] = a;
        pd[row] = b;
    } else {
        const int rr = row - nb;
        const float *ph = t.phic + (size_t)rr * t.Mp;
        float a = t.x0c[rr];
        for (int k = 0; k < t.M; ++k) a = fmaf(ph[k], xh[k], a);
        xq[rr] = a;
    }
}

// warp per body: f, D and r = pd - h (f + fprev); r also written (FP64) to a snapshot column
__global__ void k_t2_pairs(T2 t, const float *xt, const float *xq, const float *pd, const float *fprev, float *f,
                           float *D, float *r, double *rcol) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= t.n) return;
    const float tx = xt[i], ty = xt[t.n + i];
    float u = 0.f, v = 0.f, d00 = 0.f, d01 = 0.f, d10n = 0.f;
    for (int e = t.off[i] + lane; e < t.off[i + 1]; e += 32) {
        const int c = t.idx[e];
        const float a = tx - xq[c], b = ty - xq[t.Nc + c];
        const float d2 = fmaf(a, a, b * b);
        float rr = 1.0f / (d2 + t.delta);
        rr = (d2 == 0.f) ? 0.f : rr;
        const float q = t.gc[c] * rr;
        u = fmaf(q, b, u);
        v = fmaf(q, a, v);
        const float p2 = 2.f * q * rr;
        d00 = fmaf(p2 * a, b, d00);
        d01 += fmaf(p2 * b, b, -q);
        d10n += fmaf(p2 * a, a, -q);
    }
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_xor_sync(0xffffffffu, u, o);
        v += __shfl_xor_sync(0xffffffffu, v, o);
        d00 += __shfl_xor_sync(0xffffffffu, d00, o);
        d01 += __shfl_xor_sync(0xffffffffu, d01, o);
        d10n += __shfl_xor_sync(0xffffffffu, d10n, o);
    }
    if (lane == 0) {
        f[i] = -u;
        f[t.n + i] = v;
        D[i] = d00;
        D[t.n + i] = d01;
        D[2 * t.n + i] = -d10n;
        const float r0 = pd[i] - t.h * (-u + fprev[i]) - t.u[i];
        const float r1 = pd[t.n + i] - t.h * (v + fprev[t.n + i]) - t.u[t.n + i];
        r[i] = r0;
        r[t.n + i] = r1;
        if (rcol) {
            rcol[i] = r0;
            rcol[t.n + i] = r1;
        }
    }
}

// Normal equations of min ||C nu + r||, C = (I - h blockdiag D) Phi:
// per block of 64 bodies, FP32 partials of C^T C (M x M) and C^T r (M).
constexpr int kT2Bodies = 64;
__global__ void k_t2_normal(T2 t, const float *D, const float *r, float *part) {
    extern __shared__ float sc[];  // [2*kT2Bodies][Mp] C rows, then [2*kT2Bodies] r
    float *rs = sc + 2 * kT2Bodies * t.Mp;
    const int i0 = blockIdx.x * kT2Bodies;
    const int nbod = min(kT2Bodies, t.n - i0);
    for (int e = threadIdx.x; e < 2 * kT2Bodies * t.Mp; e += blockDim.x) {
        const int slot = e / t.Mp, k = e % t.Mp, j = slot >> 1;
        float val = 0.f;
        if (j < nbod && k < t.M) {
            const int i = i0 + j;
            const float pc = t.phi[(size_t)i * t.Mp + k], pp = t.phi[(size_t)(t.n + i) * t.Mp + k];
            const float d00 = D[i], d01 = D[t.n + i], d10 = D[2 * t.n + i];
            val = (slot & 1) ? pp - t.h * (d10 * pc - d00 * pp) : pc - t.h * (d00 * pc + d01 * pp);
        }
        sc[e] = val;
    }
    for (int s = threadIdx.x; s < 2 * kT2Bodies; s += blockDim.x) {
        const int j = s >> 1;
        rs[s] = j < nbod ? ((s & 1) ? r[t.n + i0 + j] : r[i0 + j]) : 0.f;
    }
    __syncthreads();
    const int nout = t.M * t.M + t.M;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        float acc = 0.f;
        if (o < t.M * t.M) {
            const int a = o / t.M, b = o % t.M;
            for (int s = 0; s < 2 * kT2Bodies; ++s) acc = fmaf(sc[s * t.Mp + a], sc[s * t.Mp + b], acc);
        } else {
            const int a = o - t.M * t.M;
            for (int s = 0; s < 2 * kT2Bodies; ++s) acc = fmaf(sc[s * t.Mp + a], rs[s], acc);
        }
        part[(size_t)blockIdx.x * nout + o] = acc;
    }
}

// FP64 sum of the block partials (fixed order)
__global__ void k_t2_reduce(int nblocks, int nout, const float *part, double *out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += (double)part[(size_t)b * nout + o];
    out[o] = s;
}

__global__ void k_reconstruct(int n, int M, const double *phi, const double *x0, const double *xh, const int *rows,
                              int nrows, double *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * nrows) return;
    const int j = e < nrows ? e : e - nrows;
    const int body = rows[j];
    const int row = e < nrows ? body : n + body;
    double s = x0[row];
    for (int k = 0; k < M; ++k) s += phi[(size_t)row * M + k] * xh[k];
    out[e] = s;
}

// ------------------------------------------------------------------ quadtree (host)
struct QNode {
    double box[4];   // xmin, xmax, ymin, ymax
    int first, count;
    int child[4], nchild;
    int depth, canon;
    double cen[2];
};

struct QTree {
    std::vector<QNode> nodes;
    std::vector<int> perm, pos, leaf_of;
    const double *P;  // [n][2]
    int build(int first, int count, const double box[4], int depth) {
        const int id = (int)nodes.size();
        nodes.push_back(QNode{});
        QNode nd{};
        memcpy(nd.box, box, sizeof nd.box);
        nd.first = first;
        nd.count = count;
        nd.depth = depth;
        nd.nchild = 0;
        nodes[id] = nd;
        if (count <= 1 || depth >= 40) {
            for (int k = 0; k < count; ++k) leaf_of[perm[first + k]] = id;
            return id;
        }
        const double xm = 0.5 * (box[0] + box[1]), ym = 0.5 * (box[2] + box[3]);
        std::vector<int> q[4];
        for (int k = 0; k < count; ++k) {
            const int b = perm[first + k];
            q[(P[2 * b] >= xm ? 1 : 0) + (P[2 * b + 1] >= ym ? 2 : 0)].push_back(b);
        }
        int at = first;
        int starts[4];
        for (int c = 0; c < 4; ++c) {
            starts[c] = at;
            for (int b : q[c]) perm[at++] = b;
        }
        const double boxes[4][4] = {{box[0], xm, box[2], ym}, {xm, box[1], box[2], ym},
                                    {box[0], xm, ym, box[3]}, {xm, box[1], ym, box[3]}};
        for (int c = 0; c < 4; ++c) {
            if (q[c].empty()) continue;
            const int ch = build(starts[c], (int)q[c].size(), boxes[c], depth + 1);
            QNode &me = nodes[id];
            me.child[me.nchild++] = ch;
        }
        return id;
    }
    void make(const double *pts, int n) {
        P = pts;
        perm.resize(n);
        pos.resize(n);
        leaf_of.assign(n, -1);
        for (int i = 0; i < n; ++i) perm[i] = i;
        double lo[2] = {pts[0], pts[1]}, hi[2] = {pts[0], pts[1]};
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 2; ++a) {
                lo[a] = std::min(lo[a], pts[2 * i + a]);
                hi[a] = std::max(hi[a], pts[2 * i + a]);
            }
        double side = std::max(hi[0] - lo[0], hi[1] - lo[1]);
        if (side == 0.0) side = 1.0;
        const double box[4] = {lo[0], lo[0] + side, lo[1], lo[1] + side};
        nodes.reserve(4 * (size_t)n);
        build(0, n, box, 0);
        for (int k = 0; k < n; ++k) pos[perm[k]] = k;
        for (int id = (int)nodes.size() - 1; id >= 0; --id) {  // children after parents
            QNode &nd = nodes[id];
            nd.canon = nd.nchild == 1 ? nodes[nd.child[0]].canon : id;
        }
    }
    double width(int id) const {
        const QNode &n = nodes[id];
        return std::max(n.box[1] - n.box[0], n.box[3] - n.box[2]);
    }
};

struct ClusterSet {
    std::vector<int> off, idx;     // per target CSR of cluster indices
    std::vector<long long> keys;   // per cluster: canonical key
    std::unordered_map<long long, int> index;
};

// Alg. 2 FindClusters/Traverse with Alg. 3 checkPrune for one target.
void find_clusters(const QTree &T, const std::vector<double> &pts, const std::vector<double> &cen, int i,
                   int criterion, double theta, double p_c, std::vector<long long> &out) {
    out.clear();
    const QNode &leaf = T.nodes[T.leaf_of[i]];
    const double wt = std::max(leaf.box[1] - leaf.box[0], leaf.box[3] - leaf.box[2]);
    const double H[4] = {leaf.box[0] - p_c * wt, leaf.box[1] + p_c * wt, leaf.box[2] - p_c * wt, leaf.box[3] + p_c * wt};
    const int nnodes = (int)T.nodes.size();
    std::vector<int> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const int id = stack.back();
        stack.pop_back();
        const QNode &nd = T.nodes[id];
        const bool contains = T.pos[i] >= nd.first && T.pos[i] < nd.first + nd.count;
        bool prune = false;
        if (!contains) {
            if (criterion == PTROM_BARNES_HUT) {
                const double dx = cen[2 * id] - pts[2 * i], dy = cen[2 * id + 1] - pts[2 * i + 1];
                const double d = sqrt(dx * dx + dy * dy);
                prune = d > 0.0 && T.width(id) / d <= theta;
            } else {
                const bool ox = H[1] > nd.box[0] && H[0] < nd.box[1];
                const bool oy = H[3] > nd.box[2] && H[2] < nd.box[3];
                prune = !(ox && oy);
            }
        }
        if (prune) {
            if (nd.count == 1) {
                const int b = T.perm[nd.first];
                const int lf = T.leaf_of[b];
                out.push_back(T.nodes[lf].count == 1 ? lf : (long long)nnodes + b);
            } else {
                out.push_back(nd.canon);
            }
            continue;
        }
        if (nd.nchild == 0) {
            for (int k = 0; k < nd.count; ++k) {
                const int b = T.perm[nd.first + k];
                if (b == i) continue;
                out.push_back(nd.count == 1 ? id : (long long)nnodes + b);
            }
        } else {
            for (int c = nd.nchild - 1; c >= 0; --c) stack.push_back(nd.child[c]);
        }
    }
}

// Members of a cluster key.
void key_members(const QTree &T, long long key, std::vector<int> &mem) {
    mem.clear();
    const int nnodes = (int)T.nodes.size();
    if (key >= nnodes) {
        mem.push_back((int)(key - nnodes));
        return;
    }
    const QNode &nd = T.nodes[(int)key];
    for (int k = 0; k < nd.count; ++k) mem.push_back(T.perm[nd.first + k]);
    std::sort(mem.begin(), mem.end());
}

// |Gamma|-weighted means (unweighted when all weights are zero) of rows for a
// member set: Phi~ (2 x M: chi row, psi row), x0_QT (2), Gamma~ (signed sum).
void cluster_values(const std::vector<int> &mem, int n, int M, const double *phi, const double *x0, const double *G,
                    double *phic_chi, double *phic_psi, double *x0c, double *gc) {
    double wsum = 0.0, gsum = 0.0;
    for (int b : mem) {
        wsum += fabs(G[b]);
        gsum += G[b];
    }
    *gc = gsum;
    if (mem.size() == 1) {
        const int b = mem[0];
        for (int k = 0; k < M; ++k) {
            phic_chi[k] = phi[(size_t)b * M + k];
            phic_psi[k] = phi[(size_t)(n + b) * M + k];
        }
        x0c[0] = x0[b];
        x0c[1] = x0[n + b];
        return;
    }
    const bool unw = wsum == 0.0;
    const double W = unw ? (double)mem.size() : wsum;
    for (int k = 0; k < M; ++k) {
        double a = 0.0, c = 0.0;
        for (int b : mem) {
            const double w = unw ? 1.0 : fabs(G[b]);
            a += w * phi[(size_t)b * M + k];
            c += w * phi[(size_t)(n + b) * M + k];
        }
        phic_chi[k] = a / W;
        phic_psi[k] = c / W;
    }
    double a = 0.0, c = 0.0;
    for (int b : mem) {
        const double w = unw ? 1.0 : fabs(G[b]);
        a += w * x0[b];
        c += w * x0[n + b];
    }
    x0c[0] = a / W;
    x0c[1] = c / W;
}

// Covariance C = S S^T (nd x nd, upper triangle) of the nd x K column-major S.
__global__ void k_cov(int nd, int K, const double *__restrict__ S, double *__restrict__ C) {
    __shared__ double ta[32][33], tb[32][33];
    const int a0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
    if (b0 < a0) return;  // upper triangle only (mirrored on the host)
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    double acc[4] = {0, 0, 0, 0};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int q = ty; q < 32; q += 8) {  // rows a0.., b0.. of snapshots k0 + q (coalesced along the rows)
            const int k = k0 + q;
            ta[q][tx] = (k < K && a0 + tx < nd) ? S[(size_t)k * nd + a0 + tx] : 0.0;
            tb[q][tx] = (k < K && b0 + tx < nd) ? S[(size_t)k * nd + b0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 32; ++kk) {
            const double bv = tb[kk][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += ta[kk][ty + 8 * u] * bv;
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u) {
        const int a = a0 + ty + 8 * u, b = b0 + tx;
        if (a < nd && b < nd) C[(size_t)a * nd + b] = acc[u];
    }
}

// ---------------------------------------------------------------- randomized POD
// Above this size of min(nd, K) the POD uses a randomized range finder instead
// of an exact host eigensolve of the Gram or covariance matrix.
std::atomic<int> g_pod_exact_max{2048};

#define PTROM_CUBLAS(call)                                                              \
    do {                                                                                \
        const cublasStatus_t _b = (call);                                               \
        if (_b != CUBLAS_STATUS_SUCCESS)                                                \
            return set_error(PTROM_ECUDA, "%s: cuBLAS status %d", #call, (int)_b);      \
    } while (0)

// A cuBLAS handle per device (created on first use), bound to `st`.
static int cublas_for(cudaStream_t st, cublasHandle_t *out) {
    static std::mutex mu;
    static cublasHandle_t hs[64] = {};
    int dev = 0;
    PTROM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(PTROM_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!hs[dev]) PTROM_CUBLAS(cublasCreate(&hs[dev]));
    PTROM_CUBLAS(cublasSetStream(hs[dev], st));
    *out = hs[dev];
    return PTROM_OK;
}

// A cuSOLVER dense handle per device (created on first use), bound to `st`.
static int cusolver_for(cudaStream_t st, cusolverDnHandle_t *out) {
    static std::mutex mu;
    static cusolverDnHandle_t hs[64] = {};
    int dev = 0;
    PTROM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(PTROM_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!hs[dev] && cusolverDnCreate(&hs[dev]) != CUSOLVER_STATUS_SUCCESS)
        return set_error(PTROM_ECUDA, "cusolverDnCreate failed");
    if (cusolverDnSetStream(hs[dev], st) != CUSOLVER_STATUS_SUCCESS)
        return set_error(PTROM_ECUDA, "cusolverDnSetStream failed");
    *out = hs[dev];
    return PTROM_OK;
}

// Eigen-decomposition of the symmetric n x n host matrix A (row-major, which
// for a symmetric matrix is also its column-major form) by cuSOLVER's
// divide-and-conquer syevd on the GPU, FP64.  On return w holds the
// eigenvalues in descending order and V (n x n, row-major) the eigenvectors as
// columns.  If the library reports a failure to converge, the host cyclic
// Jacobi method above is used instead.
static int sym_eig(cudaStream_t st, int n, const std::vector<double> &A, std::vector<double> &w,
                   std::vector<double> &V) {
    cusolverDnHandle_t h;
    PTROM_TRY(cusolver_for(st, &h));
    int lwork = 0;
    if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, nullptr, n, nullptr,
                                    &lwork) != CUSOLVER_STATUS_SUCCESS)
        return set_error(PTROM_ECUDA, "cusolverDnDsyevd_bufferSize failed (n=%d)", n);
    double *dA = nullptr, *dw = nullptr, *dwork = nullptr;
    int *dinfo = nullptr;
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&dA, sizeof(double) * (size_t)n * n));
    PTROM_TRY(sc.alloc(&dw, sizeof(double) * (size_t)n));
    PTROM_TRY(sc.alloc(&dwork, sizeof(double) * (size_t)std::max(lwork, 1)));
    PTROM_TRY(sc.alloc(&dinfo, sizeof(int)));
    PTROM_CUDA(cudaMemcpyAsync(dA, A.data(), sizeof(double) * (size_t)n * n, cudaMemcpyHostToDevice, st));
    if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, dA, n, dw, dwork, lwork, dinfo) !=
        CUSOLVER_STATUS_SUCCESS)
        return set_error(PTROM_ECUDA, "cusolverDnDsyevd failed (n=%d)", n);
    std::vector<double> ev((size_t)n * n), wa(n);
    int info = 0;
    PTROM_CUDA(cudaMemcpyAsync(ev.data(), dA, sizeof(double) * ev.size(), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaMemcpyAsync(wa.data(), dw, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaMemcpyAsync(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sc.release());
    if (info != 0) {
        jacobi_eig(n, A, w, V);
        return PTROM_OK;
    }
    // syevd: ascending eigenvalues, eigenvector j in column j (column-major)
    w.resize(n);
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        const int src = n - 1 - j;
        w[j] = wa[src];
        for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = ev[(size_t)src * n + i];
    }
    return PTROM_OK;
}

// Orthonormalise the m x r column-major device block A in place (SVQB: with
// A^T A = V L V^T, A <- A V L^{-1/2}), dropping directions whose eigenvalue is
// below 1e-20 of the largest; r may shrink.  T: m x r scratch.
static int svqb(cublasHandle_t h, int m, int &r, double *A, double *T, double *Gd, double *Wd, cudaStream_t st) {
    const double one = 1.0, zero = 0.0;
    PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, r, r, m, &one, A, m, A, m, &zero, Gd, r));
    std::vector<double> G((size_t)r * r), w, V;
    PTROM_CUDA(cudaMemcpyAsync(G.data(), Gd, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sym_eig(st, r, G, w, V));
    int keep = 0;
    while (keep < r && w[keep] > 1e-20 * w[0]) ++keep;
    if (keep == 0) return set_error(PTROM_EINVAL, "ptrom_build: POD range block has rank 0");
    std::vector<double> W((size_t)r * keep);  // column-major r x keep
    for (int j = 0; j < keep; ++j)
        for (int i = 0; i < r; ++i) W[(size_t)j * r + i] = V[(size_t)i * r + j] / sqrt(w[j]);
    PTROM_CUDA(cudaMemcpyAsync(Wd, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, st));
    PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, m, keep, r, &one, A, m, Wd, r, &zero, T, m));
    PTROM_CUDA(cudaMemcpyAsync(A, T, sizeof(double) * (size_t)m * keep, cudaMemcpyDeviceToDevice, st));
    r = keep;
    return PTROM_OK;
}

// Randomized POD (range finder with two power iterations, each step
// orthonormalised twice; then the exact SVD of the small projected block):
// M leading modes of S (nd x K) to ~machine precision for the fast-decaying
// spectra of snapshot matrices, with O(nd K (M + 32)) GEMM work on the GPU and
// O((M + 32)^3) on the host.
static int pod_randomized(int nd, int K, const double *S, int &M, cudaStream_t st, std::vector<double> &Phi,
                          std::vector<double> &sigma, bool clamp) {
    cublasHandle_t h;
    PTROM_TRY(cublas_for(st, &h));
    int r = std::min(M + 32, std::min(nd, K));
    const int r0 = r;
    double *Om, *Y, *Z, *T, *Gd, *Wd, *Bm;
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&Om, sizeof(double) * (size_t)K * r0));
    PTROM_TRY(sc.alloc(&Y, sizeof(double) * (size_t)nd * r0));
    PTROM_TRY(sc.alloc(&Z, sizeof(double) * (size_t)K * r0));
    PTROM_TRY(sc.alloc(&T, sizeof(double) * (size_t)std::max(nd, K) * r0));
    PTROM_TRY(sc.alloc(&Gd, sizeof(double) * (size_t)r0 * r0));
    PTROM_TRY(sc.alloc(&Wd, sizeof(double) * (size_t)r0 * r0));
    PTROM_TRY(sc.alloc(&Bm, sizeof(double) * (size_t)r0 * K));
    {
        std::vector<double> om((size_t)K * r0);
        std::mt19937_64 rng(20210302ull);
        std::normal_distribution<double> normal(0.0, 1.0);
        for (double &v : om) v = normal(rng);
        PTROM_CUDA(cudaMemcpyAsync(Om, om.data(), sizeof(double) * om.size(), cudaMemcpyHostToDevice, st));
        PTROM_CUDA(cudaStreamSynchronize(st));
    }
    const double one = 1.0, zero = 0.0;
    PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, nd, r, K, &one, S, nd, Om, K, &zero, Y, nd));
    for (int pass = 0; pass < 2; ++pass) PTROM_TRY(svqb(h, nd, r, Y, T, Gd, Wd, st));
    for (int it = 0; it < 2; ++it) {
        PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, K, r, nd, &one, S, nd, Y, nd, &zero, Z, K));
        for (int pass = 0; pass < 2; ++pass) PTROM_TRY(svqb(h, K, r, Z, T, Gd, Wd, st));
        PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, nd, r, K, &one, S, nd, Z, K, &zero, Y, nd));
        for (int pass = 0; pass < 2; ++pass) PTROM_TRY(svqb(h, nd, r, Y, T, Gd, Wd, st));
    }
    // B = Y^T S (r x K); its left singular vectors by the eigenvectors of B B^T
    PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, r, K, nd, &one, Y, nd, S, nd, &zero, Bm, r));
    PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, r, r, K, &one, Bm, r, Bm, r, &zero, Gd, r));
    std::vector<double> G((size_t)r * r), w, V;
    PTROM_CUDA(cudaMemcpyAsync(G.data(), Gd, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sym_eig(st, r, G, w, V));
    if (clamp) {
        int q = 0;
        while (q < M && q < r && w[q] > 1e-24 * w[0]) ++q;
        M = std::max(q, 1);
    }
    if (M > r) return set_error(PTROM_EINVAL, "ptrom_build: POD rank %d exceeds the snapshot rank %d", M, r);
    sigma.resize(M);
    std::vector<double> Vm((size_t)r * M);  // column-major r x M
    for (int m = 0; m < M; ++m) {
        if (!(w[m] > 0.0)) return set_error(PTROM_EINVAL, "ptrom_build: POD rank %d exceeds the snapshot rank", M);
        sigma[m] = sqrt(w[m]);
        for (int i = 0; i < r; ++i) Vm[(size_t)m * r + i] = V[(size_t)i * r + m];
    }
    PTROM_CUDA(cudaMemcpyAsync(Wd, Vm.data(), sizeof(double) * Vm.size(), cudaMemcpyHostToDevice, st));
    PTROM_CUBLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, nd, M, r, &one, Y, nd, Wd, r, &zero, T, nd));
    std::vector<double> P((size_t)nd * M);
    PTROM_CUDA(cudaMemcpyAsync(P.data(), T, sizeof(double) * P.size(), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sc.release());
    Phi.resize((size_t)nd * M);
    for (int m = 0; m < M; ++m) {
        int best = 0;
        for (int d = 1; d < nd; ++d)
            if (fabs(P[(size_t)m * nd + d]) > fabs(P[(size_t)m * nd + best])) best = d;
        const double sgn = P[(size_t)m * nd + best] < 0 ? -1.0 : 1.0;  // largest-magnitude entry positive
        for (int d = 0; d < nd; ++d) Phi[(size_t)d * M + m] = sgn * P[(size_t)m * nd + d];
    }
    return PTROM_OK;
}

// POD of the nd x K column-major device matrix S: M leading modes (Phi host
// [nd][M] row-major) and singular values: by the Gram matrix S^T S (method of
// snapshots) when there are fewer snapshots than dofs, else by the covariance
// S S^T, whose eigenvectors are the modes themselves; the host eigensolver
// then works on the smaller of the two (O(min(nd, K)^3)).
// With clamp, M is lowered to the number of modes whose eigenvalue exceeds
// 1e-24 of the largest (the numerical rank), instead of failing.
int pod_device(int nd, int K, const double *S, int &M, cudaStream_t st, std::vector<double> &Phi,
               std::vector<double> &sigma, bool clamp = false) {
    if (M > K) return set_error(PTROM_EINVAL, "ptrom_build: POD rank %d exceeds the %d snapshots", M, K);
    if (std::min(nd, K) > g_pod_exact_max.load()) return pod_randomized(nd, K, S, M, st, Phi, sigma, clamp);
    if (nd < K) {
        double *C = nullptr;
        ScratchScope sc(st);
        PTROM_TRY(sc.alloc(&C, sizeof(double) * (size_t)nd * nd));
        dim3 grid((nd + 31) / 32, (nd + 31) / 32);
        k_cov<<<grid, 256, 0, st>>>(nd, K, S, C);
        count_launch();
        std::vector<double> Ch((size_t)nd * nd);
        PTROM_CUDA(cudaMemcpyAsync(Ch.data(), C, sizeof(double) * Ch.size(), cudaMemcpyDeviceToHost, st));
        PTROM_CUDA(cudaStreamSynchronize(st));
        PTROM_TRY(sc.release());
        for (int a = 0; a < nd; ++a)
            for (int b = 0; b < a; ++b) Ch[(size_t)a * nd + b] = Ch[(size_t)b * nd + a];
        std::vector<double> w, V;
        PTROM_TRY(sym_eig(st, nd, Ch, w, V));
        if (clamp) {
            int r = 0;
            while (r < M && w[r] > 1e-24 * w[0]) ++r;
            M = std::max(r, 1);
        }
        sigma.resize(M);
        Phi.resize((size_t)nd * M);
        for (int m = 0; m < M; ++m) {
            if (!(w[m] > 0.0)) return set_error(PTROM_EINVAL, "ptrom_build: POD rank %d exceeds the snapshot rank", M);
            sigma[m] = sqrt(w[m]);
            for (int d = 0; d < nd; ++d) Phi[(size_t)d * M + m] = V[(size_t)d * nd + m];
        }
        for (int m = 0; m < M; ++m) {  // sign convention: each column's largest-magnitude entry is positive
            int best = 0;
            for (int d = 1; d < nd; ++d)
                if (fabs(Phi[(size_t)d * M + m]) > fabs(Phi[(size_t)best * M + m])) best = d;
            if (Phi[(size_t)best * M + m] < 0)
                for (int d = 0; d < nd; ++d) Phi[(size_t)d * M + m] = -Phi[(size_t)d * M + m];
        }
        return PTROM_OK;
    }
    double *G = nullptr, *Wd = nullptr, *Pd = nullptr;
    ScratchScope sc(st);
    PTROM_TRY(sc.alloc(&G, sizeof(double) * (size_t)K * K));
    dim3 grid((K + 31) / 32, (K + 31) / 32);
    k_gram<<<grid, 256, 0, st>>>(nd, K, S, G);
    count_launch();
    std::vector<double> Gh((size_t)K * K);
    PTROM_CUDA(cudaMemcpyAsync(Gh.data(), G, sizeof(double) * Gh.size(), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sc.release());
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < a; ++b) Gh[(size_t)a * K + b] = Gh[(size_t)b * K + a];
    std::vector<double> w, V;
    PTROM_TRY(sym_eig(st, K, Gh, w, V));
    if (clamp) {
        int r = 0;
        while (r < M && w[r] > 1e-24 * w[0]) ++r;
        M = std::max(r, 1);
    }
    sigma.resize(M);
    std::vector<double> Wm((size_t)K * M);
    for (int m = 0; m < M; ++m) {
        if (!(w[m] > 0.0)) return set_error(PTROM_EINVAL, "ptrom_build: POD rank %d exceeds the snapshot rank", M);
        sigma[m] = sqrt(w[m]);
        for (int k = 0; k < K; ++k) Wm[(size_t)k * M + m] = V[(size_t)k * K + m] / sigma[m];
    }
    PTROM_TRY(sc.alloc(&Wd, sizeof(double) * Wm.size()));
    PTROM_TRY(sc.alloc(&Pd, sizeof(double) * (size_t)nd * M));
    PTROM_CUDA(cudaMemcpyAsync(Wd, Wm.data(), sizeof(double) * Wm.size(), cudaMemcpyHostToDevice, st));
    k_combine<<<(nd + 127) / 128, 128, 0, st>>>(nd, K, M, S, Wd, Pd);
    count_launch();
    Phi.resize((size_t)nd * M);
    PTROM_CUDA(cudaMemcpyAsync(Phi.data(), Pd, sizeof(double) * Phi.size(), cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(sc.release());
    // Phi = S V / sigma loses orthogonality for modes with tiny sigma (the Gram
    // matrix squares the condition number); two modified Gram-Schmidt passes
    // restore orthonormal columns.
    for (int pass = 0; pass < 2; ++pass) {
        for (int m = 0; m < M; ++m) {
            for (int q = 0; q < m; ++q) {
                double dot = 0.0;
                for (int d = 0; d < nd; ++d) dot += Phi[(size_t)d * M + q] * Phi[(size_t)d * M + m];
                for (int d = 0; d < nd; ++d) Phi[(size_t)d * M + m] -= dot * Phi[(size_t)d * M + q];
            }
            double nrm = 0.0;
            for (int d = 0; d < nd; ++d) nrm += Phi[(size_t)d * M + m] * Phi[(size_t)d * M + m];
            nrm = sqrt(nrm);
            if (nrm > 0.0)
                for (int d = 0; d < nd; ++d) Phi[(size_t)d * M + m] /= nrm;
        }
    }
    // sign convention: each column's largest-magnitude entry is positive
    for (int m = 0; m < M; ++m) {
        int best = 0;
        for (int d = 1; d < nd; ++d)
            if (fabs(Phi[(size_t)d * M + m]) > fabs(Phi[(size_t)best * M + m])) best = d;
        if (Phi[(size_t)best * M + m] < 0)
            for (int d = 0; d < nd; ++d) Phi[(size_t)d * M + m] = -Phi[(size_t)d * M + m];
    }
    return PTROM_OK;
}

// Alg. 1 greedy sampling on Phi_r (host, [2n][Mr] row-major).
std::vector<int> greedy_sample(const std::vector<double> &Pr, int n, int Mr, int ns) {
    std::vector<int> chosen;
    std::vector<char> taken(n, 0);
    const int n_a = ns, n_d = 2 * ns;
    const int n_c = std::min(Mr, n_d);
    const int n_it = std::min(n_c, n_a);
    int n_b = 0;
    std::vector<double> err(n);
    for (int it = 1; it <= n_it; ++it) {
        const int n_ci = n_c / n_it + (it <= n_c % n_it ? 1 : 0);
        const int n_ai = n_a / n_it + (it <= n_a % n_it ? 1 : 0);
        // R = next n_ci columns, minus their gappy reconstruction from the first n_b
        std::vector<double> R((size_t)2 * n * n_ci);
        for (int d = 0; d < 2 * n; ++d)
            for (int q = 0; q < n_ci; ++q) R[(size_t)q * 2 * n + d] = Pr[(size_t)d * Mr + n_b + q];
        if (it > 1 && n_b > 0) {
            const int m = 2 * (int)chosen.size();
            std::vector<double> A((size_t)m * n_b), B((size_t)m * n_ci), X;
            for (int s = 0; s < (int)chosen.size(); ++s) {
                const int rows[2] = {chosen[s], n + chosen[s]};
                for (int h = 0; h < 2; ++h) {
                    const int ri = 2 * s + h;
                    for (int c = 0; c < n_b; ++c) A[(size_t)c * m + ri] = Pr[(size_t)rows[h] * Mr + c];
                    for (int q = 0; q < n_ci; ++q) B[(size_t)q * m + ri] = R[(size_t)q * 2 * n + rows[h]];
                }
            }
            // rows ordered (chi, psi) per body here; the least-squares solution does not depend on row order.
            // The minimum-norm solution: the gappy fit on few sampled dofs is
            // under-determined or rank deficient when fewer dofs than columns
            // are sampled or the columns coincide there.
            lstsq_minnorm(m, n_b, A, B, n_ci, X);
            for (int q = 0; q < n_ci; ++q)
                for (int d = 0; d < 2 * n; ++d) {
                    double s = 0.0;
                    for (int c = 0; c < n_b; ++c) s += Pr[(size_t)d * Mr + c] * X[(size_t)q * n_b + c];
                    R[(size_t)q * 2 * n + d] -= s;
                }
        }
        for (int l = 0; l < n; ++l) {
            double e = 0.0;
            for (int q = 0; q < n_ci; ++q) {
                const double a = R[(size_t)q * 2 * n + l], b = R[(size_t)q * 2 * n + n + l];
                e += a * a + b * b;
            }
            err[l] = e;
        }
        for (int k = 0; k < n_ai; ++k) {
            int best = -1;
            for (int l = 0; l < n; ++l)
                if (!taken[l] && (best < 0 || err[l] > err[best])) best = l;
            if (best < 0) break;
            taken[best] = 1;
            chosen.push_back(best);
        }
        n_b += n_ci;
    }
    return chosen;
}

// A = [P Phi_r]^+ (Moore-Penrose, Eq. gappySolution): Ah [M_r][2 n_s]
// row-major, P picking both dofs (chi rows, then psi rows) of each sampled
// body.  P Phi_r is n_d x M_r; with n_d >= M_r and full column rank A is its
// left inverse; with n_d < M_r (the gappy problem under-determined, as in the
// paper's mushroom cloud, n_d = 150 < M_r = 185) the minimum-norm right inverse.
void gappy_operator(const std::vector<double> &Pr, int n, int Mr, const std::vector<int> &sampled,
                    std::vector<double> &Ah) {
    const int ns = (int)sampled.size(), m2 = 2 * ns;
    std::vector<double> PP((size_t)m2 * Mr), Iden((size_t)m2 * m2, 0.0), X;
    for (int s = 0; s < ns; ++s)
        for (int c = 0; c < Mr; ++c) {
            PP[(size_t)c * m2 + s] = Pr[(size_t)sampled[s] * Mr + c];
            PP[(size_t)c * m2 + ns + s] = Pr[(size_t)(n + sampled[s]) * Mr + c];
        }
    for (int d = 0; d < m2; ++d) Iden[(size_t)d * m2 + d] = 1.0;
    lstsq_minnorm(m2, Mr, PP, Iden, m2, X);  // X = (P Phi_r)^+ (M_r x m2, column-major)
    Ah.assign((size_t)Mr * m2, 0.0);
    for (int d = 0; d < m2; ++d)
        for (int r = 0; r < Mr; ++r) Ah[(size_t)r * m2 + d] = X[(size_t)d * Mr + r];
}

}  // namespace
}  // namespace ptrom

using namespace ptrom;

extern "C" int ptrom_build(const ptrom_build_params *p, int n, int n_params, const double *x0s,
                           const double *gammas, ptrom_model **out, ptrom_build_info *info,
                           ptrom_stream_t stream) {
    if (!p || !x0s || !gammas || !out) return set_error(PTROM_EINVAL, "ptrom_build: NULL argument");
    if (n < 2 || n > 131072 || n_params < 1 || p->steps < 1 || (long long)n_params * p->steps > 65536 ||
        (double)n_params * p->steps * 2 * n * 8 > 64e9)
        return set_error(PTROM_EINVAL, "ptrom_build: sizes out of range (n=%d params=%d steps=%d)", n, n_params, p->steps);
    if (p->M < 1 || p->M > kMaxM || p->M_r < 1 || p->M_r > kMaxMr || p->n_s < 1 || p->n_s > std::min(kMaxNs, n))
        return set_error(PTROM_EINVAL, "ptrom_build: M/M_r/n_s out of range");
    if (p->criterion != PTROM_BARNES_HUT && p->criterion != PTROM_NEIGHBOR)
        return set_error(PTROM_EINVAL, "ptrom_build: bad criterion");
    cudaStream_t st = (cudaStream_t)stream;
    ptrom_build_info inf{};
    const int nd = 2 * n, M = p->M, Mr = p->M_r, ns = p->n_s;
    const double dt = p->fom.dt, delta = p->fom.delta;
    // ---------------- Stage 1: FOM snapshots (or the caller's)
    auto t0 = Clock::now();
    const int K = n_params * p->steps;
    double *S_own = nullptr, *x = nullptr, *f = nullptr;
    void *work = nullptr;
    const size_t wbytes = fom_workspace_bytes(&p->fom, n);
    if (!wbytes) return set_error(PTROM_EINVAL, "ptrom_build: bad FOM parameters");
    ScratchScope sc(st);  // every training buffer below, released on all paths
    if (!p->snapshots) PTROM_TRY(sc.alloc(&S_own, sizeof(double) * (size_t)nd * K));
    const double *S = p->snapshots ? p->snapshots : S_own;
    PTROM_TRY(sc.alloc(&x, sizeof(double) * nd));
    PTROM_TRY(sc.alloc(&f, sizeof(double) * nd));
    PTROM_TRY(sc.alloc(&work, wbytes));
    for (int q = 0; q < n_params && !p->snapshots; ++q) {
        const double *x0 = x0s + (size_t)q * nd, *G = gammas + (size_t)q * n;
        ptrom_fom_params fq = p->fom;
        fq.u_inf = p->u_infs ? p->u_infs + (size_t)q * nd : nullptr;
        PTROM_CUDA(cudaMemcpyAsync(x, x0, sizeof(double) * nd, cudaMemcpyDeviceToDevice, st));
        PTROM_TRY(velocity(n, x, n, x, G, delta, f, nullptr, p->fom.prec, st));
        for (int s = 0; s < p->steps; ++s) {
            const int stt = fom_step(&fq, n, G, x, f, work, wbytes, nullptr, stream);
            if (stt != PTROM_OK && stt != PTROM_ENOCONV) return stt;
            k_snapshot<<<(nd + 255) / 256, 256, 0, st>>>(nd, x, S_own + (size_t)(q * p->steps + s) * nd);
            count_launch();
        }
    }
    PTROM_CUDA(cudaStreamSynchronize(st));
    inf.n_snapshots = K;
    inf.seconds_fom = secs(t0);
    // ---------------- Stage 2: POD, quadtree, clusters
    t0 = Clock::now();
    std::vector<double> Phi, sigma;
    int Mpod = M;
    PTROM_TRY(pod_device(nd, K, S, Mpod, st, Phi, sigma));
    inf.sigma_ratio = sigma[M - 1] / sigma[0];
    inf.seconds_pod = secs(t0);
    t0 = Clock::now();
    std::vector<double> x0h(nd), Gh(n);
    PTROM_CUDA(cudaMemcpyAsync(x0h.data(), x0s, sizeof(double) * nd, cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaMemcpyAsync(Gh.data(), gammas, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    std::vector<double> pts(2 * (size_t)n);  // W = Phi sigma, one 2-D point per body
    for (int i = 0; i < n; ++i) {
        double a = 0.0, b = 0.0;
        for (int m = 0; m < M; ++m) {
            a += Phi[(size_t)i * M + m] * sigma[m];
            b += Phi[(size_t)(n + i) * M + m] * sigma[m];
        }
        pts[2 * i] = a;
        pts[2 * i + 1] = b;
    }
    QTree T;
    T.make(pts.data(), n);
    // WeightedMean in W (node centroids, |Gamma| weights)
    std::vector<double> cen(2 * T.nodes.size());
    for (size_t id = 0; id < T.nodes.size(); ++id) {
        const QNode &nd_ = T.nodes[id];
        double ws = 0.0, a = 0.0, b = 0.0;
        for (int k = 0; k < nd_.count; ++k) {
            const int bb = T.perm[nd_.first + k];
            ws += fabs(Gh[bb]);
        }
        const bool unw = ws == 0.0;
        for (int k = 0; k < nd_.count; ++k) {
            const int bb = T.perm[nd_.first + k];
            const double w = unw ? 1.0 : fabs(Gh[bb]);
            a += w * pts[2 * bb];
            b += w * pts[2 * bb + 1];
        }
        const double W = unw ? nd_.count : ws;
        cen[2 * id] = a / W;
        cen[2 * id + 1] = b / W;
    }
    // FindClusters for every body (Tier II) + UniqueSearch
    ClusterSet all;
    all.off.push_back(0);
    std::vector<long long> tmp;
    for (int i = 0; i < n; ++i) {
        find_clusters(T, pts, cen, i, p->criterion, p->theta, p->p_c, tmp);
        for (long long key : tmp) {
            auto it = all.index.find(key);
            int c;
            if (it == all.index.end()) {
                c = (int)all.keys.size();
                all.index.emplace(key, c);
                all.keys.push_back(key);
            } else {
                c = it->second;
            }
            all.idx.push_back(c);
        }
        all.off.push_back((int)all.idx.size());
    }
    const int NcA = (int)all.keys.size();
    inf.N_c_all = NcA;
    inf.mean_list_all = (double)all.idx.size() / n;
    // cluster values for the first training parameter (Tier II recomputes them for the
    // others; the online model starts at this one)
    const int Mp = (M + 3) & ~3;
    std::vector<double> phicA((size_t)2 * NcA * M), x0cA(2 * (size_t)NcA), gcA(NcA);
    std::vector<int> mem;
    for (int c = 0; c < NcA; ++c) {
        key_members(T, all.keys[c], mem);
        double xc[2];
        cluster_values(mem, n, M, Phi.data(), x0h.data(), Gh.data(), &phicA[(size_t)c * M],
                       &phicA[(size_t)(NcA + c) * M], xc, &gcA[c]);
        x0cA[c] = xc[0];
        x0cA[NcA + c] = xc[1];
    }
    inf.seconds_tree = secs(t0);
    // ---------------- Stage 3: Tier-II LSPG over all bodies, residual snapshots
    t0 = Clock::now();
    const double ox = x0h[0], oy = x0h[n];
    std::vector<float> phif((size_t)nd * Mp, 0.f), x0f(nd), phicf((size_t)2 * NcA * Mp, 0.f), x0cf(2 * (size_t)NcA),
        gcf(NcA);
    for (int d = 0; d < nd; ++d)
        for (int m = 0; m < M; ++m) phif[(size_t)d * Mp + m] = (float)Phi[(size_t)d * M + m];
    const int nblk = (n + kT2Bodies - 1) / kT2Bodies, nout = M * M + M;
    // residual snapshots kept (all Gauss-Newton iterates of every step and
    // parameter, up to 24 GB of FP64 columns)
    const long long want_res = (long long)n_params * p->steps * std::min(std::max(p->max_gn, 1), 10);
    const int maxres = (int)std::min<long long>(std::min<long long>(want_res, 262144), (long long)(24e9 / (8.0 * nd)));
    // device buffers for Tier II
    float *dphi, *dx0, *dphic, *dx0c, *dgc, *dxt, *dpd, *dxq, *dxh, *ddx, *df, *dfp, *dD, *dr, *dpart, *du;
    int *doff, *didx;
    double *dout, *R;
    auto falloc = [&](float **pp, size_t cnt) { return sc.alloc(pp, sizeof(float) * std::max<size_t>(cnt, 4)); };
    PTROM_TRY(falloc(&dphi, phif.size()));
    PTROM_TRY(falloc(&dx0, nd));
    PTROM_TRY(falloc(&dphic, phicf.size()));
    PTROM_TRY(falloc(&dx0c, 2 * (size_t)NcA));
    PTROM_TRY(falloc(&dgc, NcA));
    PTROM_TRY(falloc(&dxt, nd));
    PTROM_TRY(falloc(&dpd, nd));
    PTROM_TRY(falloc(&dxq, 2 * (size_t)NcA));
    PTROM_TRY(falloc(&dxh, Mp));
    PTROM_TRY(falloc(&ddx, Mp));
    PTROM_TRY(falloc(&df, nd));
    PTROM_TRY(falloc(&dfp, nd));
    PTROM_TRY(falloc(&dD, 3 * (size_t)n));
    PTROM_TRY(falloc(&dr, nd));
    PTROM_TRY(falloc(&dpart, (size_t)nblk * nout));
    PTROM_TRY(falloc(&du, nd));
    PTROM_TRY(sc.alloc(&doff, sizeof(int) * (n + 1)));
    PTROM_TRY(sc.alloc(&didx, sizeof(int) * std::max<size_t>(all.idx.size(), 1)));
    PTROM_TRY(sc.alloc(&dout, sizeof(double) * nout));
    PTROM_TRY(sc.alloc(&R, sizeof(double) * (size_t)nd * maxres));
    PTROM_CUDA(cudaMemcpyAsync(dphi, phif.data(), sizeof(float) * phif.size(), cudaMemcpyHostToDevice, st));
    PTROM_CUDA(cudaMemcpyAsync(doff, all.off.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    if (!all.idx.empty())
        PTROM_CUDA(cudaMemcpyAsync(didx, all.idx.data(), sizeof(int) * all.idx.size(), cudaMemcpyHostToDevice, st));
    T2 t2{n, NcA, M, Mp, (float)(0.5 * dt), (float)delta, dphi, dx0, dphic, dx0c, dgc, doff, didx, du};
    std::vector<double> uq(nd, 0.0), u_first(nd, 0.0);
    std::vector<float> uf(nd, 0.f);
    const int gth = 256;
    const int grows = (nd + 2 * NcA + gth - 1) / gth;
    const int gpair = (n * 32 + gth - 1) / gth;
    const size_t smem_normal = sizeof(float) * (2 * kT2Bodies * (size_t)Mp + 2 * kT2Bodies);
    PTROM_CUDA(cudaFuncSetAttribute(k_t2_normal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_normal));
    std::vector<float> xhf(Mp, 0.f), dxf(Mp, 0.f);
    std::vector<double> xh(M, 0.0), xprev(M), outh(nout);
    int nres = 0;
    std::vector<double> tier2_traj;  // [n_params][steps + 1][M]
    tier2_traj.reserve((size_t)n_params * (p->steps + 1) * M);
    // Tier II for every training parameter: its reference state, and the
    // cluster values recomputed from the stored memberships (as Sec. 5.2
    // reloads them), each run from xhat = 0
    std::vector<double> xq(nd), Gq(n), phicQ((size_t)2 * NcA * M), x0cQ(2 * (size_t)NcA), gcQ(NcA);
    for (int q = 0; q < n_params; ++q) {
    if (q == 0) {
        xq = x0h;
        Gq = Gh;
        phicQ = phicA;
        x0cQ = x0cA;
        gcQ = gcA;
    } else {
        PTROM_CUDA(cudaMemcpyAsync(xq.data(), x0s + (size_t)q * nd, sizeof(double) * nd, cudaMemcpyDeviceToHost, st));
        PTROM_CUDA(cudaMemcpyAsync(Gq.data(), gammas + (size_t)q * n, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        PTROM_CUDA(cudaStreamSynchronize(st));
        for (int c = 0; c < NcA; ++c) {
            key_members(T, all.keys[c], mem);
            double xc[2];
            cluster_values(mem, n, M, Phi.data(), xq.data(), Gq.data(), &phicQ[(size_t)c * M],
                           &phicQ[(size_t)(NcA + c) * M], xc, &gcQ[c]);
            x0cQ[c] = xc[0];
            x0cQ[NcA + c] = xc[1];
        }
    }
    if (p->u_infs) {
        PTROM_CUDA(cudaMemcpyAsync(uq.data(), p->u_infs + (size_t)q * nd, sizeof(double) * nd, cudaMemcpyDeviceToHost, st));
        PTROM_CUDA(cudaStreamSynchronize(st));
        if (q == 0) u_first = uq;
    }
    for (int d = 0; d < nd; ++d) uf[d] = (float)(dt * uq[d]);
    PTROM_CUDA(cudaMemcpyAsync(du, uf.data(), sizeof(float) * nd, cudaMemcpyHostToDevice, st));
    for (int d = 0; d < nd; ++d) x0f[d] = (float)(xq[d] - (d < n ? ox : oy));
    for (int rr = 0; rr < 2 * NcA; ++rr) {
        for (int m = 0; m < M; ++m) phicf[(size_t)rr * Mp + m] = (float)phicQ[(size_t)rr * M + m];
        x0cf[rr] = (float)(x0cQ[rr] - (rr < NcA ? ox : oy));
    }
    for (int c = 0; c < NcA; ++c) gcf[c] = (float)(gcQ[c] * kInv2Pi);
    PTROM_CUDA(cudaMemcpyAsync(dx0, x0f.data(), sizeof(float) * nd, cudaMemcpyHostToDevice, st));
    PTROM_CUDA(cudaMemcpyAsync(dphic, phicf.data(), sizeof(float) * phicf.size(), cudaMemcpyHostToDevice, st));
    PTROM_CUDA(cudaMemcpyAsync(dx0c, x0cf.data(), sizeof(float) * x0cf.size(), cudaMemcpyHostToDevice, st));
    PTROM_CUDA(cudaMemcpyAsync(dgc, gcf.data(), sizeof(float) * NcA, cudaMemcpyHostToDevice, st));
    std::fill(xh.begin(), xh.end(), 0.0);
    tier2_traj.insert(tier2_traj.end(), xh.begin(), xh.end());
    // f~ at xhat = 0 (R11)
    PTROM_CUDA(cudaMemsetAsync(dxh, 0, sizeof(float) * Mp, st));
    PTROM_CUDA(cudaMemsetAsync(ddx, 0, sizeof(float) * Mp, st));
    PTROM_CUDA(cudaMemsetAsync(dfp, 0, sizeof(float) * nd, st));
    k_t2_gather<<<grows, gth, 0, st>>>(t2, dxh, ddx, dxt, dpd, dxq);
    k_t2_pairs<<<gpair, gth, 0, st>>>(t2, dxt, dxq, dpd, dfp, dfp, dD, dr, nullptr);
    count_launch(2);
    for (int s = 0; s < p->steps; ++s) {
        xprev = xh;
        double first = -1.0;
        for (int k = 0; k < p->max_gn; ++k) {
            for (int m = 0; m < M; ++m) {
                xhf[m] = (float)xh[m];
                dxf[m] = (float)(xh[m] - xprev[m]);
            }
            PTROM_CUDA(cudaMemcpyAsync(dxh, xhf.data(), sizeof(float) * Mp, cudaMemcpyHostToDevice, st));
            PTROM_CUDA(cudaMemcpyAsync(ddx, dxf.data(), sizeof(float) * Mp, cudaMemcpyHostToDevice, st));
            k_t2_gather<<<grows, gth, 0, st>>>(t2, dxh, ddx, dxt, dpd, dxq);
            double *rcol = nres < maxres ? R + (size_t)nres * nd : nullptr;
            k_t2_pairs<<<gpair, gth, 0, st>>>(t2, dxt, dxq, dpd, dfp, df, dD, dr, rcol);
            k_t2_normal<<<nblk, 256, smem_normal, st>>>(t2, dD, dr, dpart);
            k_t2_reduce<<<(nout + 127) / 128, 128, 0, st>>>(nblk, nout, dpart, dout);
            count_launch(4);
            if (rcol) ++nres;
            PTROM_CUDA(cudaMemcpyAsync(outh.data(), dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, st));
            PTROM_CUDA(cudaStreamSynchronize(st));
            std::vector<double> Gm(outh.begin(), outh.begin() + (size_t)M * M);
            std::vector<double> rhs(M);
            double g2 = 0.0;
            for (int m = 0; m < M; ++m) {
                rhs[m] = -outh[(size_t)M * M + m];
                g2 += rhs[m] * rhs[m];
            }
            const double g = sqrt(g2);
            // C = (I - dt/2 blockdiag D~) Phi has orthonormal Phi and a small
            // perturbation, so its condition number is ~1 and the normal
            // equations C^T C nu = -C^T r lose no accuracy against a QR of C;
            // Cholesky solves them.  If C^T C is singular (a mode the dynamics
            // leaves exactly unexcited), the minimum-norm solution
            // nu = -(C^T C)^+ C^T r = -C^+ r is taken from its eigen-decomposition.
            if (!chol_solve(M, Gm, rhs)) {
                std::vector<double> w, V;
                jacobi_eig(M, Gm, w, V);
                const double cut = M * 2.220446049250313e-16 * std::max(w[0], 0.0);
                std::vector<double> b(M);
                for (int a = 0; a < M; ++a) b[a] = -outh[(size_t)M * M + a];
                std::fill(rhs.begin(), rhs.end(), 0.0);
                for (int j = 0; j < M; ++j) {
                    if (!(w[j] > cut)) continue;
                    double c = 0.0;
                    for (int a = 0; a < M; ++a) c += V[(size_t)a * M + j] * b[a];
                    c /= w[j];
                    for (int a = 0; a < M; ++a) rhs[a] += c * V[(size_t)a * M + j];
                }
                if (!std::isfinite(rhs[0])) return set_error(PTROM_ENAN, "ptrom_build: non-finite Tier-II step");
            }
            for (int m = 0; m < M; ++m) xh[m] += rhs[m];
            if (first < 0.0) first = g;
            const double eps = first > 0.0 ? g / first : 0.0;
            if ((eps <= p->tol && k > 0) || first == 0.0) break;
        }
        PTROM_CUDA(cudaMemcpyAsync(dfp, df, sizeof(float) * nd, cudaMemcpyDeviceToDevice, st));
        tier2_traj.insert(tier2_traj.end(), xh.begin(), xh.end());
    }
    }  // training parameters
    PTROM_CUDA(cudaStreamSynchronize(st));
    inf.n_res_snapshots = nres;
    inf.seconds_tier2 = secs(t0);
    // ---------------- Stage 3b/4: residual POD, greedy sampling, A
    t0 = Clock::now();
    std::vector<double> Phir, sigr;
    int Mr_eff = std::min(Mr, nres);
    PTROM_TRY(pod_device(nd, nres, R, Mr_eff, st, Phir, sigr, true));
    std::vector<int> sampled = greedy_sample(Phir, n, Mr_eff, ns);
    if ((int)sampled.size() != ns) return set_error(PTROM_EINVAL, "ptrom_build: sampling found %zu bodies", sampled.size());
    const int m2 = 2 * ns;
    std::vector<double> Ah;
    gappy_operator(Phir, n, Mr_eff, sampled, Ah);
    // clusters of the sampled bodies, numbered by first appearance
    std::vector<int> off(ns + 1, 0), idx;
    std::vector<int> remap(NcA, -1), order;
    for (int s = 0; s < ns; ++s) {
        const int i = sampled[s];
        for (int e = all.off[i]; e < all.off[i + 1]; ++e) {
            const int c = all.idx[e];
            if (remap[c] < 0) {
                remap[c] = (int)order.size();
                order.push_back(c);
            }
            idx.push_back(remap[c]);
        }
        off[s + 1] = (int)idx.size();
    }
    const int Nc = (int)order.size();
    std::vector<double> phi_s((size_t)m2 * M), x0_s(m2), phi_c((size_t)2 * Nc * M), x0_c(2 * (size_t)Nc), g_c(Nc);
    for (int s = 0; s < ns; ++s) {
        for (int m = 0; m < M; ++m) {
            phi_s[(size_t)s * M + m] = Phi[(size_t)sampled[s] * M + m];
            phi_s[(size_t)(ns + s) * M + m] = Phi[(size_t)(n + sampled[s]) * M + m];
        }
        x0_s[s] = x0h[sampled[s]];
        x0_s[ns + s] = x0h[n + sampled[s]];
    }
    std::vector<int> cl_off(Nc + 1, 0), cl_mem;
    for (int c = 0; c < Nc; ++c) {
        const int a = order[c];
        for (int m = 0; m < M; ++m) {
            phi_c[(size_t)c * M + m] = phicA[(size_t)a * M + m];
            phi_c[(size_t)(Nc + c) * M + m] = phicA[(size_t)(NcA + a) * M + m];
        }
        x0_c[c] = x0cA[a];
        x0_c[Nc + c] = x0cA[NcA + a];
        g_c[c] = gcA[a];
        key_members(T, all.keys[a], mem);
        cl_mem.insert(cl_mem.end(), mem.begin(), mem.end());
        cl_off[c + 1] = (int)cl_mem.size();
    }
    inf.N_c = Nc;
    inf.mean_list = (double)idx.size() / ns;
    inf.seconds_sample = secs(t0);
    // free the stage buffers
    PTROM_TRY(sc.release());
    PTROM_CUDA(cudaStreamSynchronize(st));
    PTROM_TRY(scratch_trim());  // hand the training buffers back to the device
    // ---------------- the online model
    ptrom_model_desc desc{};
    desc.n_s = ns;
    desc.M = M;
    desc.M_r = Mr_eff;
    desc.N_c = Nc;
    desc.dt = dt;
    desc.delta = delta;
    desc.tol = p->tol;
    desc.max_gn = p->max_gn;
    desc.qr_prec = p->qr_prec;
    desc.phi_s = phi_s.data();
    desc.x0_s = x0_s.data();
    desc.phi_c = phi_c.data();
    desc.x0_c = x0_c.data();
    desc.gamma_c = g_c.data();
    desc.A = Ah.data();
    desc.off = off.data();
    desc.idx = idx.empty() ? off.data() : idx.data();
    std::vector<double> u_s(2 * (size_t)ns);
    for (int s = 0; s < ns; ++s) {
        u_s[s] = u_first[sampled[s]];
        u_s[ns + s] = u_first[n + sampled[s]];
    }
    desc.u_s = p->u_infs ? u_s.data() : nullptr;
    ptrom_model *m = nullptr;
    PTROM_TRY(ptrom_model_create(&desc, &m));
    m->built = true;
    m->n = n;
    m->phi = Phi;
    m->sigma = sigma;
    m->sampled = sampled;
    m->A = Ah;
    m->cl_off = cl_off;
    m->cl_mem = cl_mem;
    m->phi_r = Phir;
    m->tier2_traj.swap(tier2_traj);
    m->n_params = n_params;
    m->steps = p->steps;
    const int e = model_store_basis(m, Phi.data(), x0h.data());
    if (e != PTROM_OK) {
        ptrom_free(m);
        return set_error(e, "ptrom_build: could not store the basis");
    }
    if (info) *info = inf;
    *out = m;
    return PTROM_OK;
}

int ptrom::model_store_basis(ptrom_model *m, const double *phi, const double *x0) {
    const size_t nphi = (size_t)2 * m->n * m->d.M, nd = 2 * (size_t)m->n;
    void *pd = nullptr;
    if (cudaMalloc(&pd, sizeof(double) * nphi) != cudaSuccess) return PTROM_ENOMEM;
    m->bufs.push_back(pd);
    m->phi_dev = (double *)pd;
    if (cudaMemcpy(pd, phi, sizeof(double) * nphi, cudaMemcpyHostToDevice) != cudaSuccess) return PTROM_ECUDA;
    if (cudaMalloc(&pd, sizeof(double) * nd) != cudaSuccess) return PTROM_ENOMEM;
    m->bufs.push_back(pd);
    m->x0_dev = (double *)pd;
    if (cudaMemcpy(pd, x0, sizeof(double) * nd, cudaMemcpyHostToDevice) != cudaSuccess) return PTROM_ECUDA;
    m->x0_full.assign(x0, x0 + nd);
    return PTROM_OK;
}

extern "C" int ptrom_set_pod_exact_max(int n) {
    if (n < 1) return set_error(PTROM_EINVAL, "ptrom_set_pod_exact_max: n=%d must be >= 1", n);
    g_pod_exact_max.store(n);
    return PTROM_OK;
}

extern "C" int ptrom_set_param_full(ptrom_model *m, const double *x0, const double *Gamma, ptrom_stream_t stream) {
    if (!m || !m->built) return set_error(PTROM_EINVAL, "ptrom_set_param_full: model not made by ptrom_build");
    if (!x0 || !Gamma) return set_error(PTROM_EINVAL, "ptrom_set_param_full: NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = m->n, M = m->d.M, ns = m->d.ns, Nc = m->d.Nc;
    std::vector<double> xh(2 * (size_t)n), Gh(n);
    PTROM_CUDA(cudaMemcpyAsync(xh.data(), x0, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaMemcpyAsync(Gh.data(), Gamma, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    std::vector<double> x0_s(2 * (size_t)ns), phi_c((size_t)2 * Nc * M), x0_c(2 * (size_t)Nc), g_c(Nc);
    for (int s = 0; s < ns; ++s) {
        x0_s[s] = xh[m->sampled[s]];
        x0_s[ns + s] = xh[n + m->sampled[s]];
    }
    std::vector<int> mem;
    for (int c = 0; c < Nc; ++c) {
        mem.assign(m->cl_mem.begin() + m->cl_off[c], m->cl_mem.begin() + m->cl_off[c + 1]);
        double xc[2];
        cluster_values(mem, n, M, m->phi.data(), xh.data(), Gh.data(), &phi_c[(size_t)c * M],
                       &phi_c[(size_t)(Nc + c) * M], xc, &g_c[c]);
        x0_c[c] = xc[0];
        x0_c[Nc + c] = xc[1];
    }
    PTROM_TRY(model_fill_param(m, x0_s.data(), phi_c.data(), x0_c.data(), g_c.data()));
    PTROM_CUDA(cudaMemcpyAsync(m->x0_dev, x0, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, st));
    m->x0_full = xh;
    return PTROM_OK;
}

extern "C" int ptrom_set_inflow_full(ptrom_model *m, const double *u, ptrom_stream_t stream) {
    if (!m || !m->built) return set_error(PTROM_EINVAL, "ptrom_set_inflow_full: model not made by ptrom_build");
    if (!u) return ptrom_set_inflow(m, nullptr);
    cudaStream_t st = (cudaStream_t)stream;
    const int n = m->n, ns = m->d.ns;
    std::vector<double> uh(2 * (size_t)n), u_s(2 * (size_t)ns);
    PTROM_CUDA(cudaMemcpyAsync(uh.data(), u, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st));
    PTROM_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < ns; ++s) {
        u_s[s] = uh[m->sampled[s]];
        u_s[ns + s] = uh[n + m->sampled[s]];
    }
    return ptrom_set_inflow(m, u_s.data());
}

extern "C" int ptrom_reconstruct(const ptrom_model *m, const double *xhat, const int *rows, int nrows, double *out,
                                 ptrom_stream_t stream) {
    if (!m || !m->built) return set_error(PTROM_EINVAL, "ptrom_reconstruct: model not made by ptrom_build");
    if (!xhat || !rows || !out || nrows < 1) return set_error(PTROM_EINVAL, "ptrom_reconstruct: bad arguments");
    k_reconstruct<<<(2 * nrows + 127) / 128, 128, 0, (cudaStream_t)stream>>>(m->n, m->d.M, m->phi_dev, m->x0_dev, xhat,
                                                                             rows, nrows, out);
    PTROM_CUDA(cudaGetLastError());
    count_launch();
    return PTROM_OK;
}

extern "C" int ptrom_model_query(const ptrom_model *m, int *n, int *M, int *M_r, int *n_s, int *N_c, double *phi,
                                 double *sigma, int *sampled, double *A) {
    if (!m) return set_error(PTROM_EINVAL, "ptrom_model_query: NULL model");
    if (n) *n = m->n;
    if (M) *M = m->d.M;
    if (M_r) *M_r = m->d.Mr;
    if (n_s) *n_s = m->d.ns;
    if (N_c) *N_c = m->d.Nc;
    if ((phi || sigma || sampled || A) && !m->built)
        return set_error(PTROM_EINVAL, "ptrom_model_query: model not made by ptrom_build");
    if (phi) std::copy(m->phi.begin(), m->phi.end(), phi);
    if (sigma) std::copy(m->sigma.begin(), m->sigma.end(), sigma);
    if (sampled) std::copy(m->sampled.begin(), m->sampled.end(), sampled);
    if (A) std::copy(m->A.begin(), m->A.end(), A);
    return PTROM_OK;
}

extern "C" int ptrom_greedy_sample(int n, int M_r, const double *phi_r, int n_s, int *sampled) {
    if (n < 1 || M_r < 1 || n_s < 1 || n_s > n || !phi_r || !sampled)
        return set_error(PTROM_EINVAL, "ptrom_greedy_sample: bad arguments (n=%d M_r=%d n_s=%d)", n, M_r, n_s);
    std::vector<double> Pr(phi_r, phi_r + (size_t)2 * n * M_r);
    const std::vector<int> s = greedy_sample(Pr, n, M_r, n_s);
    if ((int)s.size() != n_s) return set_error(PTROM_EINVAL, "ptrom_greedy_sample: found %zu bodies", s.size());
    std::copy(s.begin(), s.end(), sampled);
    return PTROM_OK;
}

extern "C" int ptrom_gappy_operator(int n, int M_r, const double *phi_r, int n_s, const int *sampled, double *A) {
    if (n < 1 || M_r < 1 || n_s < 1 || n_s > n || !phi_r || !sampled || !A)
        return set_error(PTROM_EINVAL, "ptrom_gappy_operator: bad arguments (n=%d M_r=%d n_s=%d)", n, M_r, n_s);
    for (int s = 0; s < n_s; ++s)
        if (sampled[s] < 0 || sampled[s] >= n)
            return set_error(PTROM_EINVAL, "ptrom_gappy_operator: sampled[%d]=%d out of range", s, sampled[s]);
    std::vector<double> Pr(phi_r, phi_r + (size_t)2 * n * M_r), Ah;
    gappy_operator(Pr, n, M_r, std::vector<int>(sampled, sampled + n_s), Ah);
    std::copy(Ah.begin(), Ah.end(), A);
    return PTROM_OK;
}

extern "C" int ptrom_model_query_training(const ptrom_model *m, int *M_r, int *n_params, int *steps, double *phi_r,
                                          double *tier2_xhat) {
    if (!m) return set_error(PTROM_EINVAL, "ptrom_model_query_training: NULL model");
    if (!m->built || m->phi_r.empty())
        return set_error(PTROM_EINVAL, "ptrom_model_query_training: no training data (the model was not made by "
                                       "ptrom_build in this process)");
    if (M_r) *M_r = m->d.Mr;
    if (n_params) *n_params = m->n_params;
    if (steps) *steps = m->steps;
    if (phi_r) std::copy(m->phi_r.begin(), m->phi_r.end(), phi_r);
    if (tier2_xhat) std::copy(m->tier2_traj.begin(), m->tier2_traj.end(), tier2_xhat);
    return PTROM_OK;
}

extern "C" int ptrom_model_query_clusters(const ptrom_model *m, int *N_c, int *n_list, int *n_members, int *list_off,
                                          int *list_idx, int *mem_off, int *mem, double *phi_c, double *x0_c,
                                          double *gamma_c) {
    if (!m) return set_error(PTROM_EINVAL, "ptrom_model_query_clusters: NULL model");
    if (N_c) *N_c = m->d.Nc;
    if (n_list) *n_list = (int)m->h_idx.size();
    if (n_members) *n_members = (int)m->cl_mem.size();
    if ((mem_off || mem) && !m->built)
        return set_error(PTROM_EINVAL, "ptrom_model_query_clusters: memberships kept only by ptrom_build models");
    if (list_off) std::copy(m->h_off.begin(), m->h_off.end(), list_off);
    if (list_idx) std::copy(m->h_idx.begin(), m->h_idx.end(), list_idx);
    if (mem_off) std::copy(m->cl_off.begin(), m->cl_off.end(), mem_off);
    if (mem) std::copy(m->cl_mem.begin(), m->cl_mem.end(), mem);
    if (phi_c) std::copy(m->h_phi_c.begin(), m->h_phi_c.end(), phi_c);
    if (x0_c) std::copy(m->h_x0_c.begin(), m->h_x0_c.end(), x0_c);
    if (gamma_c) std::copy(m->h_gamma_c.begin(), m->h_gamma_c.end(), gamma_c);
    return PTROM_OK;
}

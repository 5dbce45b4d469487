// Biot-Savart all-pairs kernels and their C-ABI entry points:
//   bs_velocity (Sec. 2, Eq. 1-2) with the optional per-body self block
//   (the inexact kernel Jacobian of Sec. 2), bs_jvp and bs_vjp.
//
// Per pair, with target t, source j, (a, b) = t - s_j, s = a^2 + b^2 + delta,
// r = 1/s and q = gamma_j r (gamma = Gamma / 2 pi):
//   velocity:  f += q (-b, a)
//   self block D += gamma_j A(a, b), A = [[2ab r^2, -r + 2b^2 r^2], [r - 2a^2 r^2, -2ab r^2]]
//   J v:       (J v)_t += gamma_j A (v_t - v_j)                     (difference form)
//   J^T w:     (J^T w)_t += A^T (gamma_j w_t - gamma_t w_j)          (A is even in r)
//   dGamma:    g_t += w_j . e3 x (s_j - t) r / (2 pi)
// The difference forms make the j == t term vanish identically and avoid the
// cancellation of D_t v_t against the off-diagonal sum.
#include <math.h>

#include <vector>

#include "internal.h"
#include "pairsum.cuh"

// Resident CTAs per SM each op's register budget must allow (compile-time
// tunables; the defaults are the measured best on GB300).
#ifndef PTROM_MINB_VEL
#define PTROM_MINB_VEL 4
#endif
#ifndef PTROM_MINB_VELD
#define PTROM_MINB_VELD 2
#endif
#ifndef PTROM_MINB_JVP
#define PTROM_MINB_JVP 3
#endif
#ifndef PTROM_MINB_VJP
#define PTROM_MINB_VJP 3
#endif
namespace ptrom {

constexpr int kVelSets4MinTargets = 32768;

struct Origin2 {
    double x, y;
};

// Two adjacent 2-wide values loaded as one 16-byte (FP32) access.
template <typename V>
__device__ __forceinline__ void ld_pair(const V *p, V &a, V &b) {
    a = p[0];
    b = p[1];
}
template <>
__device__ __forceinline__ void ld_pair<float2>(const float2 *p, float2 &a, float2 &b) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
}

// ---------------------------------------------------------------- velocity
// SETS: target sets per lane (2 targets each, FP32 only); 4 sets read each
// source record from shared memory once per 8 targets of a lane.
template <typename R, bool WITH_D, bool MASK, int SETS = 1>
struct VelOp {
    using Real = R;
    using T2 = VT<R>;
    using V = typename T2::V;
    using Origin = Origin2;
    static constexpr int NACC = WITH_D ? 5 : 2;
    static constexpr int kSets = sizeof(R) == 8 ? 1 : SETS;
    static constexpr int kMinBlocks = sizeof(R) == 8 ? 2 : (WITH_D ? PTROM_MINB_VELD : (SETS > 1 ? 2 : PTROM_MINB_VEL));
    static constexpr int kKind = WITH_D ? PTROM_K_VELOCITY_D : PTROM_K_VELOCITY;
    struct Args {
        int nt, ns;
        const double *xt, *xs, *G;
        double delta;
        double *f, *D;
    };
    struct __align__(16) Rec { V nx, ny, g; };  // -x, -y duplicated; gamma duplicated
    struct Tgt { V x, y, dd; };

    static __device__ __forceinline__ Origin origin(const Args &a) { return {a.xs[0], a.xs[a.ns]}; }
    static __device__ __forceinline__ int num_targets(const Args &a) { return a.nt; }
    static __device__ __forceinline__ Rec pack(const Args &a, int j, const Origin &o) {
        Rec r;
        const bool in = j < a.ns;
        const R x = (R)(in ? a.xs[j] - o.x : 0.0), y = (R)(in ? a.xs[a.ns + j] - o.y : 0.0);
        const R g = (R)(in ? a.G[j] * kInv2Pi : 0.0);
        r.nx = T2::mk(-x, -x);
        r.ny = T2::mk(-y, -y);
        r.g = T2::mk(g, g);
        return r;
    }
    static __device__ __forceinline__ void load_tgt(const Args &a, int t0, int t1, const Origin &o, Tgt &T) {
        const double x0 = t0 < a.nt ? a.xt[t0] - o.x : 0.0, y0 = t0 < a.nt ? a.xt[a.nt + t0] - o.y : 0.0;
        const double x1 = t1 < a.nt ? a.xt[t1] - o.x : 0.0, y1 = t1 < a.nt ? a.xt[a.nt + t1] - o.y : 0.0;
        T.x = T2::mk((R)x0, (R)x1);
        T.y = T2::mk((R)y0, (R)y1);
        T.dd = T2::mk((R)a.delta, (R)a.delta);
    }
    static __device__ __forceinline__ void pair(const Rec &c, const Tgt &T, V *p) {
        V nx, ny;
        ld_pair(&c.nx, nx, ny);
        const V a = T2::add(T.x, nx);
        const V b = T2::add(T.y, ny);
        V r;
        if (WITH_D || MASK) {
            const V d2 = T2::fma(a, a, T2::mul(b, b));
            r = mask_zero(T2::rcp(T2::add(d2, T.dd)), d2);
        } else {
            V s = T2::fma(a, a, T.dd);
            s = T2::fma(b, b, s);
            r = T2::rcp(s);
        }
        const V q = T2::mul(c.g, r);
        p[0] = T2::fma(q, b, p[0]);  // sum q b  (f_chi = -sum q b)
        p[1] = T2::fma(q, a, p[1]);  // sum q a  (f_psi)
        if (WITH_D) {
            const V qr = T2::mul(q, r);
            const V p2 = T2::add(qr, qr);
            const V pa = T2::mul(p2, a);
            const V pb = T2::mul(p2, b);
            const V nq = T2::mk(-q.x, -q.y);
            p[2] = T2::fma(pa, b, p[2]);               // D00 = sum 2 q r a b
            p[3] = T2::add(p[3], T2::fma(pb, b, nq));  // D01 = sum (2 q r b^2 - q)
            p[4] = T2::add(p[4], T2::fma(pa, a, nq));  // -D10 = sum (2 q r a^2 - q)
        }
    }
    static __device__ __forceinline__ void finalize(const Args &a, int t, const double *s) {
        a.f[t] = -s[0];
        a.f[a.nt + t] = s[1];
        if (WITH_D) {
            a.D[t] = s[2];
            a.D[a.nt + t] = s[3];
            a.D[2 * a.nt + t] = -s[4];
        }
    }
};

// bs_velocity_noalloc reserves kNoAllocRecordBytes per source for the packed
// records of whichever velocity kernel a call takes.
static_assert(sizeof(VelOp<double, true, true>::Rec) <= kNoAllocRecordBytes, "noalloc record size");
static_assert(sizeof(VelOp<double, false, true>::Rec) <= kNoAllocRecordBytes, "noalloc record size");
static_assert(sizeof(VelOp<double, false, false>::Rec) <= kNoAllocRecordBytes, "noalloc record size");
static_assert(sizeof(VelOp<float, true, true>::Rec) <= kNoAllocRecordBytes, "noalloc record size");
static_assert(sizeof(VelOp<float, false, true>::Rec) <= kNoAllocRecordBytes, "noalloc record size");
static_assert(sizeof(VelOp<float, false, false>::Rec) <= kNoAllocRecordBytes, "noalloc record size");
static_assert(sizeof(VelOp<float, false, false, 4>::Rec) <= kNoAllocRecordBytes, "noalloc record size");

// ---------------------------------------------------------------- J v
template <typename R, bool MASK>
struct JvpOp {
    using Real = R;
    using T2 = VT<R>;
    using V = typename T2::V;
    using Origin = Origin2;
    static constexpr int NACC = 4;
    static constexpr int kMinBlocks = sizeof(R) == 8 ? 2 : PTROM_MINB_JVP;
    static constexpr int kSets = 1;
    static constexpr int kKind = PTROM_K_JVP;
    struct Args {
        int n;
        const double *x, *G, *v;
        double delta;
        double *jv;
        const double *lz;  // optional: jv := lz - lhdt * (J v)
        double lhdt;
    };
    struct __align__(16) Rec { V nx, ny, nvx, nvy, g; };
    struct Tgt { V x, y, vx, vy, dd; };

    static __device__ __forceinline__ Origin origin(const Args &a) { return {a.x[0], a.x[a.n]}; }
    static __device__ __forceinline__ int num_targets(const Args &a) { return a.n; }
    static __device__ __forceinline__ Rec pack(const Args &a, int j, const Origin &o) {
        Rec r;
        const bool in = j < a.n;
        const R x = (R)(in ? a.x[j] - o.x : 0.0), y = (R)(in ? a.x[a.n + j] - o.y : 0.0);
        const R g = (R)(in ? a.G[j] * kInv2Pi : 0.0);
        const R vx = (R)(in ? a.v[j] : 0.0), vy = (R)(in ? a.v[a.n + j] : 0.0);
        r.nx = T2::mk(-x, -x);
        r.ny = T2::mk(-y, -y);
        r.nvx = T2::mk(-vx, -vx);
        r.nvy = T2::mk(-vy, -vy);
        r.g = T2::mk(g, g);
        return r;
    }
    static __device__ __forceinline__ void load_tgt(const Args &a, int t0, int t1, const Origin &o, Tgt &T) {
        const bool in0 = t0 < a.n, in1 = t1 < a.n;
        T.x = T2::mk((R)(in0 ? a.x[t0] - o.x : 0.0), (R)(in1 ? a.x[t1] - o.x : 0.0));
        T.y = T2::mk((R)(in0 ? a.x[a.n + t0] - o.y : 0.0), (R)(in1 ? a.x[a.n + t1] - o.y : 0.0));
        T.vx = T2::mk((R)(in0 ? a.v[t0] : 0.0), (R)(in1 ? a.v[t1] : 0.0));
        T.vy = T2::mk((R)(in0 ? a.v[a.n + t0] : 0.0), (R)(in1 ? a.v[a.n + t1] : 0.0));
        T.dd = T2::mk((R)a.delta, (R)a.delta);
    }
    static __device__ __forceinline__ void pair(const Rec &c, const Tgt &T, V *p) {
        V nx, ny, nvx, nvy;
        ld_pair(&c.nx, nx, ny);
        ld_pair(&c.nvx, nvx, nvy);
        const V a = T2::add(T.x, nx);
        const V b = T2::add(T.y, ny);
        V r;
        if (MASK) {
            const V d2 = T2::fma(a, a, T2::mul(b, b));
            r = mask_zero(T2::rcp(T2::add(d2, T.dd)), d2);
        } else {
            V s = T2::fma(a, a, T.dd);
            s = T2::fma(b, b, s);
            r = T2::rcp(s);
        }
        const V q = T2::mul(c.g, r);
        const V dvx = T2::add(T.vx, nvx);
        const V dvy = T2::add(T.vy, nvy);
        const V tt = T2::fma(b, dvy, T2::mul(a, dvx));  // a dvx + b dvy
        const V m = T2::mul(T2::mul(q, r), tt);         // q r (a dvx + b dvy)
        p[0] = T2::fma(b, m, p[0]);                     // sum b m
        p[1] = T2::fma(q, dvy, p[1]);                   // sum q dvy
        p[2] = T2::fma(q, dvx, p[2]);                   // sum q dvx
        p[3] = T2::fma(a, m, p[3]);                     // sum a m
    }
    static __device__ __forceinline__ void finalize(const Args &a, int t, const double *s) {
        double o0 = 2.0 * s[0] - s[1], o1 = s[2] - 2.0 * s[3];
        if (a.lz) {
            o0 = a.lz[t] - a.lhdt * o0;
            o1 = a.lz[a.n + t] - a.lhdt * o1;
        }
        a.jv[t] = o0;
        a.jv[a.n + t] = o1;
    }
};

// ---------------------------------------------------------------- J^T w
template <typename R, bool MASK, bool GX, bool GG>
struct VjpOp {
    using Real = R;
    using T2 = VT<R>;
    using V = typename T2::V;
    using Origin = Origin2;
    static constexpr int NACC = (GX ? 4 : 0) + (GG ? 1 : 0);
    static constexpr int kMinBlocks = sizeof(R) == 8 ? 2 : PTROM_MINB_VJP;
    static constexpr int kSets = 1;
    static constexpr int kKind = PTROM_K_VJP;
    struct Args {
        int n;
        const double *x, *G, *w;
        double delta;
        double *gx, *gG;
        const double *lz;  // optional: gx := lz - lhdt * (J^T w)
        double lhdt;
    };
    struct __align__(16) Rec { V nx, ny, wx, nwy, g; };
    struct Tgt { V x, y, wx, wy, g, ng, dd; };

    static __device__ __forceinline__ Origin origin(const Args &a) { return {a.x[0], a.x[a.n]}; }
    static __device__ __forceinline__ int num_targets(const Args &a) { return a.n; }
    static __device__ __forceinline__ Rec pack(const Args &a, int j, const Origin &o) {
        Rec r;
        const bool in = j < a.n;
        const R x = (R)(in ? a.x[j] - o.x : 0.0), y = (R)(in ? a.x[a.n + j] - o.y : 0.0);
        const R g = (R)(in ? a.G[j] * kInv2Pi : 0.0);
        const R wx = (R)(in ? a.w[j] : 0.0), wy = (R)(in ? a.w[a.n + j] : 0.0);
        r.nx = T2::mk(-x, -x);
        r.ny = T2::mk(-y, -y);
        r.wx = T2::mk(wx, wx);
        r.nwy = T2::mk(-wy, -wy);
        r.g = T2::mk(g, g);
        return r;
    }
    static __device__ __forceinline__ void load_tgt(const Args &a, int t0, int t1, const Origin &o, Tgt &T) {
        const bool in0 = t0 < a.n, in1 = t1 < a.n;
        T.x = T2::mk((R)(in0 ? a.x[t0] - o.x : 0.0), (R)(in1 ? a.x[t1] - o.x : 0.0));
        T.y = T2::mk((R)(in0 ? a.x[a.n + t0] - o.y : 0.0), (R)(in1 ? a.x[a.n + t1] - o.y : 0.0));
        T.wx = T2::mk((R)(in0 ? a.w[t0] : 0.0), (R)(in1 ? a.w[t1] : 0.0));
        T.wy = T2::mk((R)(in0 ? a.w[a.n + t0] : 0.0), (R)(in1 ? a.w[a.n + t1] : 0.0));
        const R g0 = (R)(in0 ? a.G[t0] * kInv2Pi : 0.0), g1 = (R)(in1 ? a.G[t1] * kInv2Pi : 0.0);
        T.g = T2::mk(g0, g1);
        T.ng = T2::mk(-g0, -g1);
        T.dd = T2::mk((R)a.delta, (R)a.delta);
    }
    static __device__ __forceinline__ void pair(const Rec &c, const Tgt &T, V *p) {
        V nx, ny, wx, nwy;
        ld_pair(&c.nx, nx, ny);
        ld_pair(&c.wx, wx, nwy);
        const V a = T2::add(T.x, nx);  // t - s_j
        const V b = T2::add(T.y, ny);
        V r;
        if (MASK) {
            const V d2 = T2::fma(a, a, T2::mul(b, b));
            r = mask_zero(T2::rcp(T2::add(d2, T.dd)), d2);
        } else {
            V s = T2::fma(a, a, T.dd);
            s = T2::fma(b, b, s);
            r = T2::rcp(s);
        }
        if (GX) {
            const V dwx = T2::fma(c.g, T.wx, T2::mul(T.ng, wx));   // gamma_j w_t - gamma_t w_j
            const V dwy = T2::fma(c.g, T.wy, T2::mul(T.g, nwy));
            const V na = T2::mk(-a.x, -a.y);
            const V tt = T2::fma(b, dwx, T2::mul(na, dwy));       // b dwx - a dwy
            const V m = T2::mul(T2::mul(r, r), tt);
            p[0] = T2::fma(r, dwy, p[0]);
            p[1] = T2::fma(a, m, p[1]);
            p[2] = T2::fma(r, dwx, p[2]);
            p[3] = T2::fma(b, m, p[3]);
        }
        if (GG) {
            const V tg = T2::fma(b, wx, T2::mul(a, nwy));  // b w_jx - a w_jy
            p[GX ? 4 : 0] = T2::fma(r, tg, p[GX ? 4 : 0]);
        }
    }
    static __device__ __forceinline__ void finalize(const Args &a, int t, const double *s) {
        if (GX) {
            double o0 = s[0] + 2.0 * s[1], o1 = -s[2] + 2.0 * s[3];
            if (a.lz) {
                o0 = a.lz[t] - a.lhdt * o0;
                o1 = a.lz[a.n + t] - a.lhdt * o1;
            }
            a.gx[t] = o0;
            a.gx[a.n + t] = o1;
        }
        if (GG) a.gG[t] = s[GX ? 4 : 0] * kInv2Pi;
    }
};

// ---------------------------------------------------------------- dispatch
template <typename R>
static int velocity_impl(int nt, const double *xt, int ns, const double *xs, const double *G,
                         double delta, double *f, double *D, cudaStream_t st, const LaunchOpts &o) {
    if (D) {
        typename VelOp<R, true, true>::Args a{nt, ns, xt, xs, G, delta, f, D};
        return launch_pairs<VelOp<R, true, true>>(a, nt, ns, st, o);
    }
    if (delta == 0.0) {
        typename VelOp<R, false, true>::Args a{nt, ns, xt, xs, G, delta, f, nullptr};
        return launch_pairs<VelOp<R, false, true>>(a, nt, ns, st, o);
    }
    typename VelOp<R, false, false>::Args a{nt, ns, xt, xs, G, delta, f, nullptr};
    // FP32 with many targets: 4 target sets per lane (measured on GB300: +8 %
    // at N = 65536, equal at 16384, slower below 8192 where the 256-target
    // blocks leave SMs idle)
    if (sizeof(R) == 4 && nt >= kVelSets4MinTargets) {
        typename VelOp<R, false, false, 4>::Args a4{nt, ns, xt, xs, G, delta, f, nullptr};
        return launch_pairs<VelOp<R, false, false, 4>>(a4, nt, ns, st, o);
    }
    return launch_pairs<VelOp<R, false, false>>(a, nt, ns, st, o);
}

template <typename R>
static int jvp_impl(int n, const double *x, const double *G, double delta, const double *v,
                    double *jv, cudaStream_t st, const LaunchOpts &o) {
    if (delta == 0.0) {
        typename JvpOp<R, true>::Args a{n, x, G, v, delta, jv, o.lin.z, o.lin.hdt};
        return launch_pairs<JvpOp<R, true>>(a, n, n, st, o);
    }
    typename JvpOp<R, false>::Args a{n, x, G, v, delta, jv, o.lin.z, o.lin.hdt};
    return launch_pairs<JvpOp<R, false>>(a, n, n, st, o);
}

template <typename R, bool MASK>
static int vjp_impl2(int n, const double *x, const double *G, double delta, const double *w,
                     double *gx, double *gG, cudaStream_t st, const LaunchOpts &o) {
    if (gx && gG) {
        typename VjpOp<R, MASK, true, true>::Args a{n, x, G, w, delta, gx, gG, o.lin.z, o.lin.hdt};
        return launch_pairs<VjpOp<R, MASK, true, true>>(a, n, n, st, o);
    }
    if (gx) {
        typename VjpOp<R, MASK, true, false>::Args a{n, x, G, w, delta, gx, gG, o.lin.z, o.lin.hdt};
        return launch_pairs<VjpOp<R, MASK, true, false>>(a, n, n, st, o);
    }
    typename VjpOp<R, MASK, false, true>::Args a{n, x, G, w, delta, gx, gG, nullptr, 0.0};
    return launch_pairs<VjpOp<R, MASK, false, true>>(a, n, n, st, o);
}

template <typename R>
static int vjp_impl(int n, const double *x, const double *G, double delta, const double *w,
                    double *gx, double *gG, cudaStream_t st, const LaunchOpts &o) {
    if (delta == 0.0) return vjp_impl2<R, true>(n, x, G, delta, w, gx, gG, st, o);
    return vjp_impl2<R, false>(n, x, G, delta, w, gx, gG, st, o);
}

static int check_common(const char *fn, int nt, int ns, double delta, int prec) {
    if (nt < 1 || ns < 1) return set_error(PTROM_EINVAL, "%s: sizes must be >= 1 (nt=%d ns=%d)", fn, nt, ns);
    if (!(delta >= 0.0)) return set_error(PTROM_EINVAL, "%s: delta must be >= 0", fn);
    if (prec != PTROM_FP32C && prec != PTROM_FP64) return set_error(PTROM_EINVAL, "%s: bad prec %d", fn, prec);
    return PTROM_OK;
}

// Internal entry points used by the solvers (explicit source split for tests).
int velocity(int nt, const double *xt, int ns, const double *xs, const double *G, double delta,
             double *f, double *D, int prec, cudaStream_t st, const LaunchOpts &o) {
    return prec == PTROM_FP64 ? velocity_impl<double>(nt, xt, ns, xs, G, delta, f, D, st, o)
                              : velocity_impl<float>(nt, xt, ns, xs, G, delta, f, D, st, o);
}
int jvp(int n, const double *x, const double *G, double delta, const double *v, double *jv,
        int prec, cudaStream_t st, const LaunchOpts &o) {
    return prec == PTROM_FP64 ? jvp_impl<double>(n, x, G, delta, v, jv, st, o)
                              : jvp_impl<float>(n, x, G, delta, v, jv, st, o);
}
int vjp(int n, const double *x, const double *G, double delta, const double *w, double *gx,
        double *gG, int prec, cudaStream_t st, const LaunchOpts &o) {
    return prec == PTROM_FP64 ? vjp_impl<double>(n, x, G, delta, w, gx, gG, st, o)
                              : vjp_impl<float>(n, x, G, delta, w, gx, gG, st, o);
}
size_t pack_scratch_bytes(int nt, int ns) { return pack_scratch_bytes_impl(nt, ns); }

// Batched velocity over B instances (one pack + one cluster launch).
template <typename R, bool WD, bool MASK>
static int velocity_batched_impl(int B, const int *n, const double *const *x, const double *const *G,
                                 const double *delta, double *const *f, double *const *D, cudaStream_t st, int S) {
    using Op = VelOp<R, WD, MASK>;
    std::vector<typename Op::Args> args(B);
    for (int b = 0; b < B; ++b) args[b] = typename Op::Args{n[b], n[b], x[b], x[b], G[b], delta[b], f[b], WD ? D[b] : nullptr};
    return launch_pairs_batched<Op>(args.data(), n, n, B, st, S);
}

int velocity_batched(int B, const int *n, const double *const *x, const double *const *G, const double *delta,
                     double *const *f, double *const *D, int prec, cudaStream_t st, int S) {
    bool any0 = false, withD = D != nullptr;
    for (int b = 0; b < B; ++b) any0 = any0 || delta[b] == 0.0;
    if (S <= 0) S = 1;
    if (prec == PTROM_FP64) {
        if (withD) return velocity_batched_impl<double, true, true>(B, n, x, G, delta, f, D, st, S);
        if (any0) return velocity_batched_impl<double, false, true>(B, n, x, G, delta, f, D, st, S);
        return velocity_batched_impl<double, false, false>(B, n, x, G, delta, f, D, st, S);
    }
    if (withD) return velocity_batched_impl<float, true, true>(B, n, x, G, delta, f, D, st, S);
    if (any0) return velocity_batched_impl<float, false, true>(B, n, x, G, delta, f, D, st, S);
    return velocity_batched_impl<float, false, false>(B, n, x, G, delta, f, D, st, S);
}

}  // namespace ptrom

using namespace ptrom;

extern "C" int bs_velocity_batched(int B, const int *n, const double *const *x, const double *const *Gamma,
                                   const double *delta, double *const *f_out, double *const *selfjac_out, int prec,
                                   ptrom_stream_t stream) {
    if (B < 1 || !n || !x || !Gamma || !delta || !f_out)
        return set_error(PTROM_EINVAL, "bs_velocity_batched: bad arguments");
    if (prec != PTROM_FP32C && prec != PTROM_FP64) return set_error(PTROM_EINVAL, "bs_velocity_batched: bad prec");
    for (int b = 0; b < B; ++b) {
        if (n[b] < 1 || !x[b] || !Gamma[b] || !f_out[b] || !(delta[b] >= 0.0) || (selfjac_out && !selfjac_out[b]))
            return set_error(PTROM_EINVAL, "bs_velocity_batched: bad instance %d", b);
    }
    const int S = g_source_split.load() > 0 ? g_source_split.load() : 2;
    return velocity_batched(B, n, x, Gamma, delta, f_out, selfjac_out, prec, (cudaStream_t)stream, S);
}

extern "C" int bs_velocity(int nt, const double *xt, int ns, const double *xs, const double *Gamma,
                           double delta, double *f_out, double *selfjac_out, int prec,
                           ptrom_stream_t stream) {
    PTROM_TRY(check_common("bs_velocity", nt, ns, delta, prec));
    if (!xt || !xs || !Gamma || !f_out) return set_error(PTROM_EINVAL, "bs_velocity: NULL array");
    return velocity(nt, xt, ns, xs, Gamma, delta, f_out, selfjac_out, prec, (cudaStream_t)stream);
}

extern "C" int bs_jvp(int n, const double *x, const double *Gamma, double delta, const double *v,
                      double *jv, int prec, ptrom_stream_t stream) {
    PTROM_TRY(check_common("bs_jvp", n, n, delta, prec));
    if (n < 2) return set_error(PTROM_EINVAL, "bs_jvp: n must be >= 2");
    if (!x || !Gamma || !v || !jv) return set_error(PTROM_EINVAL, "bs_jvp: NULL array");
    return jvp(n, x, Gamma, delta, v, jv, prec, (cudaStream_t)stream);
}

extern "C" int bs_vjp(int n, const double *x, const double *Gamma, double delta, const double *w,
                      double *gx_out, double *gGamma_out, int prec, ptrom_stream_t stream) {
    PTROM_TRY(check_common("bs_vjp", n, n, delta, prec));
    if (n < 2) return set_error(PTROM_EINVAL, "bs_vjp: n must be >= 2");
    if (!x || !Gamma || !w) return set_error(PTROM_EINVAL, "bs_vjp: NULL array");
    if (!gx_out && !gGamma_out) return PTROM_OK;
    return vjp(n, x, Gamma, delta, w, gx_out, gGamma_out, prec, (cudaStream_t)stream);
}

extern "C" int ptrom_tune_pairs(int n, int prec, double delta, ptrom_stream_t stream) {
    using namespace ptrom;
    PTROM_TRY(check_common("ptrom_tune_pairs", n, n, delta, prec));
    if (n < 2) return set_error(PTROM_EINVAL, "ptrom_tune_pairs: n must be >= 2");
    cudaStream_t st = (cudaStream_t)stream;
    // synthetic bodies: a jittered lattice in the unit square, Gamma = 1/n, v = w = x;
    // kernel times do not depend on the values
    std::vector<double> h((size_t)2 * n + n);
    const int m = (int)ceil(sqrt((double)n));
    for (int i = 0; i < n; ++i) {
        h[i] = (i % m + 0.37 * ((i * 7919) % 13) / 13.0) / m;
        h[n + i] = (i / m + 0.41 * ((i * 104729) % 17) / 17.0) / m;
        h[2 * (size_t)n + i] = 1.0 / n;
    }
    double *d = nullptr;
    PTROM_TRY(scratch_alloc((void **)&d, sizeof(double) * ((size_t)2 * n + n + (size_t)2 * n + 3 * (size_t)n), st));
    double *x = d, *G = d + 2 * (size_t)n, *out = G + n, *D = out + 2 * (size_t)n;
    cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st);
    int s = e == cudaSuccess ? PTROM_OK : check_cuda(e, "ptrom_tune_pairs: upload");
    LaunchOpts o;
    o.tune = true;
    if (s == PTROM_OK) s = velocity(n, x, n, x, G, delta, out, nullptr, prec, st, o);
    if (s == PTROM_OK) s = velocity(n, x, n, x, G, delta, out, D, prec, st, o);
    if (s == PTROM_OK) s = jvp(n, x, G, delta, x, out, prec, st, o);
    if (s == PTROM_OK) s = vjp(n, x, G, delta, x, out, nullptr, prec, st, o);
    if (s == PTROM_OK) s = vjp(n, x, G, delta, x, out, D, prec, st, o);
    const int s2 = scratch_free(d, st);
    if (s == PTROM_OK) s = s2;
    if (s == PTROM_OK) {
        const cudaError_t es = cudaStreamSynchronize(st);
        if (es != cudaSuccess) s = check_cuda(es, "ptrom_tune_pairs");
    }
    return s;
}

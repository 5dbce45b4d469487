// Internal (C++) entry points shared between translation units of libptrom.so.
#pragma once

#include <cuda_runtime.h>

namespace ptrom {

// Optional epilogue of the J v / J^T w launches: with z != nullptr the
// output is z - hdt * (J v) (the Newton matrix (I - hdt J) applied to z when
// v = z), written in place of J v.
struct LinEpi {
    const double *z = nullptr;
    double hdt = 0.0;
};

// Options of one all-pairs launch (bs_pair.cu):
//   split   0 -> automatic cluster split, S in 1..8 -> forced;
//   scratch device buffer for the packed sources and the split's partial
//           sums, of scratch_bytes bytes (pack_scratch_bytes(nt, ns) bytes
//           always suffice; one that holds the records only makes the launch
//           combine its split through a thread-block cluster), or nullptr
//           (stream-ordered allocation from the pool);
//   lin     J v / J^T w only: the (I - hdt J) epilogue;
//   skip    optional device flag: nonzero at launch -> the launch does nothing;
//   slots   optional: collects the launches' timing slots (so a launch that
//           turned out to be skipped can be left out of the timing totals).
struct Slots {
    int s[16];
    int n = 0;
    void add(int v) {
        if (v >= 0 && n < 16) s[n++] = v;
    }
};
struct LaunchOpts {
    int split = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    LinEpi lin;
    const int *skip = nullptr;
    Slots *slots = nullptr;
    bool tune = false;  // autotune this launch's split if it has no cached value
};

int velocity(int nt, const double *xt, int ns, const double *xs, const double *G, double delta,
             double *f, double *D, int prec, cudaStream_t st, const LaunchOpts &o = {});
int jvp(int n, const double *x, const double *G, double delta, const double *v, double *jv,
        int prec, cudaStream_t st, const LaunchOpts &o = {});
int vjp(int n, const double *x, const double *G, double delta, const double *w, double *gx,
        double *gG, int prec, cudaStream_t st, const LaunchOpts &o = {});
size_t pack_scratch_bytes(int nt, int ns);
// Bytes per source that bs_velocity_noalloc's fixed scratch reserves: the
// largest packed record of any velocity kernel (checked at compile time in
// bs_pair.cu against every VelOp record).
constexpr size_t kNoAllocRecordBytes = 48;
// Batched velocity (+ self blocks when D != nullptr) over B instances; S = source split.
int velocity_batched(int B, const int *n, const double *const *x, const double *const *G, const double *delta,
                     double *const *f, double *const *D, int prec, cudaStream_t st, int S);
// J Phi (jphi.cu); split = source split over gridDim.z (0 = automatic).
int jphi(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out, int prec,
         cudaStream_t st, int split);
// J Phi on the tensor cores, TF32 split in three (jphi_tc.cu); split as jphi.
int jphi_tc(int n, const double *x, const double *G, double delta, const double *phi, int M, double *out,
            cudaStream_t st, int split);

}  // namespace ptrom

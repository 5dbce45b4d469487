// bs_velocity_noalloc: the velocity sum of bs_velocity for callers that must
// not allocate device memory at call time.
//
// bs_velocity packs its sources into a scratch buffer that it takes, stream-
// ordered, from a library memory pool.  Some callers cannot allow that: a
// control or serving loop whose memory policy forbids any device allocation
// after start-up (an allocation can block, fail under memory pressure, or
// change the memory footprint mid-run), or a host process whose device memory
// is owned by another framework's allocator.  This entry point instead keeps
// the packed sources in one fixed array compiled into the library
// (kNoAllocMaxSources sources, 3 MiB), which every GPU that loads the library
// holds until the process exits.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace ptrom {
namespace {

constexpr int kNoAllocMaxSources = PTROM_NOALLOC_MAX_SOURCES;
// kNoAllocRecordBytes (internal.h): the largest packed-source record of the
// velocity kernels, the FP64 one (three 16-byte pairs; FP32 records are 32
// bytes), tied to the records' sizes by static_asserts in bs_pair.cu.
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxSources * kNoAllocRecordBytes;

// The shared scratch.  In host code this name is only a stand-in for the
// device object, never a device address: the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (the first call on a device does this set-up).
int noalloc_scratch(void **out) {
    int dev = 0;
    PTROM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(PTROM_EINVAL, "bs_velocity_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return check_cuda(e, "bs_velocity_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PTROM_OK;
}

}  // namespace
}  // namespace ptrom

extern "C" int bs_velocity_noalloc(int nt, const double *xt, int ns, const double *xs, const double *Gamma,
                                   double delta, double *f_out, double *selfjac_out, int prec,
                                   ptrom_stream_t stream) {
    using namespace ptrom;
    if (nt < 1 || ns < 1)
        return set_error(PTROM_EINVAL, "bs_velocity_noalloc: sizes must be >= 1 (nt=%d ns=%d)", nt, ns);
    if (ns > kNoAllocMaxSources)
        return set_error(PTROM_EINVAL,
                         "bs_velocity_noalloc: ns=%d exceeds the fixed scratch limit of %d sources "
                         "(use bs_velocity)", ns, kNoAllocMaxSources);
    if (!(delta >= 0.0)) return set_error(PTROM_EINVAL, "bs_velocity_noalloc: delta must be >= 0");
    if (prec != PTROM_FP32C && prec != PTROM_FP64)
        return set_error(PTROM_EINVAL, "bs_velocity_noalloc: bad prec %d", prec);
    if (!xt || !xs || !Gamma || !f_out) return set_error(PTROM_EINVAL, "bs_velocity_noalloc: NULL array");
    void *scratch = nullptr;
    PTROM_TRY(noalloc_scratch(&scratch));
    // The pack kernel rewrites every record the pair kernel reads (all
    // ceil(ns/32)*32 of them, padding included) before it is read, and, when
    // the rest of the array holds the split's partial sums, zeroes their
    // arrival counters; so nothing in the array needs clearing between calls.
    // When the partials do not fit beside the records, the launch combines its
    // source split through a thread-block cluster instead.
    LaunchOpts o;
    o.scratch = scratch;
    o.scratch_bytes = kNoAllocBytes;
    return velocity(nt, xt, ns, xs, Gamma, delta, f_out, selfjac_out, prec, (cudaStream_t)stream, o);
}

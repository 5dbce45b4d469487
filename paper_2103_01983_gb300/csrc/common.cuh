// Shared helpers of libptrom.so: status/error reporting, launch geometry,
// FP32 packed arithmetic and compensated (TwoSum) accumulation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/ptrom.h"

namespace ptrom {

// ---- status --------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
int check_cuda(cudaError_t e, const char *what);
#define PTROM_CUDA(call)                                          \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return ::ptrom::check_cuda(_e, #call); \
    } while (0)
#define PTROM_TRY(expr)              \
    do {                             \
        int _s = (expr);             \
        if (_s != PTROM_OK) return _s; \
    } while (0)

int device_sm_count();
extern std::atomic<int> g_source_split;  // 0 = automatic
extern std::atomic<int> g_split_mode;    // 0 = automatic, 1 = cluster combine, 2 = global combine
extern std::atomic<int> g_autotune;      // 1: tune the all-pairs source split on first use
// Cached autotuned source split of a pair kernel at (nt, ns); 0 when none.
int tuned_split(const void *kernel, int nt, int ns);
void store_tuned_split(const void *kernel, int nt, int ns, int S);
extern std::atomic<long long> g_launches;  // kernels launched by the library
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }
// Stream-ordered scratch from a library-owned memory pool per device whose
// release threshold keeps freed blocks cached (so a steady stream of calls
// does not map and unmap memory at every synchronisation).
int scratch_alloc(void **ptr, size_t bytes, cudaStream_t st);
int scratch_free(void *ptr, cudaStream_t st);
int scratch_trim();  // release the current device pool's cached blocks
// CUDA-event timing of one launch (no-op unless ptrom_timing_enable(1)).
int timing_begin(int kind, cudaStream_t st);
void timing_end(int slot, cudaStream_t st);
void timing_discard(int slot);  // leave a launch out of the totals (it did no work)
// Per-thread, per-device pinned host buffer of at least `ndoubles` doubles and
// `nevents` events (timing disabled): small device-to-host status reads that
// the host waits for on an event while later work stays queued.
int host_mailbox(size_t ndoubles, int nevents, double **host, cudaEvent_t **events);

constexpr double kInv2Pi = 0.15915494309189533576888376337251;  // 1 / (2 pi)

// ---- FP32 helpers (device) ------------------------------------------------
// MUFU reciprocal, ~1 ulp, flushes subnormals.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) { return f2(rcp_approx(a.x), rcp_approx(a.y)); }

// Compensated accumulator: value = hi + lo, updated with Knuth's TwoSum
// (error-free transformation of one FP32 addition).  Used once per chunk of
// sources, after a plain FP32 partial sum over the chunk.
struct CSum2 {
    float2 hi, lo;
    __device__ __forceinline__ void zero() { hi = f2(0.f, 0.f); lo = f2(0.f, 0.f); }
    __device__ __forceinline__ void add(float2 p) {
        float2 s = add2(hi, p);
        float2 bb = add2(s, f2(-hi.x, -hi.y));
        float2 e1 = add2(hi, f2(-(s.x - bb.x), -(s.y - bb.y)));
        float2 e2 = add2(p, f2(-bb.x, -bb.y));
        lo = add2(lo, add2(e1, e2));
        hi = s;
    }
    __device__ __forceinline__ double x() const { return (double)hi.x + (double)lo.x; }
    __device__ __forceinline__ double y() const { return (double)hi.y + (double)lo.y; }
};

}  // namespace ptrom

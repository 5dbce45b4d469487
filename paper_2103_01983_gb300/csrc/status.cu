// Status codes and per-thread error messages of the C ABI.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace ptrom {

static thread_local char g_msg[512] = "no error";
static thread_local int g_code = PTROM_OK;

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    g_code = code;
    return code;
}

int check_cuda(cudaError_t e, const char *what) {
    return set_error(PTROM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cached[dev] = v;
    }
    return cached[dev];
}

}  // namespace ptrom

extern "C" int ptrom_last_error(char *buf, size_t len) {
    if (buf && len) {
        strncpy(buf, ptrom::g_msg, len - 1);
        buf[len - 1] = '\0';
    }
    return ptrom::g_code;
}

extern "C" int ptrom_version(void) { return 100; }

namespace ptrom {
std::atomic<int> g_source_split{0};
}

extern "C" int ptrom_set_source_split(int S) {
    if (S < 0 || S > 16) return ptrom::set_error(PTROM_EINVAL, "ptrom_set_source_split: S=%d outside [0, 16]", S);
    ptrom::g_source_split.store(S);
    return PTROM_OK;
}

namespace ptrom {
std::atomic<int> g_split_mode{0};
std::atomic<int> g_autotune{0};
static std::mutex g_tune_mu;
static std::map<std::tuple<const void *, int, int, int>, int> g_tuned;  // (kernel, device, nt, ns) -> S

int tuned_split(const void *kernel, int nt, int ns) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tuned.find(std::make_tuple(kernel, dev, nt, ns));
    return it == g_tuned.end() ? 0 : it->second;
}

void store_tuned_split(const void *kernel, int nt, int ns, int S) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(kernel, dev, nt, ns)] = S;
}
}  // namespace ptrom

extern "C" int ptrom_set_autotune(int on) {
    if (on < 0 || on > 1) return ptrom::set_error(PTROM_EINVAL, "ptrom_set_autotune: on=%d outside [0, 1]", on);
    ptrom::g_autotune.store(on);
    return PTROM_OK;
}

extern "C" int ptrom_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(ptrom::g_tune_mu);
    ptrom::g_tuned.clear();
    return PTROM_OK;
}

extern "C" int ptrom_set_split_mode(int mode) {
    if (mode < 0 || mode > 2) return ptrom::set_error(PTROM_EINVAL, "ptrom_set_split_mode: mode=%d outside [0, 2]", mode);
    ptrom::g_split_mode.store(mode);
    return PTROM_OK;
}

// ---------------------------------------------------------------- instrumentation
namespace ptrom {
std::atomic<long long> g_launches{0};
static std::atomic<int> g_timing{0};
static std::mutex g_tmu;
static std::vector<cudaEvent_t> g_ev;       // pairs (start, stop)
static std::vector<int> g_kind;
static size_t g_used = 0;
constexpr size_t kMaxTimed = 65536;

bool timing_active() { return g_timing.load(std::memory_order_relaxed) != 0; }

int timing_begin(int kind, cudaStream_t st) {
    const int mask = g_timing.load(std::memory_order_relaxed);
    if (!mask || kind < 0 || kind >= 31 || !(mask & (1 << kind))) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_used >= kMaxTimed) return -1;
    while (g_ev.size() < 2 * (g_used + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        g_ev.push_back(e);
    }
    const int slot = (int)g_used++;
    if ((int)g_kind.size() <= slot) g_kind.resize(slot + 1);
    g_kind[slot] = kind;
    cudaEventRecord(g_ev[2 * slot], st);
    return slot;
}

void timing_end(int slot, cudaStream_t st) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    cudaEventRecord(g_ev[2 * slot + 1], st);
}

void timing_discard(int slot) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    if ((size_t)slot < g_used && (size_t)slot < g_kind.size()) g_kind[slot] = -1;
}

namespace {
struct Mailbox {
    double *host = nullptr;
    size_t n = 0;
    std::vector<cudaEvent_t> ev;
    ~Mailbox() {
        if (host) cudaFreeHost(host);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};
thread_local Mailbox t_mailbox[64];
}  // namespace

int host_mailbox(size_t ndoubles, int nevents, double **host, cudaEvent_t **events) {
    int dev = 0;
    PTROM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(PTROM_EINVAL, "host_mailbox: device %d out of range", dev);
    Mailbox &mb = t_mailbox[dev];
    if (mb.n < ndoubles) {
        if (mb.host) cudaFreeHost(mb.host);
        mb.host = nullptr;
        mb.n = 0;
        PTROM_CUDA(cudaHostAlloc((void **)&mb.host, sizeof(double) * ndoubles, cudaHostAllocDefault));
        mb.n = ndoubles;
    }
    while ((int)mb.ev.size() < nevents) {
        cudaEvent_t e;
        PTROM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        mb.ev.push_back(e);
    }
    *host = mb.host;
    *events = mb.ev.data();
    return PTROM_OK;
}
}  // namespace ptrom

extern "C" long long ptrom_launch_count(void) { return ptrom::g_launches.load(); }

extern "C" int ptrom_timing_enable(int on) {
    ptrom::g_timing.store(on == 1 ? 0x7fffffff : (on > 0 ? on : 0));
    return PTROM_OK;
}

extern "C" int ptrom_timing_read(double *ms, long long *count, int nkinds) {
    using namespace ptrom;
    if (!ms || !count || nkinds < 1) return set_error(PTROM_EINVAL, "ptrom_timing_read: bad arguments");
    for (int k = 0; k < nkinds; ++k) { ms[k] = 0.0; count[k] = 0; }
    std::lock_guard<std::mutex> lk(g_tmu);
    for (size_t i = 0; i < g_used; ++i) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(g_ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, g_ev[2 * i], g_ev[2 * i + 1]);
        if (e != cudaSuccess) { g_used = 0; return check_cuda(e, "ptrom_timing_read"); }
        const int k = g_kind[i];
        if (k >= 0 && k < nkinds) { ms[k] += t; count[k] += 1; }
    }
    g_used = 0;
    return PTROM_OK;
}

// ---------------------------------------------------------------- scratch pool
namespace ptrom {
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static int pool_for_current(cudaMemPool_t *out) {
    int dev = 0;
    PTROM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(PTROM_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        PTROM_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;
        PTROM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return PTROM_OK;
}

int scratch_alloc(void **ptr, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool;
    PTROM_TRY(pool_for_current(&pool));
    PTROM_CUDA(cudaMallocFromPoolAsync(ptr, bytes, pool, st));
    return PTROM_OK;
}

int scratch_free(void *ptr, cudaStream_t st) {
    PTROM_CUDA(cudaFreeAsync(ptr, st));
    return PTROM_OK;
}

int scratch_trim() {
    cudaMemPool_t pool;
    PTROM_TRY(pool_for_current(&pool));
    PTROM_CUDA(cudaMemPoolTrimTo(pool, 0));
    return PTROM_OK;
}
}  // namespace ptrom

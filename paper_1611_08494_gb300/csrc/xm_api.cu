// xm_api.cu -- runtime of the C ABI: status strings, last-error text,
// allocator hook, counters, kernel timing, and the galactic frame rotation.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "xm_internal.cuh"

namespace xm {

namespace {

thread_local char g_err[512] = "";

struct AllocHook {
    void* (*alloc)(size_t, void*, void*) = nullptr;
    void (*release)(void*, void*, void*) = nullptr;
    void* ctx = nullptr;
};
AllocHook g_hook;
std::mutex g_hook_mu;

std::atomic<unsigned long long> g_stats[6];

struct ProfPending {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfPending> g_pending;
std::vector<cudaEvent_t> g_event_pool;
std::map<std::string, std::pair<double, int64_t>> g_prof_tot;
thread_local cudaEvent_t t_begin = nullptr;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void drain_locked() {
    for (auto& p : g_pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            auto& t = g_prof_tot[p.name];
            t.first += ms;
            t.second += 1;
        }
        g_event_pool.push_back(p.a);
        g_event_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

xm_status set_error(xm_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

xm_status cuda_fail(cudaError_t e, const char* what) {
    return set_error(XM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---- device memory
//
// Blocks the library frees are kept per device for reuse instead of going
// back to the stream-ordered pool at once: taking a block of gigabytes from
// the pool was measured to hold the calling thread for 10-60 ms while copies
// ran on the copy engines (whether the pool reused freed memory or grew), and
// a pipelined caller allocates and frees blocks of the same sizes every step.
// A kept block carries an event recorded on the freeing stream at the free
// point. An allocation takes the smallest kept block of at least its size
// (and at most about twice it) that is already free on the GPU: its event has
// completed, or it was freed on the allocating stream (stream order covers
// it). The allocating stream waits on that event (a no-op then, and still
// correct if a destroyed stream's handle was handed out again). Failing that
// the block comes from the pool; when the pool has no memory left, kept
// blocks still in use on other streams are taken (the allocating stream
// waits for them on the GPU), and then every kept block goes back to the pool
// before one more try. The kept total is capped (half the device's memory
// unless xm_set_cache_limit says otherwise); past it the oldest blocks go
// back first. While a stream is being captured into a graph its allocations
// and frees go to the pool directly.
namespace {

struct Kept {
    void* p;
    size_t bytes;
    cudaStream_t s;
    cudaEvent_t ev;
    bool done;  // ev known to have completed
    uint64_t age;
};

struct DevMem {
    std::mutex mu;
    bool ready = false;
    std::unordered_map<void*, size_t> live;  // blocks handed out -> size
    std::vector<Kept> kept;
    std::vector<cudaEvent_t> spare;
    size_t live_bytes = 0, kept_bytes = 0, total = 0;
    uint64_t tick = 0;
};

DevMem g_mem[64];
std::atomic<long long> g_cache_limit{-1};  // bytes; < 0: half the device's memory

size_t round_block(size_t b) {
    if (b == 0) b = 1;
    const size_t g = b <= (size_t(1) << 20) ? 512 : (size_t(2) << 20);
    return (b + g - 1) / g * g;
}

size_t cache_limit(const DevMem& d) {
    const long long l = g_cache_limit.load();
    return l < 0 ? d.total / 2 : (size_t)l;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

// First use on a device: the pool keeps what goes back to it (release
// threshold raised) and the device's size sets the default cap.
void mem_init(DevMem& d, int dev) {
    if (d.ready) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) cudaGetLastError();
    d.total = tot;
    d.ready = true;
}

// Kept block i goes back to the pool, ordered after its free point on `s`.
void give_back(DevMem& d, size_t i, cudaStream_t s) {
    const Kept k = d.kept[i];
    d.kept[i] = d.kept.back();
    d.kept.pop_back();
    d.kept_bytes -= k.bytes;
    bool done = k.done;
    if (!done) {
        const cudaError_t q = cudaEventQuery(k.ev);
        if (q == cudaSuccess) done = true;
        else if (q != cudaErrorNotReady) cudaGetLastError();
    }
    if (!done && cudaStreamWaitEvent(s, k.ev, 0) != cudaSuccess) cudaGetLastError();
    if (cudaFreeAsync(k.p, s) != cudaSuccess) cudaGetLastError();
    d.spare.push_back(k.ev);
}

// A kept block of `need` bytes or a little more for stream `s`; with
// `pending`, also one still in use on another stream.
void* take(DevMem& d, size_t need, cudaStream_t s, bool pending) {
    const size_t most = 2 * need + (size_t(1) << 20);
    long best = -1;
    for (size_t i = 0; i < d.kept.size(); i++) {
        Kept& k = d.kept[i];
        if (k.bytes < need || k.bytes > most) continue;
        if (best >= 0 && k.bytes >= d.kept[best].bytes) continue;
        if (!k.done && k.s != s && !pending) {
            const cudaError_t q = cudaEventQuery(k.ev);
            if (q == cudaSuccess) {
                k.done = true;
            } else {
                if (q != cudaErrorNotReady) cudaGetLastError();
                continue;
            }
        }
        best = (long)i;
    }
    if (best < 0) return nullptr;
    const Kept k = d.kept[best];
    if (!k.done && cudaStreamWaitEvent(s, k.ev, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    d.kept[best] = d.kept.back();
    d.kept.pop_back();
    d.kept_bytes -= k.bytes;
    d.spare.push_back(k.ev);
    d.live[k.p] = k.bytes;
    d.live_bytes += k.bytes;
    return k.p;
}

void* pool_alloc(DevMem& d, size_t need, cudaStream_t s) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, need, s) != cudaSuccess) {
        cudaGetLastError();  // clear the error state of a failed allocation
        return nullptr;
    }
    d.live[p] = need;
    d.live_bytes += need;
    return p;
}

}  // namespace

// Pinned, mapped staging areas for small device -> host reads, one per
// HostReads object while it lives (taken from a pool, each with an event).
// A kernel writes the values into the area instead of a device-to-host
// copy: such copies from all streams queue in order on one copy engine, so a
// count read would wait behind whatever large result copies the caller has
// queued on other streams (a pipelined caller copying one step's results out
// while the next step's match reads its pair count). An area goes back to
// the pool with its event recorded after its last kernel, and is handed out
// again only once that event has completed.
namespace {
constexpr size_t kStageBytes = 4096;
std::mutex g_stage_mu;
std::vector<HostReads::Area> g_stage_free;

bool take_area(HostReads::Area* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    {
        std::lock_guard<std::mutex> g(g_stage_mu);
        for (size_t i = 0; i < g_stage_free.size(); i++) {
            if (g_stage_free[i].dev != dev) continue;
            const cudaError_t q = cudaEventQuery(g_stage_free[i].ev);
            if (q != cudaSuccess) {
                if (q != cudaErrorNotReady) cudaGetLastError();
                continue;
            }
            *out = g_stage_free[i];
            g_stage_free[i] = g_stage_free.back();
            g_stage_free.pop_back();
            return true;
        }
    }
    HostReads::Area A{};
    A.dev = dev;
    void* p = nullptr;
    void* dp = nullptr;
    if (cudaHostAlloc(&p, kStageBytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess ||
        cudaHostGetDevicePointer(&dp, p, 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&A.ev, cudaEventDisableTiming) != cudaSuccess) {
        if (p) cudaFreeHost(p);
        cudaGetLastError();  // no mapped pinned memory: plain copies instead
        return false;
    }
    A.p = (unsigned char*)p;
    A.dp = (unsigned char*)dp;
    *out = A;
    return true;
}

// The queued small reads, copied byte by byte into the mapped staging area.
struct StageCopies {
    const unsigned char* src[8];
    uint32_t off[8], bytes[8];
    int n;
};

__global__ void k_stage_copy(StageCopies c, unsigned char* __restrict__ dst) {
    for (int k = 0; k < c.n; k++)
        for (uint32_t b = threadIdx.x; b < c.bytes[k]; b += blockDim.x) dst[c.off[k] + b] = c.src[k][b];
    __threadfence_system();
}
}  // namespace

HostReads::~HostReads() {
    if (!have_) return;
    // a kernel still to run writes into the area: its event marks the end
    if (launched_ && !synced_ && cudaEventRecord(area_.ev, s_) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(s_);
    }
    std::lock_guard<std::mutex> g(g_stage_mu);
    g_stage_free.push_back(area_);
}

cudaError_t HostReads::add(void* host_dst, const void* dev_src, size_t bytes) {
    if (!tried_) {
        tried_ = true;
        have_ = take_area(&area_);
    }
    const size_t off = (used_ + 15) & ~size_t(15);
    if (!have_ || n_ == 8 || off + bytes > kStageBytes)  // (blocks until the copy is done)
        return cudaMemcpyAsync(host_dst, dev_src, bytes, cudaMemcpyDeviceToHost, s_);
    items_[n_++] = Item{host_dst, dev_src, off, bytes};
    used_ = off + bytes;
    launched_ = false;
    synced_ = false;
    return cudaSuccess;
}

cudaError_t HostReads::launch() {
    if (launched_ || n_ == 0) return cudaSuccess;
    StageCopies c{};
    c.n = n_;
    for (int i = 0; i < n_; i++) {
        c.src[i] = (const unsigned char*)items_[i].src;
        c.off[i] = (uint32_t)items_[i].off;
        c.bytes[i] = (uint32_t)items_[i].bytes;
    }
    k_stage_copy<<<1, 128, 0, s_>>>(c, area_.dp);
    launched_ = true;
    return cudaGetLastError();
}

cudaError_t HostReads::mark() {
    const cudaError_t el = launch();
    if (el != cudaSuccess) return el;
    if (!have_) return cudaSuccess;  // sync() waits for the whole stream
    const cudaError_t e = cudaEventRecord(area_.ev, s_);
    marked_ = e == cudaSuccess;
    return e;
}

cudaError_t HostReads::sync() {
    cudaError_t e = launch();
    if (e != cudaSuccess) return e;
    e = marked_ ? cudaEventSynchronize(area_.ev) : cudaStreamSynchronize(s_);
    marked_ = false;
    if (e != cudaSuccess) return e;
    synced_ = true;
    for (int i = 0; i < n_; i++) memcpy(items_[i].dst, area_.p + items_[i].off, items_[i].bytes);
    n_ = 0;
    used_ = 0;
    return cudaSuccess;
}

Side* side_stream() {
    static thread_local Side sd[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    Side& d = sd[dev];
    if (!d.st) {
        const bool ok = cudaStreamCreateWithFlags(&d.st, cudaStreamNonBlocking) == cudaSuccess &&
                        cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming) == cudaSuccess &&
                        cudaEventCreateWithFlags(&d.join, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            d = Side();
            return nullptr;
        }
    }
    return &d;
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 1;
    AllocHook h;
    {
        std::lock_guard<std::mutex> g(g_hook_mu);
        h = g_hook;
    }
    if (h.alloc) return h.alloc(bytes, (void*)s, h.ctx);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    DevMem& d = g_mem[dev];
    std::lock_guard<std::mutex> g(d.mu);
    mem_init(d, dev);
    if (capturing(s)) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;  // not recorded: its free goes to the pool as well
    }
    const size_t need = round_block(bytes);
    void* p = take(d, need, s, false);
    if (!p) p = pool_alloc(d, need, s);
    if (!p) p = take(d, need, s, true);
    if (!p) {
        while (!d.kept.empty()) give_back(d, d.kept.size() - 1, s);
        p = pool_alloc(d, need, s);
    }
    return p;
}

void dev_free(void* p, cudaStream_t s) {
    if (!p) return;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        cur = 0;
    }
    // the device whose cache handed the block out (the current one, as a rule)
    for (int k = 0; k < 64; k++) {
        const int dev = k == 0 ? cur : (k <= cur ? k - 1 : k);
        if (dev < 0 || dev >= 64) continue;
        DevMem& d = g_mem[dev];
        std::lock_guard<std::mutex> g(d.mu);
        if (!d.ready) continue;
        auto it = d.live.find(p);
        if (it == d.live.end()) continue;
        const size_t bytes = it->second;
        d.live.erase(it);
        d.live_bytes -= bytes;
        if (dev != cur) cudaSetDevice(dev);
        cudaEvent_t ev = nullptr;
        if (!d.spare.empty()) {
            ev = d.spare.back();
            d.spare.pop_back();
        } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            ev = nullptr;
        }
        const size_t limit = cache_limit(d);
        if (!ev || bytes > limit || capturing(s) || cudaEventRecord(ev, s) != cudaSuccess) {
            cudaGetLastError();
            if (ev) d.spare.push_back(ev);
            if (cudaFreeAsync(p, s) != cudaSuccess) cudaGetLastError();
        } else {
            d.kept.push_back(Kept{p, bytes, s, ev, false, ++d.tick});
            d.kept_bytes += bytes;
            while (d.kept_bytes > limit && !d.kept.empty()) {
                size_t old = 0;
                for (size_t i = 1; i < d.kept.size(); i++)
                    if (d.kept[i].age < d.kept[old].age) old = i;
                give_back(d, old, s);
            }
        }
        if (dev != cur) cudaSetDevice(cur);
        return;
    }
    AllocHook h;
    {
        std::lock_guard<std::mutex> g(g_hook_mu);
        h = g_hook;
    }
    if (h.release) {
        h.release(p, (void*)s, h.ctx);
        return;
    }
    cudaFreeAsync(p, s);
}

size_t kept_device_bytes() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    DevMem& d = g_mem[dev];
    std::lock_guard<std::mutex> g(d.mu);
    return d.kept_bytes;
}

void launch_begin(const char* name, cudaStream_t s) {
    (void)name;
    g_stats[5].fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_on) {
        t_begin = nullptr;
        return;
    }
    t_begin = take_event();
    if (t_begin) cudaEventRecord(t_begin, s);
}

cudaError_t launch_end(const char* name, cudaStream_t s) {
    cudaError_t e = cudaGetLastError();
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (g_prof_on && t_begin) {
        cudaEvent_t b = take_event();
        if (b) {
            cudaEventRecord(b, s);
            g_pending.push_back({name, t_begin, b});
        } else {
            g_event_pool.push_back(t_begin);
        }
    }
    t_begin = nullptr;
    return e;
}

void stats_add(const unsigned long long* c) {
    for (int k = 0; k < 5; k++) g_stats[k].fetch_add(c[k], std::memory_order_relaxed);
}

// Per-device counters the kernels add to directly (candidates, rechecked,
// flipped, members, tie_resolved, keys x sort passes), so no call waits just
// to read them.
static unsigned long long* g_dev_stats[64] = {};
static std::mutex g_dev_stats_mu;

unsigned long long* device_stats() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(g_dev_stats_mu);
    if (!g_dev_stats[dev]) {
        void* p = nullptr;
        if (cudaMalloc(&p, 8 * sizeof(unsigned long long)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, 8 * sizeof(unsigned long long));
        g_dev_stats[dev] = (unsigned long long*)p;
    }
    return g_dev_stats[dev];
}

static void device_stats_read(unsigned long long out[7]) {
    for (int k = 0; k < 7; k++) out[k] = 0;
    std::lock_guard<std::mutex> g(g_dev_stats_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < 64; d++) {
        if (!g_dev_stats[d]) continue;
        unsigned long long h[8];
        cudaSetDevice(d);
        if (cudaMemcpy(h, g_dev_stats[d], sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess)
            for (int k = 0; k < 7; k++) out[k] += h[k];
    }
    cudaSetDevice(cur);
}

static void device_stats_reset() {
    std::lock_guard<std::mutex> g(g_dev_stats_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < 64; d++) {
        if (!g_dev_stats[d]) continue;
        cudaSetDevice(d);
        cudaMemset(g_dev_stats[d], 0, 8 * sizeof(unsigned long long));
    }
    cudaSetDevice(cur);
}

// Galactic -> equatorial rotation from the IAU frame angles (north galactic
// pole at RA 192.85948 deg, Dec 27.12825 deg; galactic longitude of the north
// celestial pole 122.93192 deg), as the product of three axis rotations:
// turn the equatorial x axis onto the ascending node of the galactic plane
// (RA_NGP + 90 deg), tilt the pole by 90 deg - Dec_NGP about that node, then
// turn within the galactic plane so the node sits at longitude l_NCP - 90 deg.
void gal_to_eq(double m[9]) {
    const double ra_ngp = 192.85948 * kDeg, dec_ngp = 27.12825 * kDeg;
    const double l_node = (122.93192 - 90.0) * kDeg;
    auto rz = [](double ang, double r[9]) {
        double c = cos(ang), s = sin(ang);
        double t[9] = {c, s, 0, -s, c, 0, 0, 0, 1};
        memcpy(r, t, sizeof(t));
    };
    auto rx = [](double ang, double r[9]) {
        double c = cos(ang), s = sin(ang);
        double t[9] = {1, 0, 0, 0, c, s, 0, -s, c};
        memcpy(r, t, sizeof(t));
    };
    auto mul = [](const double* a, const double* b, double* c) {
        double t[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                t[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
        memcpy(c, t, sizeof(t));
    };
    double r1[9], r2[9], r3[9], tmp[9], e2g[9];
    rz(ra_ngp + 0.5 * kPi, r1);
    rx(0.5 * kPi - dec_ngp, r2);
    rz(-l_node, r3);
    mul(r2, r1, tmp);
    mul(r3, tmp, e2g);  // v_gal = e2g v_eq
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) m[3 * i + j] = e2g[3 * j + i];
}

}  // namespace xm

using namespace xm;

extern "C" const char* xm_status_str(xm_status s) {
    switch (s) {
        case XM_OK: return "ok";
        case XM_EINVAL: return "invalid argument";
        case XM_ENOMEM: return "out of memory";
        case XM_ECUDA: return "CUDA error";
        case XM_ETIMEOUT: return "timed out";
        case XM_EOVERFLOW: return "overflow";
        case XM_EBUSY: return "busy (admission refused)";
        case XM_EUNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

extern "C" const char* xm_last_error(void) { return g_err; }

extern "C" const char* xm_version(void) { return "xm 0.1 (sm_103a)"; }

extern "C" xm_status xm_set_allocator(void* (*alloc)(size_t, void*, void*),
                                      void (*release)(void*, void*, void*), void* ctx) {
    if ((alloc == nullptr) != (release == nullptr))
        return set_error(XM_EINVAL, "xm_set_allocator: give both functions or neither");
    std::lock_guard<std::mutex> g(g_hook_mu);
    g_hook.alloc = alloc;
    g_hook.release = release;
    g_hook.ctx = ctx;
    return XM_OK;
}

extern "C" xm_status xm_set_cache_limit(int64_t bytes) {
    g_cache_limit.store(bytes < 0 ? -1 : (long long)bytes);
    return XM_OK;
}

extern "C" xm_status xm_free_cached(void* stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(XM_EINVAL, "xm_free_cached: device %d", dev);
    DevMem& d = g_mem[dev];
    std::lock_guard<std::mutex> g(d.mu);
    while (!d.kept.empty()) give_back(d, d.kept.size() - 1, (cudaStream_t)stream);
    e = cudaGetLastError();
    return e == cudaSuccess ? XM_OK : cuda_fail(e, "xm_free_cached");
}

extern "C" xm_status xm_mem_info(int64_t* live_bytes, int64_t* kept_bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(XM_EINVAL, "xm_mem_info: device %d", dev);
    DevMem& d = g_mem[dev];
    std::lock_guard<std::mutex> g(d.mu);
    if (live_bytes) *live_bytes = (int64_t)d.live_bytes;
    if (kept_bytes) *kept_bytes = (int64_t)d.kept_bytes;
    return XM_OK;
}

extern "C" xm_status xm_get_stats(xm_stats* out) {
    if (!out) return set_error(XM_EINVAL, "xm_get_stats: NULL");
    unsigned long long d[7];
    device_stats_read(d);  // waits for the kernels that add to them
    out->candidates = g_stats[0].load() + d[0];
    out->rechecked = g_stats[1].load() + d[1];
    out->flipped = g_stats[2].load() + d[2];
    out->members = g_stats[3].load() + d[3];
    out->tie_resolved = g_stats[4].load() + d[4];
    out->kernel_launches = g_stats[5].load();
    out->sort_key_passes = d[5];
    out->sort_pay_passes = d[6];
    return XM_OK;
}

extern "C" xm_status xm_reset_stats(void) {
    for (auto& c : g_stats) c.store(0);
    device_stats_reset();
    return XM_OK;
}

extern "C" xm_status xm_prof_enable(int32_t on) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    drain_locked();
    g_prof_tot.clear();
    g_prof_on = on != 0;
    return XM_OK;
}

extern "C" xm_status xm_prof_read(const char* kernel, double* total_ms, int64_t* launches) {
    if (!kernel) return set_error(XM_EINVAL, "xm_prof_read: NULL name");
    std::lock_guard<std::mutex> g(g_prof_mu);
    drain_locked();
    auto it = g_prof_tot.find(kernel);
    if (total_ms) *total_ms = it == g_prof_tot.end() ? 0.0 : it->second.first;
    if (launches) *launches = it == g_prof_tot.end() ? 0 : it->second.second;
    return XM_OK;
}

extern "C" xm_status xm_prof_entry(int32_t i, const char** kernel, double* total_ms,
                                   int64_t* launches) {
    std::lock_guard<std::mutex> g(g_prof_mu);
    drain_locked();
    if (i < 0 || i >= (int32_t)g_prof_tot.size()) return XM_EOVERFLOW;
    auto it = g_prof_tot.begin();
    std::advance(it, i);
    if (kernel) *kernel = it->first.c_str();
    if (total_ms) *total_ms = it->second.first;
    if (launches) *launches = it->second.second;
    return XM_OK;
}

extern "C" xm_status xm_copy_to_host(void* dst, const void* src, size_t bytes, void* stream) {
    if (bytes == 0) return XM_OK;
    if (!dst || !src) return set_error(XM_EINVAL, "xm_copy_to_host: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "xm_copy_to_host");
    return XM_OK;
}

// Host-only: the library's galactic -> equatorial rotation (row major).
extern "C" xm_status xm_frame_matrix(double m[9]) {
    if (!m) return set_error(XM_EINVAL, "xm_frame_matrix: NULL");
    gal_to_eq(m);
    return XM_OK;
}

// xm_batch.cu -- many cross-match requests against one resident index in one
// pass (the batching pattern on top of paper §2.1-§2.3).
//
// The A sources of all requests form one batch-wide catalogue: batch row
// g = off[r] + i for row i of request r. The device pipeline is the one of
// xm_match run once for the batch:
//   k_batch_ingest  per batch row: request (binary search of the offsets),
//                   position in the index frame, validity, (zone, RA) key
//   radix sort      all requests together, so neighbouring warps share the
//                   index's B rows in L2 whatever request they serve
//   k_batch_prep    prepared sources with their request's region and shape
//   k_scan          persistent: a fixed grid whose warps take 32-source
//                   chunks from a device work queue until it is empty, so a
//                   mix of tiny and huge requests keeps every SM busy
//   placement, segment sorts, float64 best-pair resolution  (as xm_match)
//   k_batch_rows_a, k_batch_write_a   A-side rows of each request's join
//   k_batch_matched_b   distinct B rows of each request's selected pairs
//                   (bounded open-addressing set), giving its unmatched-B count
// Every size inside the pipeline is read from device memory and every output
// goes to an arena of known capacity, so the pipeline has no host
// synchronisation and is captured as one CUDA graph when asked; a short
// arena is detected afterwards and the batch is run again with room.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "xm_scan.cuh"

namespace xm {
namespace {

constexpr int kBlock = 256;

unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

int bits_for(int64_t v) {
    int b = 0;
    while (v > 0) { b++; v >>= 1; }
    return b;
}

struct ReqDev {
    const double* lon;
    const double* lat;
    const double* a_col;
    const double* b_col;
    const double* pa_col;
    int64_t n, off;
    int32_t rotate, shape, pa_dir, join_type;
    int32_t join_sel, pad;
    double a, b, pa, size_k, pa_zero;
};

struct BatchConst {
    const ReqDev* req;
    const int64_t* off;  // [n_req + 1]
    int32_t n_req;
    int64_t total;
    double rot_g2e[9], rot_e2g[9];  // index frame conversions
    int32_t index_frame;
    int32_t nz;
    float h_f;  // zone height of the index (rad)
};

__device__ __forceinline__ int32_t find_req(const int64_t* __restrict__ off, int32_t n_req,
                                            int64_t g) {
    int32_t lo = 0, hi = n_req;  // off[lo] <= g < off[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(&off[mid]) <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void batch_position(const BatchConst& C, const ReqDev& R, int64_t i,
                                               double* lon, double* lat, double* gamma, bool* ok) {
    const double* rot = R.rotate == 1 ? C.rot_g2e : C.rot_e2g;
    a_position_of(R.lon[i], R.lat[i], R.rotate, rot, lon, lat, gamma, ok);
}

__global__ void k_batch_ingest(BatchConst C, uint64_t* __restrict__ keys,
                               uint32_t* __restrict__ vals, int32_t* err, int32_t* bad_req) {
    pdl_wait();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= C.total) return;
    const int32_t r = find_req(C.off, C.n_req, g);
    const ReqDev& R = C.req[r];
    const int64_t i = g - R.off;
    double lon, lat, gamma;
    bool ok;
    batch_position(C, R, i, &lon, &lat, &gamma, &ok);
    const double a = col_or(R.a_col, i, R.a);
    const double b = R.shape == XM_CIRCLE ? a : col_or(R.b_col, i, R.b);
    const double pa = col_or(R.pa_col, i, R.pa);
    if (!ok) {
        atomicOr(err, kErrCoord);
        atomicMin(bad_req, r);
    }
    if (!size_ok(a, b, pa)) {
        atomicOr(err, kErrSize);
        atomicMin(bad_req, r);
    }
    if (!keys) return;  // validation only (input order)
    const PosKey k = pos_key(lon, lat, C.nz);
    keys[g] = ((uint64_t)k.z << 32) | ((uint32_t)(k.key64 >> 32) & kRaKeyMask);
    vals[g] = (uint32_t)g;
}

__global__ void k_batch_prep(BatchConst C, const uint32_t* __restrict__ vals,
                             APrep* __restrict__ out, ACold* __restrict__ cold,
                             int32_t* __restrict__ lrow) {
    pdl_wait();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.total) return;
    const int64_t g = vals ? (int64_t)vals[s] : s;
    const int32_t r = find_req(C.off, C.n_req, g);
    const ReqDev& R = C.req[r];
    const int64_t i = g - R.off;
    double lon, lat, gamma;
    bool ok;
    batch_position(C, R, i, &lon, &lat, &gamma, &ok);
    const double a = col_or(R.a_col, i, R.a);
    const double b = R.shape == XM_CIRCLE ? a : col_or(R.b_col, i, R.b);
    const double pa = col_or(R.pa_col, i, R.pa);
    make_aprep(lon, lat, gamma, ok, a, b, pa, R.shape, R.pa_dir, R.size_k, R.pa_zero, C.nz, C.h_f,
               (int32_t)g, &out[s], &cold[s]);
    lrow[g] = (int32_t)i;
}

__device__ __forceinline__ bool jt_pairs(int t) {
    return t == XM_JOIN_AND || t == XM_JOIN_OR || t == XM_JOIN_ALL1 || t == XM_JOIN_ALL2;
}
__device__ __forceinline__ bool jt_un_a(int t) {
    return t == XM_JOIN_OR || t == XM_JOIN_ALL1 || t == XM_JOIN_NOT1_2 || t == XM_JOIN_XOR;
}
__device__ __forceinline__ bool jt_un_b(int t) {
    return t == XM_JOIN_OR || t == XM_JOIN_ALL2 || t == XM_JOIN_NOT2_1 || t == XM_JOIN_XOR;
}

// A-side rows of each batch row's join, and unmatched A sources per request.
__global__ void k_batch_rows_a(BatchConst C, const int32_t* __restrict__ count,
                               int32_t* __restrict__ rows, unsigned long long* __restrict__ req_un_a) {
    pdl_wait();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= C.total) return;
    const int32_t r = find_req(C.off, C.n_req, g);
    const ReqDev& R = C.req[r];
    const int32_t c = count[g];
    int32_t n = 0;
    if (R.join_type >= 0) {
        const int32_t sel = R.join_sel == XM_SEL_ALL ? c : (c > 0 ? 1 : 0);
        n = jt_pairs(R.join_type) ? sel : 0;
        if (sel == 0 && jt_un_a(R.join_type)) n = 1;
    }
    rows[g] = n;
    // unmatched A sources per request, one atomic per request and warp
    const uint32_t peers = __match_any_sync(__activemask(), c == 0 ? r : -1);
    const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
    if (c == 0 && (peers & lt) == 0) atomicAdd(&req_un_a[r], (unsigned long long)__popc(peers));
}

__global__ void k_batch_write_a(BatchConst C, const int32_t* __restrict__ count,
                                const int64_t* __restrict__ pair_off, const int64_t* __restrict__ pb,
                                const double* __restrict__ ps, long long pair_cap,
                                const int64_t* __restrict__ best_b, const double* __restrict__ best_s,
                                const int64_t* __restrict__ row_off, long long row_cap,
                                int64_t* __restrict__ oa, int64_t* __restrict__ ob,
                                double* __restrict__ os) {
    pdl_wait();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= C.total) return;
    const int32_t r = find_req(C.off, C.n_req, g);
    const ReqDev& R = C.req[r];
    if (R.join_type < 0) return;
    const int32_t c = count[g];
    const int64_t o = row_off[g];
    const int64_t i = g - R.off;
    if (c > 0) {
        if (!jt_pairs(R.join_type)) return;
        if (R.join_sel == XM_SEL_ALL) {
            const int64_t p = pair_off[g];
            if (p + c > pair_cap || o + c > row_cap) return;
            for (int32_t k = 0; k < c; k++) {
                oa[o + k] = i;
                ob[o + k] = pb[p + k];
                os[o + k] = ps[p + k];
            }
        } else if (o < row_cap) {
            oa[o] = i;
            ob[o] = best_b[g];
            os[o] = best_s[g];
        }
    } else if (jt_un_a(R.join_type) && o < row_cap) {
        oa[o] = i;
        ob[o] = -1;
        os[o] = NAN;
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // SplitMix64 finaliser
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

// Distinct B rows among each request's selected pairs (requests whose join
// keeps unmatched B rows): inserts (request, B row) into an open-addressing
// set; each first insertion counts for its request. Probing is bounded by the
// table size (at most half full), so every insertion ends.
__global__ void k_batch_matched_b(BatchConst C, const int32_t* __restrict__ count,
                                  const int64_t* __restrict__ pair_off,
                                  const int64_t* __restrict__ pb, long long pair_cap,
                                  const int64_t* __restrict__ best_b, uint64_t* __restrict__ table,
                                  uint64_t mask, unsigned long long* __restrict__ req_mb,
                                  int32_t* err) {
    pdl_wait();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= C.total) return;
    const int32_t r = find_req(C.off, C.n_req, g);
    const ReqDev& R = C.req[r];
    if (R.join_type < 0 || !jt_un_b(R.join_type)) return;
    const int32_t c = count[g];
    if (c == 0) return;
    const bool all = R.join_sel == XM_SEL_ALL;
    const int64_t p = pair_off[g];
    if (all && p + c > pair_cap) return;
    uint32_t fresh = 0;  // this source's first insertions
    for (int32_t k = 0; k < (all ? c : 1); k++) {
        const int64_t b = all ? pb[p + k] : best_b[g];
        const uint64_t key = ((uint64_t)(uint32_t)r << 32) | (uint64_t)(uint32_t)b;
        uint64_t h = mix64(key) & mask;
        for (uint64_t probe = 0;; probe++) {
            if (probe > mask) {
                atomicOr(err, kErrOverflow);
                break;
            }
            const unsigned long long prev =
                atomicCAS((unsigned long long*)&table[h], ~0ull, (unsigned long long)key);
            if (prev == ~0ull) {
                fresh++;
                break;
            }
            if (prev == key) break;
            h = (h + 1) & mask;
        }
    }
    // counted once per request and warp (a warp's sources almost always
    // belong to one request, whose counter would otherwise take one atomic
    // per distinct B row)
    const uint32_t peers = __match_any_sync(__activemask(), fresh ? r : -1);
    const uint32_t sum = __reduce_add_sync(peers, fresh);
    const uint32_t lt = (1u << (threadIdx.x & 31)) - 1u;
    if (fresh && (peers & lt) == 0) atomicAdd(&req_mb[r], (unsigned long long)sum);
}

// Per-request bounds in the pair and row arenas.
__global__ void k_req_bounds(BatchConst C, const int64_t* __restrict__ pair_off,
                             const int64_t* __restrict__ row_off, const int64_t* totals,
                             int64_t* __restrict__ out) {
    pdl_wait();
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= C.n_req) return;
    const int64_t b = C.off[r], e = C.off[r + 1];
    out[4 * r + 0] = b < C.total ? pair_off[b] : totals[0];
    out[4 * r + 1] = e < C.total ? pair_off[e] : totals[0];
    out[4 * r + 2] = b < C.total ? row_off[b] : totals[1];
    out[4 * r + 3] = e < C.total ? row_off[e] : totals[1];
}

template <int PREC, int MODE>
xm_status launch_persistent(const char* name, const ScanArgs& a, int blocks, cudaStream_t s) {
    XM_LAUNCH(name, (unsigned)blocks, kScanThreads, kScanSmem, s, (k_scan<PREC, MODE>), a);
    return XM_OK;
}

// A non-blocking stream per device and host thread for graph capture (slots
// of a server capture concurrently).
cudaStream_t capture_stream() {
    static thread_local cudaStream_t cs[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!cs[dev] && cudaStreamCreateWithFlags(&cs[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return cs[dev];
}

xm_status launch_persistent_any(int prec, int mode, const ScanArgs& a, int blocks, cudaStream_t s) {
    if (prec == XM_PREC_FP32_RECHECK) {
        if (mode == kModeCount)
            return launch_persistent<kPrecFP32, kModeCount>("k_scan_fp32_count", a, blocks, s);
        if (mode == kModeEmit)
            return launch_persistent<kPrecFP32, kModeEmit>("k_scan_fp32_emit", a, blocks, s);
        return launch_persistent<kPrecFP32, kModeResolve>("k_scan_fp32_resolve", a, blocks, s);
    }
    if (mode == kModeCount)
        return launch_persistent<kPrecFP64, kModeCount>("k_scan_fp64_count", a, blocks, s);
    return launch_persistent<kPrecFP64, kModeEmit>("k_scan_fp64_emit", a, blocks, s);
}

// Device memory of one batch pass.
struct BatchBufs {
    // kept in the batch
    int32_t* count = nullptr;
    int64_t* pair_off = nullptr;
    int64_t* best_b = nullptr;
    double* best_sep = nullptr;
    int64_t *pa = nullptr, *pb = nullptr;
    double* ps = nullptr;
    int64_t *ra = nullptr, *rb = nullptr;
    double* rs = nullptr;
    ReqDev* req = nullptr;
    int64_t* off = nullptr;
    // temporaries of the pass
    uint64_t* keys = nullptr;
    uint32_t* vals = nullptr;
    APrep* prep = nullptr;
    ACold* cold = nullptr;
    int32_t* lrow = nullptr;
    int32_t* lists = nullptr;
    MemberRec* arena = nullptr;
    int32_t* rows = nullptr;
    int64_t* row_off = nullptr;
    uint64_t* table = nullptr;
    int64_t* small = nullptr;  // see the layout below
    int64_t* bounds = nullptr;
    double* h_in = nullptr;    // host columns staged on the device
};

// small[]: 0 total pairs, 1 total rows, 2 arena records, 3 (int32 x2) error
// bits and first bad request, 4 (int32 x4) list counts + pad, 6.. per-request
// counters follow at small + 8: unmatched A [n], matched B [n]
constexpr int kSmallWords = 8;

}  // namespace
}  // namespace xm

using namespace xm;

struct xm_batch {
    int device;
    // the stream the batch was computed on: its arrays are released in that
    // stream's order, after the work the caller queued there to read them
    cudaStream_t stream = nullptr;
    int64_t n_req, total_a, total_pairs, total_rows, n_b;
    int32_t precision;
    std::vector<int64_t> off;          // [n_req + 1]
    std::vector<int64_t> bounds;       // 4 per request
    std::vector<int64_t> un_a, un_b;   // per request
    std::vector<int32_t> join_type, join_sel, sel;
    BatchBufs B;
    double device_ms = 0.0;
};

static void free_batch_bufs(BatchBufs& B, cudaStream_t s) {
    void* p[] = {B.count, B.pair_off, B.best_b, B.pa, B.ra, B.req, B.off};
    for (void* q : p) dev_free(q, s);
    B = BatchBufs();
}

extern "C" xm_status xm_batch_free(xm_batch* X) {
    if (!X) return XM_OK;
    free_batch_bufs(X->B, X->stream);
    delete X;
    return XM_OK;
}

xm_status xm::check_request(const xm_request& q, int64_t r) {
    const xm_columns& A = q.A;
    const xm_region& g = q.region;
    if (A.n < 0 || A.n > 2147483647LL || (A.n > 0 && (!A.lon_deg || !A.lat_deg)))
        return set_error(XM_EINVAL, "request %lld: bad A columns", (long long)r);
    if (A.frame != XM_FRAME_EQ && A.frame != XM_FRAME_GAL)
        return set_error(XM_EINVAL, "request %lld: bad frame", (long long)r);
    if (g.shape < XM_CIRCLE || g.shape > XM_RECT || (g.pa_dir != 1 && g.pa_dir != -1))
        return set_error(XM_EINVAL, "request %lld: bad shape or pa_dir", (long long)r);
    if (!(isfinite(g.size_scale) && g.size_scale >= 0 && isfinite(g.size_unit_arcsec) &&
          g.size_unit_arcsec > 0 && isfinite(g.pa_zero_deg)))
        return set_error(XM_EINVAL, "request %lld: bad size scale/unit or PA zero-point", (long long)r);
    if ((!g.a_col && !(isfinite(g.a) && g.a >= 0)) ||
        (g.shape != XM_CIRCLE && !g.b_col && !(isfinite(g.b) && g.b >= 0)) ||
        (!g.pa_col && !isfinite(g.pa_deg)))
        return set_error(XM_EINVAL, "request %lld: bad fixed size or angle", (long long)r);
    if (q.selection < 1 || q.selection > 3)
        return set_error(XM_EINVAL, "request %lld: bad selection", (long long)r);
    if (q.join_type >= 0) {
        if (q.join_type > XM_JOIN_XOR)
            return set_error(XM_EINVAL, "request %lld: bad join type", (long long)r);
        if ((q.join_selection != XM_SEL_ALL && q.join_selection != XM_SEL_BEST) ||
            !(q.selection & q.join_selection))
            return set_error(XM_EINVAL, "request %lld: join selection not computed", (long long)r);
    }
    return XM_OK;
}

// One pass of the batch with given arena capacities. Sets *short_arena when
// the pair, row or set arenas were too small (the pass must be rerun).
static xm_status batch_pass(const xm_index* X, const xm_request* reqs, int64_t n,
                            const xm_batch_opts* opts, cudaStream_t s, long long pair_cap,
                            long long row_cap, xm_batch* out, bool* short_arena) {
    *short_arena = false;
    BatchBufs& B = out->B;
    const int64_t total = out->total_a;
    const int64_t nn = total > 0 ? total : 1;
    const int prec = opts ? opts->precision : XM_PREC_FP32_RECHECK;
    cudaError_t e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = (opts && opts->persistent_blocks > 0) ? opts->persistent_blocks : 4;
    // scan order of the sources: input order (request by request) unless
    // the caller asks for the sorted (zone, RA) order
    const bool sorted_a = opts && opts->a_order == XM_A_ORDER_SORTED;
    const int pblocks = std::max(1, sms * per_sm);
    const bool want_rows = std::any_of(out->join_type.begin(), out->join_type.end(),
                                       [](int32_t t) { return t >= 0; });
    const long long arena_cap = 2LL * total + (1 << 20);
    // hash set of (request, B row): at most half full
    long long sel_max = 0;
    for (int64_t r = 0; r < n; r++)
        if (out->join_type[r] >= 0 && (out->join_type[r] == XM_JOIN_OR || out->join_type[r] == XM_JOIN_ALL2 ||
                                       out->join_type[r] == XM_JOIN_NOT2_1 || out->join_type[r] == XM_JOIN_XOR))
            sel_max = 1;
    uint64_t tsize = 0;
    if (sel_max) {
        tsize = 1;
        while (tsize < 2ull * (uint64_t)std::max<long long>(pair_cap, total)) tsize <<= 1;
    }

    // ---- buffers
    B.count = (int32_t*)dev_alloc(nn * sizeof(int32_t), s);
    B.pair_off = (int64_t*)dev_alloc(nn * sizeof(int64_t), s);
    B.best_b = (int64_t*)dev_alloc(nn * (sizeof(int64_t) + sizeof(double)), s);
    B.pa = (int64_t*)dev_alloc((size_t)std::max(pair_cap, 1LL) * (2 * sizeof(int64_t) + sizeof(double)), s);
    if (want_rows)
        B.ra = (int64_t*)dev_alloc((size_t)std::max(row_cap, 1LL) * (2 * sizeof(int64_t) + sizeof(double)), s);
    if (!B.count || !B.pair_off || !B.best_b || !B.pa || (want_rows && !B.ra))
        return set_error(XM_ENOMEM, "batch of %lld A sources: result arrays", (long long)total);
    B.best_sep = (double*)(B.best_b + nn);
    B.pb = B.pa + std::max(pair_cap, 1LL);
    B.ps = (double*)(B.pb + std::max(pair_cap, 1LL));
    if (want_rows) {
        B.rb = B.ra + std::max(row_cap, 1LL);
        B.rs = (double*)(B.rb + std::max(row_cap, 1LL));
    }
    if (sorted_a) {  // sort keys and permutation (input order needs neither)
        B.keys = (uint64_t*)dev_alloc(2 * nn * sizeof(uint64_t), s);
        B.vals = (uint32_t*)dev_alloc(2 * nn * sizeof(uint32_t), s);
    }
    B.prep = (APrep*)dev_alloc(nn * sizeof(APrep), s);
    B.cold = (ACold*)dev_alloc(nn * sizeof(ACold), s);
    B.lrow = (int32_t*)dev_alloc(nn * sizeof(int32_t), s);
    B.lists = (int32_t*)dev_alloc(3 * nn * sizeof(int32_t), s);
    B.arena = (MemberRec*)dev_alloc(arena_cap * sizeof(MemberRec), s);
    B.rows = (int32_t*)dev_alloc(nn * sizeof(int32_t), s);
    B.row_off = (int64_t*)dev_alloc(nn * sizeof(int64_t), s);
    if (tsize) B.table = (uint64_t*)dev_alloc(tsize * sizeof(uint64_t), s);
    B.small = (int64_t*)dev_alloc((kSmallWords + 2 * n + 1) * sizeof(int64_t), s);
    B.bounds = (int64_t*)dev_alloc((4 * n + 1) * sizeof(int64_t), s);
    auto release_tmp = [&]() {
        void* p[] = {B.keys, B.vals, B.prep, B.cold, B.lrow, B.lists, B.arena, B.rows, B.row_off,
                     B.table, B.small, B.bounds};
        for (void* q : p) dev_free(q, s);
        B.keys = nullptr; B.vals = nullptr; B.prep = nullptr; B.cold = nullptr; B.lrow = nullptr;
        B.lists = nullptr;
        B.arena = nullptr; B.rows = nullptr; B.row_off = nullptr; B.table = nullptr;
        B.small = nullptr; B.bounds = nullptr;
    };
    if ((sorted_a && (!B.keys || !B.vals)) || !B.prep || !B.cold || !B.lrow || !B.lists ||
        !B.arena || !B.rows ||
        !B.row_off || (tsize && !B.table) || !B.small || !B.bounds) {
        release_tmp();
        return set_error(XM_ENOMEM, "batch of %lld A sources: work buffers", (long long)total);
    }

    BatchConst C;
    C.req = B.req;
    C.off = B.off;
    C.n_req = (int32_t)n;
    C.total = total;
    double m[9];
    gal_to_eq(m);
    for (int r2 = 0; r2 < 3; r2++)
        for (int c = 0; c < 3; c++) {
            C.rot_g2e[3 * r2 + c] = m[3 * r2 + c];
            C.rot_e2g[3 * r2 + c] = m[3 * c + r2];
        }
    C.index_frame = X->frame;
    C.nz = X->nz;
    C.h_f = (float)X->h;
    int32_t* err = (int32_t*)(B.small + 3);
    int32_t* bad_req = err + 1;
    int32_t* list_n = (int32_t*)(B.small + 4);
    unsigned long long* arena_n = (unsigned long long*)(B.small + 2);
    unsigned int* queue = (unsigned int*)(list_n + 3);
    unsigned long long* req_un_a = (unsigned long long*)(B.small + kSmallWords);
    unsigned long long* req_mb = req_un_a + n;

    // state that must exist before a capture (no allocation or attribute
    // change may be captured): counters, kernel attributes
    unsigned long long* stats = device_stats();
    if (!stats) {
        release_tmp();
        return set_error(XM_ENOMEM, "device counters");
    }
    prepare_kernels();
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const bool use_graph = opts && opts->use_graph;

    // The device work of the pass: no host synchronisation inside.
    auto device_work = [&](cudaStream_t s) -> xm_status {
        cudaError_t e2 = cudaMemsetAsync(B.small, 0, (kSmallWords + 2 * n + 1) * sizeof(int64_t), s);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(bad_req, 0x7f, sizeof(int32_t), s);
        if (e2 == cudaSuccess && tsize) e2 = cudaMemsetAsync(B.table, 0xff, tsize * sizeof(uint64_t), s);
        if (e2 != cudaSuccess) return cuda_fail(e2, "batch memset");
        if (total > 0) {
            if (sorted_a) {
                XM_LAUNCH("k_batch_ingest", grid_for(total), kBlock, 0, s, k_batch_ingest, C,
                          B.keys, B.vals, err, bad_req);
                xm_status r = radix_sort_u64(B.keys, B.vals, B.keys + nn, B.vals + nn, total,
                                             kSortBeginBit, 32 + bits_for(X->nz - 1), err, s);
                if (r != XM_OK) return r;
            } else {  // validation only; the scan takes the sources request by request
                XM_LAUNCH("k_batch_ingest", grid_for(total), kBlock, 0, s, k_batch_ingest, C,
                          (uint64_t*)nullptr, (uint32_t*)nullptr, err, bad_req);
            }
            XM_LAUNCH("k_batch_prep", grid_for(total), kBlock, 0, s, k_batch_prep, C,
                      sorted_a ? (const uint32_t*)B.vals : (const uint32_t*)nullptr, B.prep, B.cold,
                      B.lrow);
        }
        ScanArgs a{};
        a.G = X->geom();
        a.A = B.prep;
        a.Ac = B.cold;
        a.nA = total;
        a.want_best = 1;
        a.count = B.count;
        a.best_b = B.best_b;
        a.best_sep = B.best_sep;
        a.arena = B.arena;
        a.arena_n = arena_n;
        a.arena_cap = arena_cap;
        a.ovf_list = B.lists;
        a.tie_list = B.lists + nn;
        a.big_list = B.lists + 2 * nn;
        a.list_n = list_n;
        a.queue = queue;
        a.stats = stats;
        a.err = err;
        a.lrow = B.lrow;
        xm_status r = XM_OK;
        if (total > 0) {
            r = launch_persistent_any(prec, kModeCount, a, pblocks, s);
            if (r != XM_OK) return r;
        }
        r = exclusive_scan_i32(B.count, B.pair_off, total, B.small + 0, err, s);
        if (r != XM_OK) return r;
        if (total > 0) {
            XM_LAUNCH("k_place", 4 * sms, 256, 0, s, k_place, B.arena, arena_n, arena_cap,
                      B.pair_off, B.lrow, pair_cap, B.pa, B.pb, B.ps);
            // sources whose records did not fit the arena: scanned again
            ScanArgs b = a;
            b.list = B.lists;
            b.nlist_dev = list_n + 0;
            b.pair_off = B.pair_off;
            b.out_a = B.pa;
            b.out_b = B.pb;
            b.out_sep = B.ps;
            b.out_cap = pair_cap;
            e2 = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
            if (e2 != cudaSuccess) return cuda_fail(e2, "batch memset");
            r = launch_persistent_any(prec, kModeEmit, b, pblocks, s);
            if (r != XM_OK) return r;
            XM_LAUNCH("k_sort_small", grid_for(total), kBlock, 0, s, k_sort_small, B.count,
                      B.pair_off, total, pair_cap, B.pb, B.ps, (const int32_t*)nullptr);
            XM_LAUNCH("k_sort_warp", (unsigned)(8 * sms), 32 * kWarpSortWarps, 0, s, k_sort_warp,
                      B.count, B.pair_off, total, pair_cap, B.pb, B.ps, (const int32_t*)nullptr);
            XM_LAUNCH("k_seg_sort", (unsigned)(2 * sms), 256, 0, s, k_seg_sort, B.count,
                      B.pair_off, total, pair_cap, B.pb, B.ps, (const int32_t*)nullptr);
            if (prec == XM_PREC_FP32_RECHECK) {
                ScanArgs c = a;
                c.list = B.lists + nn;
                c.nlist_dev = list_n + 1;
                e2 = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
                if (e2 != cudaSuccess) return cuda_fail(e2, "batch memset");
                r = launch_persistent_any(prec, kModeResolve, c, pblocks, s);
                if (r != XM_OK) return r;
            }
            XM_LAUNCH("k_batch_rows_a", grid_for(total), kBlock, 0, s, k_batch_rows_a, C,
                      B.count, B.rows, req_un_a);
        }
        if (want_rows) {
            r = exclusive_scan_i32(B.rows, B.row_off, total, B.small + 1, err, s);
            if (r != XM_OK) return r;
            if (total > 0) {
                XM_LAUNCH("k_batch_write_a", grid_for(total), kBlock, 0, s, k_batch_write_a, C,
                          B.count, B.pair_off, B.pb, B.ps, pair_cap, B.best_b, B.best_sep,
                          B.row_off, row_cap, B.ra, B.rb, B.rs);
                if (tsize)
                    XM_LAUNCH("k_batch_matched_b", grid_for(total), kBlock, 0, s, k_batch_matched_b,
                              C, B.count, B.pair_off, B.pb, pair_cap, B.best_b, B.table, tsize - 1,
                              req_mb, err);
            }
        }
        if (n > 0)
            XM_LAUNCH("k_req_bounds", (unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s,
                      k_req_bounds, C, B.pair_off, want_rows ? B.row_off : B.pair_off, B.small,
                      B.bounds);
        return XM_OK;
    };

    xm_status st = XM_OK;
    if (use_graph) {
        // Captured on the library's own non-blocking stream of this device
        // (the legacy default stream cannot be captured); the graph then runs
        // on the caller's stream, after the work already queued there.
        cudaStream_t cs = capture_stream();
        if (!cs) st = set_error(XM_ECUDA, "batch: capture stream");
        if (st == XM_OK) {
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) st = cuda_fail(e, "batch: begin capture");
        }
        if (st == XM_OK) {
            st = device_work(cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (st == XM_OK && e2 != cudaSuccess) st = cuda_fail(e2, "batch: end capture");
        }
        if (st == XM_OK) {
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) st = cuda_fail(e, "batch: graph instantiate");
        }
        cudaEventRecord(ev0, s);
        if (st == XM_OK) {
            launch_begin("batch_graph", s);
            e = cudaGraphLaunch(exec, s);
            cudaError_t e2 = launch_end("batch_graph", s);
            if (e == cudaSuccess) e = e2;
            if (e != cudaSuccess) st = cuda_fail(e, "batch: graph launch");
        }
        if (st != XM_OK) cudaGetLastError();  // leave no stale error behind
    } else {
        cudaEventRecord(ev0, s);
        st = device_work(s);
    }
    cudaEventRecord(ev1, s);
    // ---- one synchronisation: totals, flags, per-request counters and bounds
    std::vector<int64_t> h_small(kSmallWords + 2 * n + 1);
    int32_t h_berr = 0;  // a deferred index build's error bits
    if (st == XM_OK) {
        e = cudaMemcpyAsync(h_small.data(), B.small, h_small.size() * sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && n > 0) {
            out->bounds.assign(4 * n, 0);
            e = cudaMemcpyAsync(out->bounds.data(), B.bounds, 4 * n * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess && X->build_err)
            e = cudaMemcpyAsync(&h_berr, X->build_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "batch sync");
        if (st == XM_OK && h_berr) st = index_build_status(h_berr);
    }
    float ms = 0.f;
    if (st == XM_OK && cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) out->device_ms = ms;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (st == XM_OK) {
        const int32_t h_err = (int32_t)(h_small[3] & 0xffffffff);
        const int32_t h_bad = (int32_t)((uint64_t)h_small[3] >> 32);
        const int32_t* h_lists = (const int32_t*)&h_small[4];
        if (h_err & kErrCoord)
            st = set_error(XM_EINVAL, "request %d: NaN/inf or |lat| > 90", h_bad);
        else if (h_err & kErrSize)
            st = set_error(XM_EINVAL, "request %d: negative or non-finite region size or angle", h_bad);
        else if (h_err & kErrTimeout)
            st = set_error(XM_ETIMEOUT, "batch sort: look-back timed out");
        if (st == XM_OK) {
            out->total_pairs = h_small[0];
            out->total_rows = want_rows ? h_small[1] : 0;
            const int64_t n_big = h_lists[2];
            if (out->total_pairs > pair_cap || out->total_rows > row_cap || (h_err & kErrOverflow))
                *short_arena = true;
            else if (n_big > 0) {
                // regions with more than 2048 members: sort them here
                xm_result view{};
                view.count = B.count;
                view.pair_off = B.pair_off;
                view.b_row = B.pb;
                view.sep = B.ps;
                st = sort_long_segments(B.lists + 2 * nn, n_big, &view, err, s);
                // the join rows copied those pairs before they were sorted
                if (st == XM_OK && want_rows && total > 0) {
                    launch_begin("k_batch_write_a", s);
                    k_batch_write_a<<<grid_for(total), kBlock, 0, s>>>(
                        C, B.count, B.pair_off, B.pb, B.ps, pair_cap, B.best_b, B.best_sep,
                        B.row_off, row_cap, B.ra, B.rb, B.rs);
                    const cudaError_t e3 = launch_end("k_batch_write_a", s);
                    if (e3 != cudaSuccess) st = cuda_fail(e3, "k_batch_write_a");
                }
            }
            out->un_a.assign(n, 0);
            out->un_b.assign(n, 0);
            for (int64_t r = 0; r < n; r++) {
                out->un_a[r] = h_small[kSmallWords + r];
                out->un_b[r] = out->n_b - h_small[kSmallWords + n + r];
            }
        }
    }
    release_tmp();
    return st;
}

extern "C" xm_status xm_match_batch(const xm_index* X, const xm_request* reqs, int64_t n,
                                    const xm_batch_opts* opts, void* stream, xm_batch** out) {
    if (!out) return set_error(XM_EINVAL, "xm_match_batch: out is NULL");
    *out = nullptr;
    if (!X || (n > 0 && !reqs) || n < 0 || n > 2147483647LL)
        return set_error(XM_EINVAL, "xm_match_batch: bad arguments");
    const int prec = opts ? opts->precision : XM_PREC_FP32_RECHECK;
    if (prec != XM_PREC_FP64 && prec != XM_PREC_FP32_RECHECK)
        return set_error(XM_EINVAL, "xm_match_batch: bad precision");
    for (int64_t r = 0; r < n; r++) {
        xm_status st = check_request(reqs[r], r);
        if (st != XM_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    xm_batch* X2 = new (std::nothrow) xm_batch();
    if (!X2) return set_error(XM_ENOMEM, "xm_match_batch: host allocation");
    cudaGetDevice(&X2->device);
    X2->stream = s;
    X2->n_req = n;
    X2->n_b = X->n;
    X2->precision = prec;
    X2->off.assign(n + 1, 0);
    X2->join_type.resize(n);
    X2->join_sel.resize(n);
    X2->sel.resize(n);
    for (int64_t r = 0; r < n; r++) {
        X2->off[r + 1] = X2->off[r] + reqs[r].A.n;
        X2->join_type[r] = reqs[r].join_type;
        X2->join_sel[r] = reqs[r].join_selection;
        X2->sel[r] = reqs[r].selection;
    }
    X2->total_a = X2->off[n];
    if (X2->total_a > 2147483647LL) {
        delete X2;
        return set_error(XM_EINVAL, "xm_match_batch: more than 2^31 - 1 A sources in one batch");
    }
    BatchBufs& B = X2->B;
    xm_status st = XM_OK;
    // request table, with host columns staged on the device
    std::vector<ReqDev> h_req(n);
    int64_t host_vals = 0;
    for (int64_t r = 0; r < n; r++)
        if (!reqs[r].A.on_device) host_vals += 5 * reqs[r].A.n;
    if (host_vals > 0) {
        B.h_in = (double*)dev_alloc(host_vals * sizeof(double), s);
        if (!B.h_in) st = set_error(XM_ENOMEM, "xm_match_batch: staging of host columns");
    }
    int64_t hpos = 0;
    for (int64_t r = 0; r < n && st == XM_OK; r++) {
        const xm_request& q = reqs[r];
        ReqDev& d = h_req[r];
        d.lon = q.A.lon_deg;
        d.lat = q.A.lat_deg;
        d.a_col = q.region.a_col;
        d.b_col = q.region.b_col;
        d.pa_col = q.region.pa_col;
        if (!q.A.on_device && q.A.n > 0) {
            const double* src[5] = {d.lon, d.lat, d.a_col, d.b_col, d.pa_col};
            const double** dst[5] = {&d.lon, &d.lat, &d.a_col, &d.b_col, &d.pa_col};
            for (int k = 0; k < 5 && st == XM_OK; k++) {
                if (!src[k]) continue;
                cudaError_t e = cudaMemcpyAsync(B.h_in + hpos, src[k], q.A.n * sizeof(double),
                                                cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) st = cuda_fail(e, "xm_match_batch: staging");
                *dst[k] = B.h_in + hpos;
                hpos += q.A.n;
            }
        }
        d.n = q.A.n;
        d.off = X2->off[r];
        d.rotate = q.A.frame == X->frame ? 0 : (q.A.frame == XM_FRAME_GAL ? 1 : 2);
        d.shape = q.region.shape;
        d.pa_dir = q.region.pa_dir;
        d.join_type = q.join_type;
        d.join_sel = q.join_selection;
        d.pad = 0;
        d.a = q.region.a;
        d.b = q.region.b;
        d.pa = q.region.pa_deg;
        d.size_k = q.region.size_scale * q.region.size_unit_arcsec * kArcsec;
        d.pa_zero = q.region.pa_zero_deg;
    }
    if (st == XM_OK) {
        B.req = (ReqDev*)dev_alloc(std::max<int64_t>(n, 1) * sizeof(ReqDev), s);
        B.off = (int64_t*)dev_alloc((n + 1) * sizeof(int64_t), s);
        if (!B.req || !B.off) st = set_error(XM_ENOMEM, "xm_match_batch: request table");
    }
    if (st == XM_OK && n > 0) {
        cudaError_t e = cudaMemcpyAsync(B.req, h_req.data(), n * sizeof(ReqDev), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B.off, X2->off.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
        // the host vectors must outlive the copies
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "xm_match_batch: request table copy");
    }
    long long pair_cap = (opts && opts->pair_capacity > 0) ? opts->pair_capacity
                                                           : 2LL * X2->total_a + (1 << 20);
    long long row_cap = (opts && opts->row_capacity > 0) ? opts->row_capacity
                                                         : pair_cap + X2->total_a;
    for (int attempt = 0; attempt < 3 && st == XM_OK; attempt++) {
        bool short_arena = false;
        st = batch_pass(X, reqs, n, opts, s, pair_cap, row_cap, X2, &short_arena);
        if (st != XM_OK || !short_arena) break;
        // room for the exact totals, then run again
        void* keep_req = B.req;
        void* keep_off = B.off;
        double* keep_h = B.h_in;
        dev_free(B.count, s);
        dev_free(B.pair_off, s);
        dev_free(B.best_b, s);
        dev_free(B.pa, s);
        dev_free(B.ra, s);
        B = BatchBufs();
        B.req = (ReqDev*)keep_req;
        B.off = (int64_t*)keep_off;
        B.h_in = keep_h;
        pair_cap = std::max(pair_cap, (long long)X2->total_pairs) * 2 + 1024;
        row_cap = std::max(row_cap, (long long)X2->total_rows) * 2 + 1024;
        if (attempt == 2) st = set_error(XM_EOVERFLOW, "xm_match_batch: arenas still short");
    }
    dev_free(B.h_in, s);
    B.h_in = nullptr;
    if (st != XM_OK) {
        xm_batch_free(X2);
        return st;
    }
    *out = X2;
    return XM_OK;
}

extern "C" xm_status xm_batch_get(const xm_batch* X, int64_t r, xm_batch_view* v) {
    if (!X || !v || r < 0 || r >= X->n_req) return set_error(XM_EINVAL, "xm_batch_get: bad arguments");
    const int64_t a0 = X->off[r];
    v->n_a = X->off[r + 1] - a0;
    const int64_t p0 = X->bounds[4 * r], p1 = X->bounds[4 * r + 1];
    const bool all = (X->sel[r] & XM_SEL_ALL) != 0;
    v->n_pairs = all ? p1 - p0 : 0;
    v->a_row = all ? X->B.pa + p0 : nullptr;
    v->b_row = all ? X->B.pb + p0 : nullptr;
    v->sep_arcsec = all ? X->B.ps + p0 : nullptr;
    v->count = X->B.count + a0;
    const bool best = (X->sel[r] & XM_SEL_BEST) != 0;
    v->best_b_row = best ? X->B.best_b + a0 : nullptr;
    v->best_sep_arcsec = best ? X->B.best_sep + a0 : nullptr;
    if (X->join_type[r] >= 0 && X->B.ra) {
        const int64_t r0 = X->bounds[4 * r + 2], r1 = X->bounds[4 * r + 3];
        v->n_rows = r1 - r0;
        v->row_a = X->B.ra + r0;
        v->row_b = X->B.rb + r0;
        v->row_sep = X->B.rs + r0;
    } else {
        v->n_rows = 0;
        v->row_a = v->row_b = nullptr;
        v->row_sep = nullptr;
    }
    v->n_unmatched_a = X->un_a.empty() ? 0 : X->un_a[r];
    const int t = X->join_type[r];
    const bool with_b = t == XM_JOIN_OR || t == XM_JOIN_ALL2 || t == XM_JOIN_NOT2_1 || t == XM_JOIN_XOR;
    v->n_unmatched_b = with_b && !X->un_b.empty() ? X->un_b[r] : -1;
    return XM_OK;
}

extern "C" xm_status xm_batch_info(const xm_batch* X, int64_t* total_a, int64_t* total_pairs,
                                   double* device_ms) {
    if (!X) return set_error(XM_EINVAL, "xm_batch_info: NULL");
    if (total_a) *total_a = X->total_a;
    if (total_pairs) *total_pairs = X->total_pairs;
    if (device_ms) *device_ms = X->device_ms;
    return XM_OK;
}

extern "C" xm_status xm_batch_join(const xm_batch* X, int64_t r, void* stream, xm_rows** out) {
    if (!out) return set_error(XM_EINVAL, "xm_batch_join: out is NULL");
    *out = nullptr;
    if (!X || r < 0 || r >= X->n_req) return set_error(XM_EINVAL, "xm_batch_join: bad arguments");
    if (X->join_type[r] < 0) return set_error(XM_EINVAL, "xm_batch_join: request %lld has no join", (long long)r);
    // a result view of the request's slice, joined as xm_join does
    const int64_t a0 = X->off[r];
    const int64_t p0 = X->bounds[4 * r];
    xm_result view{};
    view.device = X->device;
    view.selection = X->sel[r];
    view.precision = X->precision;
    view.n_a = X->off[r + 1] - a0;
    view.n_b = X->n_b;
    view.n_pairs = X->bounds[4 * r + 1] - p0;
    view.count = X->B.count + a0;
    view.a_row = X->B.pa + p0;
    view.b_row = X->B.pb + p0;
    view.sep = X->B.ps + p0;
    view.best_b = X->B.best_b + a0;
    view.best_sep = X->B.best_sep + a0;
    // pair offsets relative to the slice
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t na1 = std::max<int64_t>(view.n_a, 1);
    int64_t* rel = (int64_t*)dev_alloc((na1 + 1) * sizeof(int64_t), s);
    if (!rel) return set_error(XM_ENOMEM, "xm_batch_join: offsets");
    int32_t* err = (int32_t*)(rel + na1);
    xm_status st = XM_OK;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) st = cuda_fail(e, "xm_batch_join memset");
    if (st == XM_OK) st = exclusive_scan_i32(view.count, rel, view.n_a, nullptr, err, s);
    view.pair_off = rel;
    if (st == XM_OK) st = xm_join(&view, X->join_sel[r], X->join_type[r], stream, out);
    if (st == XM_OK) {  // the offsets' scan error bits
        int32_t h_err = 0;
        e = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "xm_batch_join");
        else if (h_err & kErrTimeout) st = set_error(XM_ETIMEOUT, "xm_batch_join: scan look-back timed out");
        if (st != XM_OK) {
            xm_rows_free(*out);
            *out = nullptr;
        }
    }
    dev_free(rel, s);
    return st;
}

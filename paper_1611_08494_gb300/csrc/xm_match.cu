// xm_match.cu -- xm_match: the Sky cross-match of paper §2.1 with the
// selections of §2.2, against a resident index of the second catalogue (§2.3).
//
// Pipeline of one call (A = the first catalogue; kernels in xm_scan.cuh):
//   k_ingest_a, radix sort, k_prep_a   A in (zone, RA) order, prepared
//   k_scan<count>   members per source, best pair, member records
//   scan of counts  pair offsets in A-row order (deterministic)
//   -- one synchronisation: pair total, list lengths, error bits --
//   k_place, k_sort_small, k_seg_sort   canonical pair list
//   k_scan<emit>    only sources whose records overflowed the arena
//   k_scan<resolve> float32 path: near-tied best pairs decided in float64
#include <math.h>

#include <new>

#include "xm_scan.cuh"

namespace xm {
namespace {

constexpr int kBlock = 256;
// Scan order when the caller leaves it to the library.
constexpr bool kDefaultSortedA = false;
// Largest member arena (records) whose pair list is placed before the pair
// count is known (the list is then sized by the arena: at most 192 MB).
constexpr long long kSpeculateRecords = 8LL << 20;

unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

int bits_for(int64_t v) {
    int b = 0;
    while (v > 0) { b++; v >>= 1; }
    return b;
}

template <int PREC, int MODE, bool FUSED = false>
xm_status launch_scan_t(const char* name, const ScanArgs& a, int64_t n_units, cudaStream_t s) {
    prepare_kernels();
    const int64_t warps = (n_units + 31) / 32;
    int64_t g = (warps + kScanWarps - 1) / kScanWarps;
    if (a.queue) {  // persistent: at most the blocks that are resident at once
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (g > 6LL * sms) g = 6LL * sms;
    }
    XM_LAUNCH(name, (unsigned)g, kScanThreads, kScanSmem, s, (k_scan<PREC, MODE, FUSED>), a);
    return XM_OK;
}

// The scan over A rows in input order that prepares each source itself
// (a.in): no separate preparation pass, no prepared records in memory.
xm_status launch_scan_fused(int prec, const ScanArgs& a, int mode, int64_t n_units, cudaStream_t s) {
    if (n_units <= 0) return XM_OK;
    if (prec == XM_PREC_FP32_RECHECK) {
        if (mode == kModeCount)
            return launch_scan_t<kPrecFP32, kModeCount, true>("k_scan_fp32_count", a, n_units, s);
        if (mode == kModeEmit)
            return launch_scan_t<kPrecFP32, kModeEmit, true>("k_scan_fp32_emit", a, n_units, s);
        return launch_scan_t<kPrecFP32, kModeResolve, true>("k_scan_fp32_resolve", a, n_units, s);
    }
    if (mode == kModeCount)
        return launch_scan_t<kPrecFP64, kModeCount, true>("k_scan_fp64_count", a, n_units, s);
    return launch_scan_t<kPrecFP64, kModeEmit, true>("k_scan_fp64_emit", a, n_units, s);
}

// The sparse count pass (k_scan_src): persistent warps, at most the blocks
// resident at once.
// Whether the count pass takes the sparse form: float32 tests in input order,
// and a region of fixed size whose bounding radius is under 0.4 zone heights,
// so a source meets at most two zones (sources with more items are left to
// k_scan by the pass itself).
bool sparse_scan(int prec, bool sorted_a, const xm_region* region, const xm_index* X) {
    if (prec != XM_PREC_FP32_RECHECK || sorted_a || region->a_col || region->b_col) return false;
    const double k = region->size_scale * region->size_unit_arcsec * kArcsec;
    const double a = fabs(region->a) * k, b = fabs(region->b) * k;
    const double R = region->shape == XM_RECT     ? hypot(a, b)
                     : region->shape == XM_CIRCLE ? a
                                                  : fmax(a, b);
    return R < 0.4 * X->h;
}

xm_status launch_scan_src(const ScanArgs& a, int32_t* defer, int32_t* n_defer, cudaStream_t s) {
    prepare_kernels();
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (a.nA + 32 * kScanWarps - 1) / (32 * kScanWarps);
    if (g > 8LL * sms) g = 8LL * sms;
    if (g < 1) g = 1;
    XM_LAUNCH("k_scan_src", (unsigned)g, kScanThreads, kSrcSmem, s, k_scan_src, a, defer, n_defer);
    return XM_OK;
}

xm_status launch_scan_any(int prec, const ScanArgs& a, int mode, int64_t n_units, cudaStream_t s) {
    if (a.A == nullptr) return launch_scan_fused(prec, a, mode, n_units, s);
    if (n_units <= 0) return XM_OK;
    if (prec == XM_PREC_FP32_RECHECK) {
        if (mode == kModeCount)
            return launch_scan_t<kPrecFP32, kModeCount>("k_scan_fp32_count", a, n_units, s);
        if (mode == kModeEmit)
            return launch_scan_t<kPrecFP32, kModeEmit>("k_scan_fp32_emit", a, n_units, s);
        return launch_scan_t<kPrecFP32, kModeResolve>("k_scan_fp32_resolve", a, n_units, s);
    }
    if (mode == kModeCount)
        return launch_scan_t<kPrecFP64, kModeCount>("k_scan_fp64_count", a, n_units, s);
    return launch_scan_t<kPrecFP64, kModeEmit>("k_scan_fp64_emit", a, n_units, s);
}

// Temporary device buffers of one call, released in reverse order on exit.
struct Temps {
    cudaStream_t s;
    void* p[32];
    int n = 0;
    explicit Temps(cudaStream_t st) : s(st) {}
    template <typename T>
    T* get(int64_t count) {
        if (n >= 32) return nullptr;
        void* q = dev_alloc((size_t)(count > 0 ? count : 1) * sizeof(T), s);
        if (q) p[n++] = q;
        return (T*)q;
    }
    ~Temps() {
        while (n > 0) dev_free(p[--n], s);
    }
};

// a_slot[row] = position of A row `row` in the sorted order.
__global__ void k_slot_of_row(const uint32_t* __restrict__ vals, int64_t n,
                              int32_t* __restrict__ a_slot) {
    pdl_wait();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) a_slot[vals[s]] = (int32_t)s;
}

// Makes `s` wait for the side stream's work when it goes out of scope (so
// temporaries freed on `s` afterwards are no longer read there).
struct Joiner {
    cudaStream_t s = nullptr;
    Side* side = nullptr;
    ~Joiner() {
        if (side) {
            cudaEventRecord(side->join, side->st);
            cudaStreamWaitEvent(s, side->join, 0);
        }
    }
};

}  // namespace
}  // namespace xm

using namespace xm;

static void free_result(xm_result* R) {
    if (!R) return;
    cudaStream_t s = R->stream;
    dev_free(R->count, s);
    dev_free(R->pair_off, s);
    dev_free(R->a_row, s);
    dev_free(R->best_b, s);
    dev_free(R->acold, s);
    dev_free(R->a_slot, s);
    delete R;
}

static xm_status check_match_args(const xm_index* X, const xm_columns* Acols,
                                  const xm_region* region, const xm_match_opts* opts) {
    if (!X || !Acols || !region || !opts) return set_error(XM_EINVAL, "xm_match: NULL argument");
    const int64_t nA = Acols->n;
    if (nA < 0 || nA > 2147483647LL || (nA > 0 && (!Acols->lon_deg || !Acols->lat_deg)))
        return set_error(XM_EINVAL, "xm_match: bad A columns");
    if (Acols->frame != XM_FRAME_EQ && Acols->frame != XM_FRAME_GAL)
        return set_error(XM_EINVAL, "xm_match: bad A frame");
    if (region->shape < XM_CIRCLE || region->shape > XM_RECT)
        return set_error(XM_EINVAL, "xm_match: bad shape %d", region->shape);
    if (region->pa_dir != 1 && region->pa_dir != -1)
        return set_error(XM_EINVAL, "xm_match: pa_dir must be +1 or -1");
    if (!(isfinite(region->size_scale) && region->size_scale >= 0 &&
          isfinite(region->size_unit_arcsec) && region->size_unit_arcsec > 0 &&
          isfinite(region->pa_zero_deg)))
        return set_error(XM_EINVAL, "xm_match: bad size scale/unit or PA zero-point");
    if (!region->a_col && !(isfinite(region->a) && region->a >= 0))
        return set_error(XM_EINVAL, "xm_match: bad fixed size a");
    if (region->shape != XM_CIRCLE && !region->b_col && !(isfinite(region->b) && region->b >= 0))
        return set_error(XM_EINVAL, "xm_match: bad fixed size b");
    if (!region->pa_col && !isfinite(region->pa_deg))
        return set_error(XM_EINVAL, "xm_match: bad fixed position angle");
    const int sel = opts->selection;
    if (sel < 1 || sel > 3) return set_error(XM_EINVAL, "xm_match: bad selection %d", sel);
    const int prec = opts->precision;
    if (prec != XM_PREC_FP64 && prec != XM_PREC_FP32_RECHECK)
        return set_error(XM_EINVAL, "xm_match: bad precision %d", prec);
    if (opts->block != 0 && opts->block != kScanThreads)
        return set_error(XM_EINVAL, "xm_match: block must be 0 or %d", kScanThreads);
    if (opts->a_order < XM_A_ORDER_DEFAULT || opts->a_order > XM_A_ORDER_INPUT)
        return set_error(XM_EINVAL, "xm_match: bad a_order %d", opts->a_order);
    return XM_OK;
}

// A match between the work it queues and its one host synchronisation:
// begin() queues the A input (copied and prepared on the side stream when it
// is host memory), the count pass, the reads of the pair total, list lengths
// and error bits, and the speculative placement; finish() waits for those
// reads and queues the rest. xm_match runs both at once; xm_match_async
// returns between them so that the caller can queue other work (an index
// build whose input copy must not go ahead of this one's, say) before the
// wait.
struct xm_pending {
    const xm_index* X;
    xm_columns A;
    xm_region region;
    int sel, prec;
    cudaStream_t s;
    xm_result* R = nullptr;
    Temps T;
    int64_t nA, nn;
    bool sorted_a = false, want_all = false;
    // the side streams' handles, copied: the per-thread records they come
    // from end with their thread, and the wait may run on another one
    Side pre_side{}, tie_side{};
    Side* pre = nullptr;  // side stream of the host A copy
    cudaStream_t ps = nullptr;
    double* a_buf = nullptr;  // A columns on the device (host input)
    long long arena_cap = 0;
    MemberRec* arena = nullptr;
    unsigned long long* arena_n = nullptr;
    int32_t *lists = nullptr, *small = nullptr, *err = nullptr, *max_count = nullptr;
    int64_t* total = nullptr;
    ScanArgs a{};
    HostReads rd;
    int32_t h_small[8] = {};
    int64_t h_total[2] = {0, 0};
    int32_t h_berr = 0;  // a deferred index build's error bits
    Side* side = nullptr;  // float64 near-tie resolve beside the placement (tie_side)
    cudaEvent_t fork = nullptr;
    int64_t np_spec = 0;

    xm_pending(const xm_index* X_, const xm_columns* A_, const xm_region* r_,
               const xm_match_opts* o, cudaStream_t s_)
        : X(X_), A(*A_), region(*r_), sel(o->selection), prec(o->precision), s(s_), T(s_),
          nA(A_->n), nn(A_->n > 0 ? A_->n : 1), rd(s_) {
        sorted_a = o->a_order == XM_A_ORDER_SORTED ||
                   (o->a_order == XM_A_ORDER_DEFAULT && kDefaultSortedA);
        want_all = (sel & XM_SEL_ALL) != 0;
    }
    xm_pending(const xm_pending&) = delete;
    xm_pending& operator=(const xm_pending&) = delete;

    xm_status begin();
    xm_status finish();
    xm_status place_and_sort(int64_t np, int64_t n_ovf);
    bool alloc_pairs(int64_t np);
    // The side stream's work joins `s`, the A copy buffer is released, and
    // (after a failure) the result: in that order, before the temporaries.
    void close(xm_status st) {
        if (pre) {  // (also when the match stopped early: nothing of it is left on ps)
            if (cudaEventRecord(pre->join, ps) == cudaSuccess) cudaStreamWaitEvent(s, pre->join, 0);
            else cudaGetLastError();
        }
        dev_free(a_buf, s);
        a_buf = nullptr;
        if (st != XM_OK && pre) cudaStreamSynchronize(ps);  // (before the result is freed)
        if (st != XM_OK) {
            free_result(R);
            R = nullptr;
        }
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
    }
};

xm_status xm_pending::begin() {
    cudaError_t e;
    R = new (std::nothrow) xm_result();
    if (!R) return set_error(XM_ENOMEM, "xm_match: host allocation");
    R->stream = s;
    cudaGetDevice(&R->device);
    R->selection = sel;
    R->precision = prec;
    R->shape = region.shape;
    R->n_a = nA;
    R->n_b = X->n;
    // per-A outputs
    R->count = (int32_t*)dev_alloc(nn * sizeof(int32_t), s);
    R->pair_off = (int64_t*)dev_alloc(nn * sizeof(int64_t), s);
    if (sel & XM_SEL_BEST) {
        R->best_b = (int64_t*)dev_alloc(nn * (sizeof(int64_t) + sizeof(double)), s);
        R->best_sep = R->best_b ? (double*)(R->best_b + nn) : nullptr;
    }
    if (!R->count || !R->pair_off || ((sel & XM_SEL_BEST) && !R->best_b))
        return set_error(XM_ENOMEM, "xm_match: result arrays");

    // host A in input order is copied and prepared on the side stream,
    // alongside what the caller's stream is still running (an index build
    // launched just before, say); its buffers are freed on `s` after it
    if (!A.on_device && nA > 0 && !sorted_a) {
        if (Side* p = side_stream()) {
            pre_side = *p;
            pre = &pre_side;
        }
    }
    ps = pre ? pre->st : s;
    // A columns on the device
    const double *lon = A.lon_deg, *lat = A.lat_deg;
    const double *ac = region.a_col, *bc = region.b_col, *pc = region.pa_col;
    if (!A.on_device && nA > 0) {
        a_buf = (double*)dev_alloc(5 * nA * sizeof(double), ps);
        if (!a_buf) return set_error(XM_ENOMEM, "A input copy");
        const double* src[5] = {lon, lat, ac, bc, pc};
        const double** dst[5] = {&lon, &lat, &ac, &bc, &pc};
        for (int k = 0; k < 5; k++) {
            if (!src[k]) continue;
            e = cudaMemcpyAsync(a_buf + k * nA, src[k], nA * sizeof(double),
                                cudaMemcpyHostToDevice, ps);
            if (e != cudaSuccess) return cuda_fail(e, "A input copy");
            *dst[k] = a_buf + k * nA;
        }
    }
    AIn I;
    I.lon = lon;
    I.lat = lat;
    I.n = nA;
    I.rotate = A.frame != X->frame;
    double m[9];
    gal_to_eq(m);
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++)
            I.rot[3 * r + c] = (A.frame == XM_FRAME_GAL) ? m[3 * r + c] : m[3 * c + r];
    I.shape = region.shape;
    I.pa_dir = region.pa_dir;
    I.a = region.a;
    I.b = region.b;
    I.pa = region.pa_deg;
    I.a_col = ac;
    I.b_col = bc;
    I.pa_col = pc;
    I.size_k = region.size_scale * region.size_unit_arcsec * kArcsec;
    I.pa_zero = region.pa_zero_deg;
    I.nz = X->nz;
    I.h_f = (float)X->h;

    // member records: room for 12 per A source on average; sources that
    // overflow it are scanned again in emit mode
    arena_cap = want_all ? 12LL * nA + 65536 : 0;
    uint64_t* keys = sorted_a ? T.get<uint64_t>(2 * nn) : nullptr;
    uint32_t* vals = sorted_a ? T.get<uint32_t>(2 * nn) : nullptr;
    // in input order the scan prepares every source itself (no prepared
    // records); sorted order prepares them in a pass of their own, in scan
    // order
    APrep* prep = nullptr;
    if (sorted_a) prep = T.get<APrep>(nn);
    // the float64 part stays with the result (float64 decisions on the pair
    // list after the match); in sorted order with the row -> slot map, in
    // input order written by the scan for the sources with members
    const bool keep_cold = sorted_a || want_all;
    R->acold = keep_cold ? (ACold*)dev_alloc(nn * sizeof(ACold), ps) : nullptr;
    ACold* cold = R->acold;
    lists = T.get<int32_t>(4 * nn);
    // [0] err, [1..3] list counts, [4] chunk queue, [5] sources the sparse
    // pass leaves, [6] largest member count, [7] their queue
    small = T.get<int32_t>(8);
    total = T.get<int64_t>(2);
    unsigned long long* stats = device_stats();
    arena = want_all ? T.get<MemberRec>(arena_cap) : nullptr;
    if ((sorted_a && (!keys || !vals || !prep)) || (keep_cold && !cold) || !lists || !small ||
        !total || !stats || (want_all && !arena))
        return set_error(XM_ENOMEM, "xm_match: work buffers");
    e = cudaMemsetAsync(small, 0, 8 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(total, 0, 2 * sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    err = small;
    arena_n = (unsigned long long*)(total + 1);
    if (nA > 0 && sorted_a) {
        XM_LAUNCH("k_ingest_a", grid_for(nA), kBlock, 0, s, k_ingest_a, I, keys, vals, err);
        xm_status r = radix_sort_u64(keys, vals, keys + nn, vals + nn, nA, kSortBeginBit,
                                     32 + bits_for(X->nz - 1), err, s);
        if (r != XM_OK) return r;
        XM_LAUNCH("k_prep_a", grid_for(nA), kBlock, 0, s, k_prep_a, I, vals, prep, cold, err);
        R->a_slot = (int32_t*)dev_alloc(nn * sizeof(int32_t), s);
        if (!R->a_slot) return set_error(XM_ENOMEM, "xm_match: slot map");
        XM_LAUNCH("k_slot_of_row", grid_for(nA), kBlock, 0, s, k_slot_of_row, vals, nA,
                  R->a_slot);
    } else if (pre) {  // the scan waits for the copy of the host columns
        e = cudaEventRecord(pre->join, ps);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pre->join, 0);
        if (e != cudaSuccess) return cuda_fail(e, "xm_match: input copy join");
    }
    a.G = X->geom();
    a.A = prep;
    a.Ac = sorted_a ? cold : nullptr;
    a.in = I;
    // the float64 part of the sources with members stays with the result
    // (only the all-pairs selection's later uses read it)
    a.acold_out = sorted_a ? nullptr : cold;
    a.nA = nA;
    a.shape = region.shape;
    a.want_best = (sel & XM_SEL_BEST) != 0;
    a.count = R->count;
    a.best_b = R->best_b;
    a.best_sep = R->best_sep;
    a.arena = arena;
    a.arena_n = arena_n;
    a.arena_cap = arena_cap;
    a.ovf_list = lists;
    a.tie_list = lists + nn;
    a.big_list = lists + 2 * nn;
    a.list_n = small + 1;
    a.stats = stats;
    a.err = err;
    // the count pass runs persistent warps that take 32-source chunks from
    // a queue, so chunks of large regions do not leave a tail; it also keeps
    // the largest member count (the segment sorts below skip the size
    // classes no row reaches)
    max_count = small + 6;
    a.max_count = max_count;
    ScanArgs cq = a;
    cq.queue = (unsigned int*)(small + 4);
    xm_status r = XM_OK;
    if (sparse_scan(prec, sorted_a, &region, X)) {
        // one lane per source where regions are small against the zones,
        // then the warp-cooperative scan over the sources it left (their
        // number read on the device)
        r = launch_scan_src(cq, lists + 3 * nn, small + 5, s);
        if (r != XM_OK) return r;
        ScanArgs cd = cq;
        cd.list = lists + 3 * nn;
        cd.nlist_dev = small + 5;
        cd.queue = (unsigned int*)(small + 7);
        r = launch_scan_any(prec, cd, kModeCount, nA, s);
    } else {
        r = launch_scan_any(prec, cq, kModeCount, nA, s);
    }
    if (r != XM_OK) return r;
    r = exclusive_scan_i32(R->count, R->pair_off, nA, total, err, s);
    if (r != XM_OK) return r;

    // the counts go to the host first; the side stream (float64 best pairs)
    // forks here, before the speculative work below
    e = rd.add(h_small, small, sizeof(h_small));
    if (e == cudaSuccess) e = rd.add(h_total, total, sizeof(h_total));
    if (e == cudaSuccess && X->build_err) e = rd.add(&h_berr, X->build_err, sizeof(int32_t));
    if (e == cudaSuccess) e = rd.mark();
    if (e != cudaSuccess) return cuda_fail(e, "xm_match count reads");
    if ((sel & XM_SEL_BEST) && prec == XM_PREC_FP32_RECHECK) {
        if (Side* p = side_stream()) {
            tie_side = *p;
            side = &tie_side;
        }
    }
    if (side && (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventRecord(fork, s) != cudaSuccess)) {
        cudaGetLastError();
        side = nullptr;
    }
    // Speculation: without overflowed sources the list holds at most the
    // arena's records, so it is placed and sorted into a list of that size
    // before the counts reach the host, and the GPU stays busy through the
    // synchronisation. (Large arenas, and overflow, take the exact size
    // after it.)
    if (want_all && nA > 0 && arena_cap <= kSpeculateRecords && alloc_pairs(arena_cap)) {
        np_spec = arena_cap;
        r = place_and_sort(np_spec, 0);
        if (r != XM_OK) return r;
    }
    return XM_OK;
}

// the pair list placed (member records -> canonical order) and its segments
// sorted, for a list of at most np slots
xm_status xm_pending::place_and_sort(int64_t np, int64_t n_ovf) {
    XM_LAUNCH("k_place", 4 * 152, 256, 0, s, k_place, arena, arena_n, arena_cap, R->pair_off,
              (const int32_t*)nullptr, (long long)np, R->a_row, R->b_row, R->sep);
    if (n_ovf > 0) {
        ScanArgs b = a;
        b.list = lists;
        b.nlist = n_ovf;
        b.pair_off = R->pair_off;
        b.out_a = R->a_row;
        b.out_b = R->b_row;
        b.out_sep = R->sep;
        b.out_cap = np;
        xm_status rr = launch_scan_any(prec, b, kModeEmit, n_ovf, s);
        if (rr != XM_OK) return rr;
    }
    const unsigned gsm = grid_for(nA) < 8u * 152u ? grid_for(nA) : 8u * 152u;
    XM_LAUNCH("k_sort_small", gsm, kBlock, 0, s, k_sort_small, R->count, R->pair_off, nA,
              (long long)np, R->b_row, R->sep, max_count);
    const int64_t gw = (nA + 32 * kWarpSortWarps - 1) / (32 * kWarpSortWarps);
    XM_LAUNCH("k_sort_warp", (unsigned)(gw < 8 * 152 ? gw : 8 * 152), 32 * kWarpSortWarps, 0, s,
              k_sort_warp, R->count, R->pair_off, nA, (long long)np, R->b_row, R->sep, max_count);
    const int64_t gs = (nA + 255) / 256;
    XM_LAUNCH("k_seg_sort", (unsigned)(gs < 2 * 152 ? gs : 2 * 152), 256, 0, s, k_seg_sort,
              R->count, R->pair_off, nA, (long long)np, R->b_row, R->sep, max_count);
    return XM_OK;
}

bool xm_pending::alloc_pairs(int64_t np) {
    R->a_row = (int64_t*)dev_alloc(np * (2 * sizeof(int64_t) + sizeof(double)), s);
    if (!R->a_row) return false;
    R->b_row = R->a_row + np;
    R->sep = (double*)(R->b_row + np);
    return true;
}

xm_status xm_pending::finish() {
    // one synchronisation: total pairs, list lengths, error bits
    cudaError_t e = rd.sync();
    if (e != cudaSuccess) return cuda_fail(e, "xm_match sync");
    if (h_berr) return index_build_status(h_berr);
    if (h_small[0] & kErrCoord) return set_error(XM_EINVAL, "A: NaN/inf or |lat| > 90");
    if (h_small[0] & kErrSize)
        return set_error(XM_EINVAL, "A: negative or non-finite region size or angle");
    if (h_small[0] & kErrTimeout) return set_error(XM_ETIMEOUT, "A sort: look-back timed out");
    const int64_t n_ovf = h_small[1], n_tie = h_small[2], n_big = h_small[3];
    R->n_pairs = want_all ? h_total[0] : 0;
    xm_status r = XM_OK;

    // near ties of the best pair, decided in float64 on the side stream
    // while the pair list is placed and sorted here
    Joiner joiner;
    if ((sel & XM_SEL_BEST) && n_tie > 0 && prec == XM_PREC_FP32_RECHECK) {
        ScanArgs b = a;
        b.list = lists + nn;
        b.nlist = n_tie;
        cudaStream_t rs = s;
        if (side && cudaStreamWaitEvent(side->st, fork, 0) == cudaSuccess) {
            joiner.s = s;
            joiner.side = side;
            rs = side->st;
        }
        r = launch_scan_any(prec, b, kModeResolve, n_tie, rs);
        if (r != XM_OK) return r;
    }
    if (want_all && !(np_spec > 0 && n_ovf == 0 && h_total[0] <= np_spec)) {
        if (np_spec > 0) {  // the speculation did not hold: the exact size
            dev_free(R->a_row, s);
            R->a_row = nullptr;
        }
        const int64_t np = h_total[0] > 0 ? h_total[0] : 1;
        if (!alloc_pairs(np))
            return set_error(XM_ENOMEM, "xm_match: %lld pairs", (long long)h_total[0]);
        if (nA > 0) {
            r = place_and_sort(np, n_ovf);
            if (r != XM_OK) return r;
        } else {
            XM_LAUNCH("k_place", 4 * 152, 256, 0, s, k_place, arena, arena_n, arena_cap,
                      R->pair_off, (const int32_t*)nullptr, (long long)np, R->a_row, R->b_row,
                      R->sep);
        }
    }
    if (want_all && n_big > 0) {
        // rare: regions holding more than kSegMax sources
        r = sort_long_segments(lists + 2 * nn, n_big, R, err, s);
        if (r != XM_OK) return r;
    }
    if (n_ovf > 0 || n_big > 0) {
        // the re-scan and the long-segment sorts can report errors
        int32_t h_err = 0;
        e = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_match sync");
        if (h_err & kErrOverflow)
            return set_error(XM_ECUDA, "xm_match: emit pass disagreed with count pass");
        if (h_err & kErrTimeout) return set_error(XM_ETIMEOUT, "xm_match: sort look-back timed out");
    }
    return XM_OK;
}

extern "C" xm_status xm_match_async(const xm_index* X, const xm_columns* Acols,
                                    const xm_region* region, const xm_match_opts* opts,
                                    void* stream, xm_pending** out) {
    if (!out) return set_error(XM_EINVAL, "xm_match: out is NULL");
    *out = nullptr;
    xm_status st = check_match_args(X, Acols, region, opts);
    if (st != XM_OK) return st;
    xm_pending* P = new (std::nothrow) xm_pending(X, Acols, region, opts, (cudaStream_t)stream);
    if (!P) return set_error(XM_ENOMEM, "xm_match: host allocation");
    st = P->begin();
    if (st != XM_OK) {
        P->close(st);
        delete P;
        return st;
    }
    *out = P;
    return XM_OK;
}

extern "C" xm_status xm_match_wait(xm_pending* P, xm_result** out) {
    if (!P) return set_error(XM_EINVAL, "xm_match_wait: NULL pending match");
    if (out) *out = nullptr;
    xm_status st = P->finish();
    if (st == XM_OK && !out) st = set_error(XM_EINVAL, "xm_match_wait: out is NULL");
    P->close(st);
    if (st == XM_OK) *out = P->R;
    delete P;
    return st;
}

extern "C" xm_status xm_match(const xm_index* X, const xm_columns* Acols, const xm_region* region,
                              const xm_match_opts* opts, void* stream, xm_result** out) {
    if (!out) return set_error(XM_EINVAL, "xm_match: out is NULL");
    *out = nullptr;
    xm_pending* P = nullptr;
    const xm_status st = xm_match_async(X, Acols, region, opts, stream, &P);
    if (st != XM_OK) return st;
    return xm_match_wait(P, out);
}

extern "C" xm_status xm_result_free(xm_result* R) {
    free_result(R);
    return XM_OK;
}

extern "C" xm_status xm_result_get(const xm_result* R, xm_result_view* v) {
    if (!R || !v) return set_error(XM_EINVAL, "xm_result_get: NULL argument");
    v->n_pairs = R->n_pairs;
    v->n_a = R->n_a;
    v->n_b = R->n_b;
    v->a_row = R->a_row;
    v->b_row = R->b_row;
    v->sep_arcsec = R->sep;
    v->count = R->count;
    v->best_b_row = R->best_b;
    v->best_sep_arcsec = R->best_sep;
    return XM_OK;
}

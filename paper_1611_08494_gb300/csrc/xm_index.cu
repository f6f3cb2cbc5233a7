// xm_index.cu -- the resident index of the second catalogue (paper §2.3).
//
// The paper files every source of the second catalogue under a sky cell so a
// source of the first catalogue need only look at nearby cells. Here the
// partition is a set of equal-height declination zones cut into RA cells,
// realised by a stable radix sort of the sources on (zone, RA key):
//   k_zone_geom   per zone: centre, its sin/cos, number and width of RA cells
//                 (once per device and zone count, then copied)
//   k_ingest_b    per source, input order: validity, fixed-point position,
//                 sort key, the float32 offsets in its cell; exact position
//                 kept by row
//   index sort    (xm_sort.cu) on a plan k_ingest_b narrows: the zone range
//                 and the RA bits that vary, so a catalogue of a small sky
//                 area sorts in fewer passes; the offsets ride along
//   k_zone_start  first sorted source of each zone (binary search)
//   k_zone_rows   rows of each zone, size of its RA bucket table (one to two
//                 buckets per source); prefix sum; k_zone_lut the offsets
//   k_gather_b    the 16-byte records in (zone, RA) order (float32 offsets
//                 in the cell's tangent frame, RA key, row) from the sorted
//                 arrays, and the bucket tables
//   k_gap_fill    the long runs of the bucket tables
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "xm_internal.cuh"

namespace xm {

namespace {

constexpr int kBlock = 256;

__global__ void k_zone_geom(int32_t nz, ZoneInfo* __restrict__ zones) {
    pdl_wait();
    const int32_t z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nz) return;
    const double h = kPi / nz;
    const double lo = -kHalfPi + z * h;
    const double hi = lo + h;
    ZoneInfo Z;
    memset(&Z, 0, sizeof(Z));
    Z.dec_c = -kHalfPi + (z + 0.5) * h;
    sincos(Z.dec_c, &Z.sin_c, &Z.cos_c);
    Z.sin_cf = (float)Z.sin_c;
    Z.cos_cf = (float)Z.cos_c;
    // widest edge of the zone: its cells are at most h wide there
    const double cos_edge = (lo <= 0.0 && hi >= 0.0) ? 1.0 : cos(fmin(fabs(lo), fabs(hi)));
    double nb = ceil(kTwoPi * cos_edge / h);
    if (nb < 1) nb = 1;
    if (nb > 1073741824.0) nb = 1073741824.0;
    Z.nbins = (uint32_t)nb;
    Z.binw = kTwoPi / nb;
    Z.binw_f = (float)Z.binw;
    zones[z] = Z;
}

// Narrows the sort plan to a block's keys: warp reductions, one lane per warp
// through shared memory, then an atomic only where the block widens what the
// plan already holds (a stale read costs one redundant atomic, never a miss).
__device__ __forceinline__ void plan_accumulate(bool has, uint32_t z, uint32_t ra,
                                                SortPlan* plan) {
    __shared__ uint32_t red[4][kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t zlo = __reduce_min_sync(0xFFFFFFFFu, has ? z : 0xFFFFFFFFu);
    const uint32_t zhi = __reduce_max_sync(0xFFFFFFFFu, has ? z : 0u);
    const uint32_t rand_ = __reduce_and_sync(0xFFFFFFFFu, has ? ra : 0xFFFFFFFFu);
    const uint32_t ror = __reduce_or_sync(0xFFFFFFFFu, has ? ra : 0u);
    if (lane == 0) {
        red[0][warp] = zlo;
        red[1][warp] = zhi;
        red[2][warp] = rand_;
        red[3][warp] = ror;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = red[0][0], b = red[1][0], c = red[2][0], d = red[3][0];
        for (int w = 1; w < kBlock / 32; w++) {
            a = min(a, red[0][w]);
            b = max(b, red[1][w]);
            c &= red[2][w];
            d |= red[3][w];
        }
        const volatile SortPlan* vp = plan;
        if (a < vp->zmin) atomicMin(&plan->zmin, a);
        if (b > vp->zmax) atomicMax(&plan->zmax, b);
        if (~c & vp->ra_and) atomicAnd(&plan->ra_and, c);
        if (d & ~vp->ra_or) atomicOr(&plan->ra_or, d);
    }
}

// The float32 offsets (xi, eta) of a source in the tangent frame of its cell
// (zone centre line, RA cell centre), from its exact fixed-point position k.
__device__ __forceinline__ void cell_offsets(const PosKey& k, float h_f, const ZoneInfo& Z,
                                             float* xi, float* eta) {
    const uint32_t ra_key = (uint32_t)(k.key64 >> 32) & kRaKeyMask;
    const uint32_t bin = bin_of(ra_key, Z.nbins);
    const LatTerms L = lat_terms(h_f * k.zfrac, Z.sin_cf, Z.cos_cf);
    float sa, hav_a;
    sin_hav(Z.binw_f * cells_from_centre(k.key64, Z.nbins, bin), &sa, &hav_a);
    *xi = L.cd * sa;
    *eta = fmaf(L.cd * Z.sin_cf, hav_a, L.sdd);
}

// Ingest of B, one source per thread in input order: validity, longitude
// mod 360, the exact position kept by row, the sort key (zone above the RA
// key to 2^-24 of a turn; the sort orders on the zone and the top 16 RA
// bits only), and the record's float32 offsets in its cell as the sort's
// payload (x in the low word, y in the high word), so the records are
// formed in index order without reading positions at random rows.
__global__ void __launch_bounds__(kBlock) k_ingest_b(
    const double* __restrict__ lon, const double* __restrict__ lat, int64_t n, int32_t nz,
    float h_f, const ZoneInfo* __restrict__ zones, uint64_t* __restrict__ keys,
    uint32_t* __restrict__ vals, uint64_t* __restrict__ pay, double2* __restrict__ pos,
    double* __restrict__ px, double* __restrict__ py, double* __restrict__ pz, SortPlan* plan,
    int32_t* err) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool has = i < n;
    uint32_t z = 0, ra = 0;
    if (has) {
        double lo = lon[i], la = lat[i];
        const bool ok = coord_ok(lo, la);
        if (!ok) atomicOr(err, kErrCoord);
        lo = keep_or_zero(lo, ok);
        la = keep_or_zero(la, ok);
        lo = lon_mod360(lo);
        const PosKey k = pos_key(lo, la, nz);
        z = (uint32_t)k.z;
        const uint32_t rk = (uint32_t)(k.key64 >> 32) & kRaKeyMask;
        ra = (rk & kIndexRaMask) >> kIndexSortBeginBit;
        keys[i] = ((uint64_t)z << 32) | rk;
        vals[i] = (uint32_t)i;
        float xi, eta;
        cell_offsets(k, h_f, zones[z], &xi, &eta);
        pay[i] = (uint64_t)__float_as_uint(xi) | ((uint64_t)__float_as_uint(eta) << 32);
        pos[i] = make_double2(lo, la);
        if (px) unit64_deg(lo, la, &px[i], &py[i], &pz[i]);
    }
    plan_accumulate(has, z, ra, plan);
}

// The sorted keys and rows of an index build: where the plan's passes left
// them.
struct Sorted {
    const uint64_t* k0;
    const uint32_t* v0;
    const uint64_t* p0;
    const uint64_t* k1;
    const uint32_t* v1;
    const uint64_t* p1;
    const SortPlan* plan;
    __device__ __forceinline__ const uint64_t* keys() const { return sorted_in_scratch(plan) ? k1 : k0; }
    __device__ __forceinline__ const uint32_t* vals() const { return sorted_in_scratch(plan) ? v1 : v0; }
    __device__ __forceinline__ const uint64_t* pays() const { return sorted_in_scratch(plan) ? p1 : p0; }
};

__global__ void k_zone_start(Sorted S, int64_t n, int32_t nz, int64_t* __restrict__ zone_start) {
    pdl_wait();
    const int32_t z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z > nz) return;
    const uint64_t* __restrict__ keys = S.keys();
    const uint64_t target = (uint64_t)z << 32;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (keys[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    zone_start[z] = lo;
}

__global__ void k_zone_rows(int32_t nz, const int64_t* __restrict__ zone_start, Sorted S,
                            ZoneInfo* __restrict__ zones, int32_t* __restrict__ lut_cnt) {
    pdl_wait();
    const int32_t z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nz) return;
    const uint64_t* __restrict__ keys = S.keys();
    ZoneInfo& Z = zones[z];
    Z.start = zone_start[z];
    Z.end = zone_start[z + 1];
    // RA buckets over the zone's own key range: a power of two, one to two
    // per source (a window's candidates are the rows of the buckets it
    // touches), at most 2^24
    const int64_t m = Z.end - Z.start;
    int lg = 0;
    while (lg < 24 && ((int64_t)1 << lg) < m) lg++;
    uint32_t kmin = 0, range = 0;
    if (m > 0) {  // (the keys are in order of their top 16 RA bits only)
        kmin = (uint32_t)keys[Z.start] & kIndexRaMask;
        range = ((uint32_t)keys[Z.end - 1] & kIndexRaMask) - kmin;
    }
    const int bits = range ? 32 - __clz(range) : 0;
    // buckets no finer than the order of the sorted keys (which keep only
    // the top bits of the RA key), then as many as range >> shift needs
    int shift = bits > lg ? bits - lg : 0;
    if (shift < kIndexSortBeginBit) shift = kIndexSortBeginBit;
    lg = bits > shift ? bits - shift : 0;  // range >> shift < 2^lg
    Z.lut_shift = (uint32_t)shift;
    Z.lut_kmin = kmin;
    Z.lut_nb = 1u << lg;
    lut_cnt[z] = (1 << lg) + 1;
}

__global__ void k_zone_lut(int32_t nz, const int64_t* __restrict__ lut_off,
                           ZoneInfo* __restrict__ zones, ZoneHot* __restrict__ zhot,
                           uint32_t* __restrict__ lut) {
    pdl_wait();
    const int32_t z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nz) return;
    const int64_t base = lut_off[z];
    zones[z].lut_base = base;
    const ZoneInfo& Z = zones[z];
    ZoneHot H;
    H.start = (uint32_t)Z.start;
    H.lut_rel = (int32_t)(base - 2 * Z.start);
    H.lut_kmin = Z.lut_kmin;
    H.shift_lg = Z.lut_shift | ((uint32_t)(__ffs(Z.lut_nb) - 1) << 8);
    H.nbins = Z.nbins;
    H.sin_cf = Z.sin_cf;
    H.cos_cf = Z.cos_cf;
    H.binw_f = Z.binw_f;
    zhot[z] = H;
    if (zones[z].end == zones[z].start) {  // empty zone: one empty bucket
        lut[base] = 0;
        lut[base + 1] = 0;
    }
}

__device__ __forceinline__ uint32_t bucket_of(uint64_t key, const ZoneInfo& Z) {
    return (((uint32_t)key & kIndexRaMask) - Z.lut_kmin) >> Z.lut_shift;
}

// A run of bucket-table entries that take one value, too long for the
// thread that found it (filled by k_gap_fill).
struct LutGap {
    int64_t first;   // index into the table array
    uint32_t count;  // entries
    uint32_t value;  // row (relative to the zone)
};

constexpr uint32_t kGapInline = 32;  // longest run written by the finding thread

// Records into index order, and each zone's RA bucket table: bucket k holds
// the first row (relative to the zone) whose key reaches it. The first row of
// each run of equal buckets writes the entries from just after the previous
// row's bucket up to its own; the zone's last row also writes the entries
// after its bucket (the value: the zone's row count). Runs longer than
// kGapInline go to a list for k_gap_fill.
__global__ void k_gather_b(Sorted S, int64_t n, const ZoneInfo* __restrict__ zones,
                           uint32_t* __restrict__ lut, BRec* __restrict__ rec,
                           LutGap* __restrict__ gaps, unsigned long long* __restrict__ n_gaps,
                           long long gap_cap, int32_t* err) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t* __restrict__ keys = S.keys();
    const uint64_t key = keys[i];
    const ZoneInfo& Z = zones[key >> 32];
    const uint64_t off = S.pays()[i];
    BRec r;
    r.xi = __uint_as_float((uint32_t)off);
    r.eta = __uint_as_float((uint32_t)(off >> 32));
    r.ra_key = (uint32_t)key;
    r.row = (int32_t)S.vals()[i];
    rec[i] = r;
    const int64_t rows = Z.end - Z.start, rel = i - Z.start;
    const int64_t b = bucket_of(key, Z);
    const int64_t pb = rel == 0 ? -1 : (int64_t)bucket_of(keys[i - 1], Z);
    auto run = [&](int64_t first, int64_t count, uint32_t value) {
        if (count <= 0) return;
        if (count <= kGapInline) {
            for (int64_t k = 0; k < count; k++) lut[Z.lut_base + first + k] = value;
        } else {
            const unsigned long long g = atomicAdd(n_gaps, 1ull);
            if ((long long)g < gap_cap) gaps[g] = LutGap{Z.lut_base + first, (uint32_t)count, value};
            else atomicOr(err, kErrOverflow);
        }
    };
    run(pb + 1, b - pb, (uint32_t)rel);
    if (rel == rows - 1) run(b + 1, (int64_t)Z.lut_nb - b, (uint32_t)rows);
}

// The long runs of the bucket tables, one block per run.
__global__ void k_gap_fill(const LutGap* __restrict__ gaps, const unsigned long long* n_gaps,
                           long long gap_cap, uint32_t* __restrict__ lut) {
    pdl_wait();
    const long long ng = min((long long)*n_gaps, gap_cap);
    for (long long g = blockIdx.x; g < ng; g += gridDim.x) {
        const LutGap G = gaps[g];
        for (uint32_t k = threadIdx.x; k < G.count; k += blockDim.x) lut[G.first + k] = G.value;
    }
}

// Zone geometry depends only on the zone count: it is computed once per
// (device, zone count) into a table kept for the life of the process and
// copied into each new index.
struct GeomCache {
    int device;
    int32_t nz;
    ZoneInfo* zones;
};

xm_status zone_geometry(int32_t nz, ZoneInfo* zones, cudaStream_t s) {
    static std::mutex mu;
    static std::vector<GeomCache> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    const ZoneInfo* src = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        for (const GeomCache& c : cache)
            if (c.device == dev && c.nz == nz) src = c.zones;
        if (!src && cache.size() < 64) {
            ZoneInfo* t = nullptr;
            if (cudaMalloc(&t, (size_t)nz * sizeof(ZoneInfo)) == cudaSuccess) {
                k_zone_geom<<<(unsigned)((nz + kBlock - 1) / kBlock), kBlock>>>(nz, t);
                if (cudaDeviceSynchronize() == cudaSuccess) {
                    cache.push_back(GeomCache{dev, nz, t});
                    src = t;
                } else {
                    cudaFree(t);
                }
            }
            cudaGetLastError();
        }
    }
    if (src) {
        e = cudaMemcpyAsync(zones, src, (size_t)nz * sizeof(ZoneInfo), cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? XM_OK : cuda_fail(e, "zone geometry copy");
    }
    XM_LAUNCH("k_zone_geom", (unsigned)((nz + kBlock - 1) / kBlock), kBlock, 0, s, k_zone_geom, nz,
              zones);
    return XM_OK;
}

int bits_for(int64_t v) {
    int b = 0;
    while (v > 0) { b++; v >>= 1; }
    return b;
}

}  // namespace

}  // namespace xm

using namespace xm;

extern "C" xm_status xm_build_index(const xm_columns* B, const xm_index_opts* opts, void* stream,
                                    xm_index** out) {
    if (!out) return set_error(XM_EINVAL, "xm_build_index: out is NULL");
    *out = nullptr;
    if (!B || B->n < 0 || B->n > 2147483647LL || (B->n > 0 && (!B->lon_deg || !B->lat_deg)))
        return set_error(XM_EINVAL, "xm_build_index: bad catalogue columns");
    if (B->frame != XM_FRAME_EQ && B->frame != XM_FRAME_GAL)
        return set_error(XM_EINVAL, "xm_build_index: bad frame %d", B->frame);
    double h_as = (opts && opts->zone_height_arcsec > 0) ? opts->zone_height_arcsec : 20.0;
    if (!(h_as >= 1.0 && h_as <= 36000.0))
        return set_error(XM_EINVAL, "xm_build_index: zone height %g arcsec outside [1, 36000]",
                         h_as);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

    const int64_t n = B->n;
    xm_index* X = new (std::nothrow) xm_index();
    if (!X) return set_error(XM_ENOMEM, "xm_build_index: host allocation");
    X->device = dev;
    X->stream = s;
    X->frame = B->frame;
    X->n = n;
    X->nz = (int32_t)ceil(648000.0 / h_as - 1e-9);  // equal zones of height <= requested
    X->h_arcsec = 648000.0 / X->nz;
    X->h = kPi / X->nz;
    const bool fp64 = opts && opts->build_fp64;
    const bool deferred = opts && opts->deferred_check;
    const int64_t nn = n > 0 ? n : 1;

    xm_status st = XM_OK;
    // temporaries
    double *d_lon = nullptr, *d_lat = nullptr;
    uint64_t *keys = nullptr, *tk = nullptr, *pay = nullptr, *tp = nullptr;
    uint32_t *vals = nullptr, *tv = nullptr;
    int32_t* err = nullptr;
    SortPlan* plan = nullptr;
    int32_t* lut_cnt = nullptr;
    int64_t* lut_off = nullptr;
    LutGap* gaps = nullptr;
    unsigned long long* n_gaps = nullptr;
    long long gap_cap = 0;
    int32_t h_err = 0;

    auto fail = [&](xm_status code) { st = code; };
    do {
        X->rec = (BRec*)dev_alloc(nn * sizeof(BRec), s);
        X->pos = (double2*)dev_alloc(nn * sizeof(double2), s);
        X->zone_start = (int64_t*)dev_alloc((X->nz + 1) * sizeof(int64_t), s);
        X->zones = (ZoneInfo*)dev_alloc(X->nz * sizeof(ZoneInfo), s);
        X->zhot = (ZoneHot*)dev_alloc(X->nz * sizeof(ZoneHot), s);
        if (!X->rec || !X->pos || !X->zone_start || !X->zones || !X->zhot) { fail(set_error(XM_ENOMEM, "index arrays")); break; }
        X->bytes = nn * (sizeof(BRec) + sizeof(double2)) + (X->nz + 1) * sizeof(int64_t) +
                   X->nz * (sizeof(ZoneInfo) + sizeof(ZoneHot));
        if (fp64) {
            X->px = (double*)dev_alloc(3 * nn * sizeof(double), s);
            if (!X->px) { fail(set_error(XM_ENOMEM, "index unit vectors")); break; }
            X->py = X->px + nn;
            X->pz = X->py + nn;
            X->bytes += 3 * nn * sizeof(double);
        }
        if (B->id) {
            X->id = (int64_t*)dev_alloc(nn * sizeof(int64_t), s);
            if (!X->id) { fail(set_error(XM_ENOMEM, "index ids")); break; }
            X->bytes += nn * sizeof(int64_t);
            if (n > 0) {
                e = cudaMemcpyAsync(X->id, B->id, n * sizeof(int64_t),
                                    B->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) { fail(cuda_fail(e, "id copy")); break; }
            }
        }
        const double* lon = B->lon_deg;
        const double* lat = B->lat_deg;
        if (!B->on_device && n > 0) {
            d_lon = (double*)dev_alloc(2 * n * sizeof(double), s);
            if (!d_lon) { fail(set_error(XM_ENOMEM, "input copy")); break; }
            d_lat = d_lon + n;
            e = cudaMemcpyAsync(d_lon, B->lon_deg, n * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_lat, B->lat_deg, n * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) { fail(cuda_fail(e, "input copy")); break; }
            lon = d_lon;
            lat = d_lat;
        }
        keys = (uint64_t*)dev_alloc(2 * nn * sizeof(uint64_t), s);
        vals = (uint32_t*)dev_alloc(2 * nn * sizeof(uint32_t), s);
        pay = (uint64_t*)dev_alloc(2 * nn * sizeof(uint64_t), s);
        err = (int32_t*)dev_alloc(sizeof(int32_t), s);
        plan = (SortPlan*)dev_alloc(sizeof(SortPlan), s);
        lut_cnt = (int32_t*)dev_alloc(X->nz * sizeof(int32_t), s);
        lut_off = (int64_t*)dev_alloc(X->nz * sizeof(int64_t), s);
        // bucket tables: a zone of m rows has at most max(2, 2m) + 1 entries
        X->lut_n = 2 * n + 3 * (int64_t)X->nz + 16;
        X->lut = (uint32_t*)dev_alloc(X->lut_n * sizeof(uint32_t), s);
        // runs of more than kGapInline entries: at most one per kGapInline + 1
        // entries, plus one per zone for its last run
        gap_cap = X->lut_n / (kGapInline + 1) + 2 * (int64_t)X->nz + 16;
        gaps = (LutGap*)dev_alloc(gap_cap * sizeof(LutGap) + 16, s);
        n_gaps = gaps ? (unsigned long long*)(gaps + gap_cap) : nullptr;
        if (!keys || !vals || !pay || !err || !plan || !lut_cnt || !lut_off || !X->lut || !gaps) {
            fail(set_error(XM_ENOMEM, "index build buffers"));
            break;
        }
        X->bytes += X->lut_n * sizeof(uint32_t);
        tk = keys + nn;
        tv = vals + nn;
        tp = pay + nn;
        e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(n_gaps, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) { fail(cuda_fail(e, "memset")); break; }

        auto body = [&]() -> xm_status {
            const IndexGeom G = X->geom();
            const unsigned gz = (unsigned)((X->nz + kBlock) / kBlock);
            xm_status rg = zone_geometry(X->nz, X->zones, s);
            if (rg != XM_OK) return rg;
            xm_status r = sort_plan_init(plan, s);
            if (r != XM_OK) return r;
            if (n > 0) {
                const unsigned g = (unsigned)((n + kBlock - 1) / kBlock);
                XM_LAUNCH("k_ingest_b", g, kBlock, 0, s, k_ingest_b, lon, lat, n, X->nz, G.h_f,
                          X->zones, keys, vals, pay, X->pos, X->px, X->py, X->pz, plan, err);
            }
            // the virtual key: zone offset above the RA bits that vary
            const int max_passes = (bits_for(X->nz - 1) + 32 - kIndexSortBeginBit + 7) / 8;
            r = index_sort(keys, vals, pay, tk, tv, tp, n, plan, max_passes, err, s);
            if (r != XM_OK) return r;
            const Sorted S{keys, vals, pay, tk, tv, tp, plan};
            XM_LAUNCH("k_zone_start", gz, kBlock, 0, s, k_zone_start, S, n, X->nz, X->zone_start);
            XM_LAUNCH("k_zone_rows", gz, kBlock, 0, s, k_zone_rows, X->nz, X->zone_start, S,
                      X->zones, lut_cnt);
            r = exclusive_scan_i32(lut_cnt, lut_off, X->nz, nullptr, err, s);
            if (r != XM_OK) return r;
            XM_LAUNCH("k_zone_lut", gz, kBlock, 0, s, k_zone_lut, X->nz, lut_off, X->zones, X->zhot,
                      X->lut);
            if (n > 0) {
                const unsigned g = (unsigned)((n + kBlock - 1) / kBlock);
                XM_LAUNCH("k_gather_b", g, kBlock, 0, s, k_gather_b, S, n, X->zones, X->lut,
                          X->rec, gaps, n_gaps, gap_cap, err);
                XM_LAUNCH("k_gap_fill", 4 * 152, kBlock, 0, s, k_gap_fill, gaps, n_gaps, gap_cap,
                          X->lut);
            }
            return XM_OK;
        };
        st = body();
        if (st != XM_OK) break;
        if (deferred) {  // the error word stays with the index, read by its first match
            X->build_err = err;
            err = nullptr;
            break;
        }
        e = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { fail(cuda_fail(e, "xm_build_index sync")); break; }
        const xm_status bs = index_build_status(h_err);
        if (bs != XM_OK) { fail(bs); break; }
    } while (0);

    dev_free(d_lon, s);
    dev_free(keys, s);
    dev_free(vals, s);
    dev_free(pay, s);
    dev_free(err, s);
    dev_free(plan, s);
    dev_free(lut_cnt, s);
    dev_free(lut_off, s);
    dev_free(gaps, s);
    if (st != XM_OK) {
        xm_index_free(X);
        return st;
    }
    *out = X;
    return XM_OK;
}

xm_status xm::index_build_status(int32_t bits) {
    if (bits & kErrCoord) return set_error(XM_EINVAL, "B: NaN/inf or |lat| > 90");
    if (bits & kErrTimeout) return set_error(XM_ETIMEOUT, "index sort: look-back timed out");
    if (bits & kErrOverflow) return set_error(XM_ECUDA, "index bucket tables: run list overflow");
    return XM_OK;
}

// The index's memory returns to the pool in the order of the stream it was
// built on, after whatever the caller queued there.
extern "C" xm_status xm_index_free(xm_index* X) {
    if (!X) return XM_OK;
    cudaStream_t s = X->stream;
    dev_free(X->rec, s);
    dev_free(X->pos, s);
    dev_free(X->px, s);
    dev_free(X->id, s);
    dev_free(X->zone_start, s);
    dev_free(X->zones, s);
    dev_free(X->zhot, s);
    dev_free(X->lut, s);
    dev_free(X->build_err, s);
    delete X;
    return XM_OK;
}

extern "C" xm_status xm_index_info(const xm_index* X, int64_t* n, int64_t* zones,
                                   double* zone_height_arcsec, int64_t* device_bytes) {
    if (!X) return set_error(XM_EINVAL, "xm_index_info: NULL index");
    if (n) *n = X->n;
    if (zones) *zones = X->nz;
    if (zone_height_arcsec) *zone_height_arcsec = X->h_arcsec;
    if (device_bytes) *device_bytes = X->bytes;
    return XM_OK;
}

// xm_index.cu -- the resident index of the second catalogue (paper §2.3).
//
// The paper assigns every source of the second catalogue to a sky cell so a
// source of the first catalogue need only look at nearby cells. Here the
// partition is a set of declination zones cut into RA cells, realised by a
// stable radix sort of the sources on (zone, RA key):
//   k_ingest_b    longitude normalisation, validity, (zone, ra_key) sort key
//   radix sort    (xm_sort.cu)
//   k_zone_table  per zone: centre, its sin/cos, number and width of RA cells
//   k_zone_start  first sorted source of each zone (binary search)
//   k_gather_b    per sorted source: float32 offsets in its cell's tangent
//                 frame, float64 (RA, Dec), optional float64 unit vector, id
#include <math.h>

#include <new>

#include "xm_internal.cuh"

namespace xm {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool coord_ok(double lon, double lat) {
    return isfinite(lon) && isfinite(lat) && lat >= -90.0 && lat <= 90.0;
}

// Longitude modulo 360 and latitude, in radians.
__device__ __forceinline__ void norm_radec(double lon, double lat, double* ra, double* dec) {
    double l = fmod(lon, 360.0);
    if (l < 0) l += 360.0;
    *ra = l * kDeg;
    *dec = lat * kDeg;
}

__global__ void k_ingest_b(const double* __restrict__ lon, const double* __restrict__ lat,
                           int64_t n, double h, int32_t nz, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals, int32_t* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo = lon[i], la = lat[i];
    if (!coord_ok(lo, la)) {
        atomicOr(err, kErrCoord);
        lo = 0.0;
        la = 0.0;
    }
    double ra, dec;
    norm_radec(lo, la, &ra, &dec);
    keys[i] = ((uint64_t)zone_of(dec, h, nz) << 32) | ra_key_of(ra);
    vals[i] = (uint32_t)i;
}

__global__ void k_zone_table(int32_t nz, double h, ZoneInfo* __restrict__ zones) {
    int32_t z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= nz) return;
    double lo = -kHalfPi + z * h;
    double hi = fmin(lo + h, kHalfPi);
    ZoneInfo Z;
    Z.dec_c = 0.5 * (lo + hi);
    sincos(Z.dec_c, &Z.sin_c, &Z.cos_c);
    Z.sin_cf = (float)Z.sin_c;
    Z.cos_cf = (float)Z.cos_c;
    // widest edge of the zone: its cells are at most h wide there
    double cos_edge = (lo <= 0.0 && hi >= 0.0) ? 1.0 : cos(fmin(fabs(lo), fabs(hi)));
    double nb = ceil(kTwoPi * cos_edge / h);
    if (nb < 1) nb = 1;
    if (nb > 1073741824.0) nb = 1073741824.0;
    Z.nbins = (uint32_t)nb;
    Z.binw = kTwoPi / nb;
    Z.pad = 0;
    zones[z] = Z;
}

__global__ void k_zone_start(const uint64_t* __restrict__ keys, int64_t n, int32_t nz,
                             int64_t* __restrict__ zone_start) {
    int32_t z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z > nz) return;
    uint64_t target = (uint64_t)z << 32;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (keys[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    zone_start[z] = lo;
}

__global__ void k_gather_b(const double* __restrict__ lon, const double* __restrict__ lat,
                           const int64_t* __restrict__ id, const uint64_t* __restrict__ keys,
                           const uint32_t* __restrict__ vals, int64_t n,
                           const ZoneInfo* __restrict__ zones, BRec* __restrict__ rec,
                           double2* __restrict__ pos, double* __restrict__ px,
                           double* __restrict__ py, double* __restrict__ pz,
                           int64_t* __restrict__ id_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t row = vals[i];
    uint64_t key = keys[i];
    int32_t z = (int32_t)(key >> 32);
    uint32_t ra_key = (uint32_t)key;
    double lo = lon[row], la = lat[row];
    if (!coord_ok(lo, la)) { lo = 0.0; la = 0.0; }  // the call fails anyway
    double ra, dec;
    norm_radec(lo, la, &ra, &dec);
    const ZoneInfo Z = zones[z];
    CellOff o = cell_offsets(ra, dec, Z, bin_of(ra_key, Z.nbins));
    BRec r;
    r.xi = o.xi;
    r.eta = o.eta;
    r.ra_key = ra_key;
    r.row = (int32_t)row;
    rec[i] = r;
    pos[i] = make_double2(ra, dec);
    if (px) unit64(ra, dec, &px[i], &py[i], &pz[i]);
    if (id_out) id_out[i] = id[row];
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
    X->frame = B->frame;
    X->n = n;
    X->h_arcsec = h_as;
    X->h = h_as * kArcsec;
    X->nz = (int32_t)ceil(648000.0 / h_as - 1e-9);
    const bool fp64 = opts && opts->build_fp64;
    const int64_t nn = n > 0 ? n : 1;

    xm_status st = XM_OK;
    // temporaries
    double *d_lon = nullptr, *d_lat = nullptr;
    int64_t* d_id = nullptr;
    uint64_t *keys = nullptr, *tk = nullptr;
    uint32_t *vals = nullptr, *tv = nullptr;
    int32_t* err = nullptr;
    int32_t h_err = 0;

    auto fail = [&](xm_status code) { st = code; };
    do {
        X->rec = (BRec*)dev_alloc(nn * sizeof(BRec), s);
        X->pos = (double2*)dev_alloc(nn * sizeof(double2), s);
        X->zone_start = (int64_t*)dev_alloc((X->nz + 1) * sizeof(int64_t), s);
        X->zones = (ZoneInfo*)dev_alloc(X->nz * sizeof(ZoneInfo), s);
        if (!X->rec || !X->pos || !X->zone_start || !X->zones) { fail(set_error(XM_ENOMEM, "index arrays")); break; }
        X->bytes = nn * (sizeof(BRec) + sizeof(double2)) + (X->nz + 1) * sizeof(int64_t) +
                   X->nz * sizeof(ZoneInfo);
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
        }
        const double* lon = B->lon_deg;
        const double* lat = B->lat_deg;
        const int64_t* idp = B->id;
        if (!B->on_device && n > 0) {
            d_lon = (double*)dev_alloc(2 * n * sizeof(double), s);
            if (!d_lon) { fail(set_error(XM_ENOMEM, "input copy")); break; }
            d_lat = d_lon + n;
            e = cudaMemcpyAsync(d_lon, B->lon_deg, n * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_lat, B->lat_deg, n * sizeof(double), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess && B->id) {
                d_id = (int64_t*)dev_alloc(n * sizeof(int64_t), s);
                if (!d_id) { fail(set_error(XM_ENOMEM, "input copy")); break; }
                e = cudaMemcpyAsync(d_id, B->id, n * sizeof(int64_t), cudaMemcpyHostToDevice, s);
            }
            if (e != cudaSuccess) { fail(cuda_fail(e, "input copy")); break; }
            lon = d_lon;
            lat = d_lat;
            idp = d_id;
        }
        keys = (uint64_t*)dev_alloc(2 * nn * sizeof(uint64_t), s);
        vals = (uint32_t*)dev_alloc(2 * nn * sizeof(uint32_t), s);
        err = (int32_t*)dev_alloc(sizeof(int32_t), s);
        if (!keys || !vals || !err) { fail(set_error(XM_ENOMEM, "sort buffers")); break; }
        tk = keys + nn;
        tv = vals + nn;
        e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) { fail(cuda_fail(e, "memset")); break; }

        auto body = [&]() -> xm_status {
            unsigned gz = (unsigned)((X->nz + kBlock) / kBlock);
            XM_LAUNCH("k_zone_table", gz, kBlock, 0, s, k_zone_table, X->nz, X->h, X->zones);
            if (n > 0) {
                unsigned g = (unsigned)((n + kBlock - 1) / kBlock);
                XM_LAUNCH("k_ingest_b", g, kBlock, 0, s, k_ingest_b, lon, lat, n, X->h, X->nz, keys,
                          vals, err);
                xm_status r = radix_sort_u64(keys, vals, tk, tv, n, 32 + bits_for(X->nz - 1), s);
                if (r != XM_OK) return r;
            }
            XM_LAUNCH("k_zone_start", gz, kBlock, 0, s, k_zone_start, keys, n, X->nz,
                      X->zone_start);
            if (n > 0) {
                unsigned g = (unsigned)((n + kBlock - 1) / kBlock);
                XM_LAUNCH("k_gather_b", g, kBlock, 0, s, k_gather_b, lon, lat, idp, keys, vals, n,
                          X->zones, X->rec, X->pos, X->px, X->py, X->pz, X->id);
            }
            return XM_OK;
        };
        st = body();
        if (st != XM_OK) break;
        e = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { fail(cuda_fail(e, "xm_build_index sync")); break; }
        if (h_err & kErrCoord) { fail(set_error(XM_EINVAL, "B: NaN/inf or |lat| > 90")); break; }
    } while (0);

    dev_free(d_lon, s);
    dev_free(d_id, s);
    dev_free(keys, s);
    dev_free(vals, s);
    dev_free(err, s);
    if (st != XM_OK) {
        xm_index_free(X);
        return st;
    }
    *out = X;
    return XM_OK;
}

extern "C" xm_status xm_index_free(xm_index* X) {
    if (!X) return XM_OK;
    cudaStream_t s = nullptr;
    dev_free(X->rec, s);
    dev_free(X->pos, s);
    dev_free(X->px, s);
    dev_free(X->id, s);
    dev_free(X->zone_start, s);
    dev_free(X->zones, s);
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

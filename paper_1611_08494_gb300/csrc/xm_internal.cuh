// xm_internal.cuh -- shared types and device geometry of the CUDA library.
//
// Geometry (paper §2.1, Sky functional case). Every position is a unit vector
// p on the sphere; a source A carries its local east/north basis (e, n). For
// a candidate B, x = p_B.e, y = p_B.n, z = p_B.p_A; rho = atan2(|(x,y)|, z) is
// the angular separation and (x, y) scaled by rho/|(x,y)| are the
// azimuthal-equidistant coordinates of B about A. A region of position angle
// theta (east of north) and sizes a, b accepts B when
//   circle:    rho <= a
//   ellipse:   (X/a)^2 + (Y/b)^2 <= 1,  X = k (x sin t + y cos t),
//   rectangle: max(|X|/a, |Y|/b) <= 1,  Y = k (x cos t - y sin t), k = rho/s.
//
// Sky partition (paper §2.3). Index-frame latitudes are cut into nz zones of
// equal height h = 180 deg / nz. A position's zone coordinate is
// t = (lat_deg + 90) * nz / 180: zone z = floor(t), and its offset from the
// zone centre line is t - z - 1/2 zones. Longitudes become 64-bit fixed-point
// keys key64 = floor(lon_deg / 360 * 2^64); the sort key of the index uses
// ra_key = key64 >> 32. Each zone is cut into `nbins` RA cells of equal width,
// nbins chosen so a cell is at most h wide on the zone's equator-side edge;
// the cell of a source is bin = (ra_key * nbins) >> 32 and its centre is at
// RA (bin + 1/2) 2pi/nbins on the zone's centre line.
//
// Precision pattern. Each B source stores float32 orthographic offsets
// (xi, eta) = (p_B.e_c, p_B.n_c) in the tangent frame of its cell centre c.
// The angles from the cell centre are formed exactly in fixed point (integer
// products of key64 and nbins, and the zone coordinate) and only then rounded
// to float32, so the offsets carry absolute errors of a few float32 ulps of
// the cell size and the float32 path needs no float64 operation per source or
// per candidate (GB300's float64 pipe runs at 1/64 of its float32 rate). An A
// source re-expresses itself in the same cell frame and tests candidates with
// ~60 float32 operations; results within a guard band of the boundary are
// re-tested in float64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <utility>

#include "xm.h"

namespace xm {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kHalfPi = 1.570796326794896619231321691639751442;
constexpr double kDeg = kPi / 180.0;
constexpr double kArcsec = kPi / 648000.0;
constexpr double kRadToArcsec = 648000.0 / kPi;
constexpr double kKey64PerDeg = 18446744073709551616.0 / 360.0;  // 2^64 / 360
constexpr double kKey64PerRad = 18446744073709551616.0 / kTwoPi;
constexpr float kKey32PerRadF = 683565275.57643158f;            // 2^32 / 2pi
constexpr float kEps32 = 5.9604645e-08f;                         // 2^-24

// error bits set by kernels (device status word)
enum : int32_t {
    kErrCoord = 1,      // NaN / inf / |lat| > 90
    kErrSize = 2,       // negative or non-finite region size or angle
    kErrTimeout = 4,    // a bounded wait ran out
    kErrOverflow = 8,   // a fixed-capacity buffer would overflow
};

// One declination zone. Its B sources are rows [start, end) of the index,
// sorted by ra_key. The RA bucket table spans the zone's own key range
// [lut_kmin, last key]: lut[lut_base + k], k = (ra_key - lut_kmin) >>
// lut_shift (k < lut_nb), holds the first row (relative to start) whose key
// reaches bucket k, and lut[lut_base + lut_nb] the zone's row count; a window
// bound is two table reads and a short search.
struct __align__(16) ZoneInfo {
    double dec_c;          // zone centre latitude (rad)
    double sin_c, cos_c;   // of dec_c, float64
    double binw;           // RA cell width (rad)
    int64_t start, end;    // index rows of the zone
    // the four fields the B ingest reads for every source, in one 32-byte
    // sector (across two sectors its pass took 2.62 ms instead of 2.00 on
    // the all-sky index)
    float sin_cf, cos_cf;  // of dec_c, float32
    float binw_f;          // RA cell width (rad), float32
    uint32_t nbins;        // RA cells
    int64_t lut_base;      // first bucket entry of the zone
    uint32_t lut_shift;    // key bits per bucket
    uint32_t lut_kmin;     // smallest ra_key of the zone
    uint32_t lut_nb;       // buckets (a power of two)
};

// The fields of a zone the candidate scan reads, packed into one 32-byte
// sector (the table of all zones stays in L2). Catalogues hold fewer than
// 2^31 rows, so the zone's first row fits 32 bits; the bucket table of a zone
// of m rows has at most 2m + 1 entries (2 when empty), so its first entry lies
// within [start + z, 2 start + 2z] and is kept relative to 2 start.
struct __align__(32) ZoneHot {
    uint32_t start;     // first index row of the zone
    int32_t lut_rel;    // first bucket entry of the zone, minus 2 * start
    uint32_t lut_kmin;  // smallest ra_key of the zone
    uint32_t shift_lg;  // key bits per bucket | log2(buckets) << 8
    uint32_t nbins;     // RA cells
    float sin_cf, cos_cf;  // of the zone centre latitude
    float binw_f;          // RA cell width (rad)
};

__device__ __forceinline__ ZoneHot load_zone_hot(const ZoneHot* p) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + 1);
    ZoneHot z;
    z.start = u.x;
    z.lut_rel = (int32_t)u.y;
    z.lut_kmin = u.z;
    z.shift_lg = u.w;
    z.nbins = v.x;
    z.sin_cf = __uint_as_float(v.y);
    z.cos_cf = __uint_as_float(v.z);
    z.binw_f = __uint_as_float(v.w);
    return z;
}

// One B source in index order (16 bytes: one vector load per candidate).
struct __align__(16) BRec {
    float xi, eta;    // offsets in the tangent frame of the source's cell
    uint32_t ra_key;  // key64 >> 32
    int32_t row;      // row in the caller's B catalogue
};

__device__ __forceinline__ BRec load_brec(const BRec* p) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    BRec b;
    b.xi = __uint_as_float(u.x);
    b.eta = __uint_as_float(u.y);
    b.ra_key = u.z;
    b.row = (int32_t)u.w;
    return b;
}

// One A source, prepared in (zone, RA) order.
struct __align__(16) APrep {
    uint64_t key64;       // fixed-point RA
    int32_t z;            // zone
    float zfrac;          // t - z - 1/2 (zones)
    float R;              // bounding radius (rad); 0 = empty region
    int32_t row;          // A row: in the caller's catalogue, or batch-wide
    float m00, m01, m10, m11;  // float32 map (x, y) -> (X/a, Y/b)
    int32_t shape;        // xm_shape of the source's region
    float g;              // guard band of the float32 test (see make_aprep)
};

// The float64 description of an A source, read only by float64 tests
// (kept apart so the scan's per-source load stays at 48 bytes).
struct ACold {
    double lon, lat;      // index-frame RA / Dec (deg)
    double theta;         // position angle in the index frame (rad)
    double a, b;          // region sizes (rad); circle: a = b = radius
};

// Geometry of a built index, passed by value to kernels.
struct IndexGeom {
    const BRec* rec;
    const double2* pos;  // (lon, lat) in degrees, index frame, by B row
    const double* px;    // float64 unit vectors by B row (nullable)
    const double* py;
    const double* pz;
    const ZoneInfo* zones;  // [nz]
    const ZoneHot* zhot;    // [nz] the scan's part of each zone
    const uint32_t* lut;    // RA bucket tables of all zones
    int32_t nz;
    double h;        // zone height (rad)
    float h_f;       // zone height (rad), float32
};

// ------------------------------------------------------ fixed-point position

// The reduction of a longitude outside [0, 360), out of line so that kernels
// whose longitudes are in range do not evaluate it: float64 instructions are
// scarce on this GPU (inline, the batch ingest of 4.2e8 sources took 9.5 ms
// instead of 6.9).
static __host__ __device__ __noinline__ double lon_reduce360(double lon) {
    double l = lon - 360.0 * floor(lon * (1.0 / 360.0));
    if (l >= 360.0) l -= 360.0;
    if (l < 0.0) l += 360.0;
    return l;
}

// Longitude (deg) reduced to [0, 360); the in-range case is decided on the
// bit pattern (0 <= lon < 360 as an integer compare; -0 counts as 0).
__host__ __device__ inline double lon_mod360(double lon) {
    uint64_t u;
    memcpy(&u, &lon, sizeof(u));
    if (u < 0x4076800000000000ull || u == 0x8000000000000000ull) return lon;  // bits of 360.0
    return lon_reduce360(lon);
}

// Selects of float64 values made on their bit patterns: a select between two
// float64 registers issues on the float64 pipe, which this GPU runs at 1/64
// of the float32 rate (two such selects per source, zeroing an invalid
// position, kept that pipe a quarter busy in the B ingest).
__device__ __forceinline__ double keep_or_zero(double x, bool keep) {
    return __longlong_as_double(keep ? __double_as_longlong(x) : 0ll);
}
// p[i] when a column is given, else the constant v.
__device__ __forceinline__ double col_or(const double* __restrict__ p, int64_t i, double v) {
    long long b = __double_as_longlong(v);
    if (p) b = __ldg(reinterpret_cast<const long long*>(p) + i);
    return __longlong_as_double(b);
}

// Finite longitude and |lat| <= 90 (NaN fails), decided on the bit patterns.
__device__ __forceinline__ bool coord_ok(double lon, double lat) {
    const uint64_t bl = (uint64_t)__double_as_longlong(lon) & 0x7FFFFFFFFFFFFFFFull;
    const uint64_t bb = (uint64_t)__double_as_longlong(lat) & 0x7FFFFFFFFFFFFFFFull;
    return bl < 0x7FF0000000000000ull && bb <= 0x4056800000000000ull;  // bits of 90.0
}

struct PosKey {
    uint64_t key64;  // floor(lon / 360 * 2^64)
    int32_t z;       // zone
    float zfrac;     // zone coordinate minus zone centre line, in zones
};

// High 64 bits of the 128-bit product (host and device).
__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// floor(m * 2^s / 45) for m < 2^53 and s <= 18, exactly, in integer
// arithmetic (long division in base 2^32); *exact tells whether the quotient
// had no remainder.
__host__ __device__ __forceinline__ uint64_t fx_div45(uint64_t m, int s, bool* exact) {
    if (s < 0) {
        if (s <= -54) {  // m * 2^s < 1
            *exact = m == 0;
            return 0;
        }
        const uint64_t t = m >> (-s);
        const uint64_t q = t / 45u;
        *exact = (t << (-s)) == m && q * 45u == t;
        return q;
    }
    const uint64_t lo = m << s;
    const uint64_t hi = s ? (m >> (64 - s)) : 0;  // N = hi * 2^64 + lo < 45 * 2^64
    const uint64_t t1 = (hi << 32) | (lo >> 32);
    const uint64_t q1 = t1 / 45u;
    const uint64_t t0 = ((t1 - q1 * 45u) << 32) | (lo & 0xFFFFFFFFull);
    const uint64_t q0 = t0 / 45u;
    *exact = q0 * 45u == t0;
    return (q1 << 32) + q0;
}

// Significand and exponent of |x| (x finite): |x| = m * 2^(e - 52).
__host__ __device__ __forceinline__ void split_double(double x, uint64_t* m, int* e) {
#ifdef __CUDA_ARCH__
    uint64_t bits = (uint64_t)__double_as_longlong(x);
#else
    uint64_t bits;
    memcpy(&bits, &x, sizeof(bits));
#endif
    bits &= 0x7FFFFFFFFFFFFFFFull;
    const int eb = (int)(bits >> 52);
    const uint64_t f = bits & 0xFFFFFFFFFFFFFull;
    *m = eb ? (f | (1ull << 52)) : f;
    *e = eb ? eb - 1023 : -1022;
}

// The single place positions (degrees, lon already in [0, 360), |lat| <= 90)
// become zone and key: every caller uses it, so zone spans and key windows
// computed from it cover the sources filed under them. All integer: the RA
// key is floor(lon / 360 * 2^64) and the latitude key floor((lat + 90) / 180
// * 2^64) (clamped below 2^64), both exact; the zone is the top part of the
// latitude key times the zone count and the zone fraction its low part.
__host__ __device__ __forceinline__ PosKey pos_key(double lon, double lat, int32_t nz) {
    PosKey k;
    uint64_t m;
    int e;
    bool exact;
    // lon * 2^64 / 360 = m * 2^(e + 9) / 45
    split_double(lon, &m, &e);
    k.key64 = fx_div45(m, e + 9, &exact);
    // |lat| * 2^64 / 180 = m * 2^(e + 10) / 45
    split_double(lat, &m, &e);
    const uint64_t u = fx_div45(m, e + 10, &exact);
    const uint64_t half = 1ull << 63;
    uint64_t lk;
    uint64_t lat_bits;
    memcpy(&lat_bits, &lat, sizeof(lat_bits));
    if ((lat_bits >> 63) == 0) lk = u >= half ? ~0ull : half + u;
    else lk = half - (u + (exact ? 0 : 1));
    k.z = (int32_t)mulhi64(lk, (uint64_t)nz);
    k.zfrac = (float)(uint32_t)((lk * (uint64_t)nz) >> 40) * 5.9604644775390625e-08f - 0.5f;  // 2^-24
    return k;
}

__device__ __forceinline__ uint32_t bin_of(uint32_t ra_key, uint32_t nbins) {
    return (uint32_t)(((uint64_t)ra_key * (uint64_t)nbins) >> 32);
}

// RA of a fixed-point key relative to the centre of cell `bin` of a zone with
// nbins cells, in cells: key64 * nbins / 2^64 - bin - 1/2, from the exact
// 128-bit product.
__device__ __forceinline__ float cells_from_centre(uint64_t key64, uint32_t nbins, uint32_t bin) {
    const uint64_t hi = __umul64hi(key64, (uint64_t)nbins);
    const uint64_t lo = key64 * (uint64_t)nbins;
    // (the 24-bit fraction converts through 32 bits: a 64-bit integer
    // conversion would take the float64 pipe)
    const float frac = (float)(uint32_t)(lo >> 40) * 5.9604644775390625e-08f;  // 2^-24
    return (float)(int32_t)((uint32_t)hi - bin) + (frac - 0.5f);
}

// sin(x) and 1 - cos(x) = 2 sin^2(x/2) in float32. Below |x| = 1/16 they are
// the Taylor series (truncation error < 3e-15 relative); above, the float32
// library functions.
__device__ __forceinline__ void sin_hav(float x, float* s, float* hav) {
    float x2 = x * x;
    if (fabsf(x) < 0.0625f) {
        *s = fmaf(x * x2, fmaf(x2, fmaf(x2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), x);
        *hav = x2 * fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 40320.0f, 1.0f / 720.0f), -1.0f / 24.0f), 0.5f);
    } else {
        *s = sinf(x);
        float h = sinf(0.5f * x);
        *hav = 2.0f * h * h;
    }
}

// Latitude terms of a position relative to a zone centre, from the latitude
// offset ddec (rad): sin/hav of ddec and cos/sin of the latitude by angle
// addition.
struct LatTerms {
    float sdd, hav_d, cd, sd;
};

__device__ __forceinline__ LatTerms lat_terms(float ddec, float sin_c, float cos_c) {
    LatTerms t;
    sin_hav(ddec, &t.sdd, &t.hav_d);
    const float cdd = 1.0f - t.hav_d;
    t.cd = cos_c * cdd - sin_c * t.sdd;
    t.sd = sin_c * cdd + cos_c * t.sdd;
    return t;
}

// zeta of a stored offset pair: p.p_c - 1 = -r2 / (1 + sqrt(1 - r2)).
__device__ __forceinline__ float zeta_of(float xi, float eta) {
    float r2 = fmaf(xi, xi, eta * eta);
    return -r2 / (1.0f + sqrtf(fmaxf(0.0f, 1.0f - r2)));
}

// Float64 basis of an A source (east/north of the index frame).
struct A64 {
    double sa, ca, sd, cd;  // sin/cos of RA and Dec
    double st, ct;          // sin/cos of theta
    double a, b;
};

__device__ __forceinline__ A64 make_a64(const ACold& A) {
    A64 r;
    sincos(A.lon * kDeg, &r.sa, &r.ca);
    sincos(A.lat * kDeg, &r.sd, &r.cd);
    sincos(A.theta, &r.st, &r.ct);
    r.a = A.a;
    r.b = A.b;
    return r;
}

// rho / sin(rho) as a series in s^2 = sin^2 rho (the arcsine series), used
// for separations below ~0.6 deg where its truncation error is < 1e-20.
__device__ __forceinline__ double rho_over_s(double s2) {
    return 1.0 + s2 * (1.0 / 6.0 + s2 * (3.0 / 40.0 + s2 * (5.0 / 112.0 + s2 * (35.0 / 1152.0))));
}

// Float64 membership of B (unit vector px, py, pz) in A's region; returns the
// separation (rad) through rho. This is the definition, written with the
// bearing folded into the east/north components.
__device__ __forceinline__ bool test64(const A64& A, int shape, double px, double py, double pz,
                                       double* rho_out) {
    double w = px * A.ca + py * A.sa;
    double x = py * A.ca - px * A.sa;
    double y = pz * A.cd - A.sd * w;
    double z = A.cd * w + pz * A.sd;
    double s2 = x * x + y * y;
    double s = sqrt(s2);
    double rho, k;
    if (z > 0.0 && s2 < 1e-4) {
        k = rho_over_s(s2);
        rho = s * k;
    } else {
        rho = atan2(s, z);
        k = s > 0.0 ? rho / s : 1.0;
    }
    *rho_out = rho;
    if (shape == XM_CIRCLE) return rho <= A.a;
    double X = x * A.st + y * A.ct;
    double Y = x * A.ct - y * A.st;
    if (shape == XM_ELLIPSE) {
        double u = X / A.a, v = Y / A.b;
        return k * k * (u * u + v * v) <= 1.0;
    }
    return k * fmax(fabs(X) / A.a, fabs(Y) / A.b) <= 1.0;
}

// Float64 normalised distance of B in A's region: the factor by which the
// region must be scaled about A to reach B (rho / r for a circle,
// sqrt((X/a)^2 + (Y/b)^2) for an ellipse, max(|X|/a, |Y|/b) for a
// rectangle, X and Y the region-frame coordinates as in test64), at most 1
// for members. Infinite for an empty region.
__device__ __forceinline__ double norm64(const A64& A, int shape, double px, double py,
                                         double pz) {
    double w = px * A.ca + py * A.sa;
    double x = py * A.ca - px * A.sa;
    double y = pz * A.cd - A.sd * w;
    double z = A.cd * w + pz * A.sd;
    double s2 = x * x + y * y;
    double s = sqrt(s2);
    double rho, k;
    if (z > 0.0 && s2 < 1e-4) {
        k = rho_over_s(s2);
        rho = s * k;
    } else {
        rho = atan2(s, z);
        k = s > 0.0 ? rho / s : 1.0;
    }
    if (A.a == 0.0 || A.b == 0.0) return INFINITY;
    if (shape == XM_CIRCLE) return rho / A.a;
    double X = x * A.st + y * A.ct;
    double Y = x * A.ct - y * A.st;
    if (shape == XM_ELLIPSE) {
        double u = X / A.a, v = Y / A.b;
        return k * sqrt(u * u + v * v);
    }
    return k * fmax(fabs(X) / A.a, fabs(Y) / A.b);
}

// Float64 unit vector of a position given in degrees.
__device__ __forceinline__ void unit64_deg(double lon, double lat, double* px, double* py,
                                           double* pz) {
    double sa, ca, sd, cd;
    sincos(lon * kDeg, &sa, &ca);
    sincos(lat * kDeg, &sd, &cd);
    *px = cd * ca;
    *py = cd * sa;
    *pz = sd;
}

// ---------------------------------------------------------------- host side

void* dev_alloc(size_t bytes, cudaStream_t s);

// A second stream per host thread and device, with a fork and a join event,
// for work of a call that can overlap the rest of it (the near-tie resolve
// beside the pair placement; host A copied and prepared beside an index
// build). Null when it cannot be created.
struct Side {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
Side* side_stream();

// Small device -> host reads gathered behind one synchronisation: add()
// queues a read; one small kernel on the stream writes them all into a
// pinned, mapped staging area this object holds while it lives (not a
// device-to-host copy: those wait in order behind every such copy queued on
// any stream); sync() waits for the stream once and hands the values out.
// Without mapped memory, or past the area's room, a read is a plain
// asynchronous copy.
class HostReads {
  public:
    explicit HostReads(cudaStream_t s) : s_(s) {}
    ~HostReads();
    HostReads(const HostReads&) = delete;
    HostReads& operator=(const HostReads&) = delete;
    cudaError_t add(void* host_dst, const void* dev_src, size_t bytes);
    // Marks the reads queued so far: sync() then waits for them only, so
    // work queued on the stream after mark() keeps the GPU busy meanwhile.
    cudaError_t mark();
    cudaError_t sync();

    struct Area {
        unsigned char* p = nullptr;   // host address
        unsigned char* dp = nullptr;  // device address of the same bytes
        cudaEvent_t ev = nullptr;     // recorded after the kernel writing it
        int dev = 0;
    };

  private:
    // queues the kernel that writes the reads into the staging area (once)
    cudaError_t launch();
    struct Item {
        void* dst;
        const void* src;
        size_t off, bytes;
    };
    cudaStream_t s_;
    Area area_;
    bool tried_ = false, have_ = false;
    size_t used_ = 0;
    int n_ = 0;
    bool marked_ = false;
    bool launched_ = false;
    bool synced_ = false;
    Item items_[8];
};
void dev_free(void* p, cudaStream_t s);
// Bytes of freed blocks kept for reuse on the current device.
size_t kept_device_bytes();

// Kernel launch bookkeeping: counts launches and, while profiling is on,
// brackets each launch with events on its stream.
void launch_begin(const char* name, cudaStream_t s);
cudaError_t launch_end(const char* name, cudaStream_t s);

// Every kernel of the library starts with pdl_wait(), and launches go out
// with programmatic dependent launch: a kernel may be scheduled while the one
// before it in the stream drains, and waits there (before any global memory
// access) until that grid has completed and its writes are visible. Without a
// programmatic predecessor the wait returns at once. This removes most of the
// gap between the many short dependent kernels of a call.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define XM_LAUNCH(name, grid, block, smem, stream, kernel, ...)             \
    do {                                                                    \
        ::xm::launch_begin(name, stream);                                   \
        const cudaError_t _l = ::xm::launch_pdl(kernel, dim3(grid), dim3(block), (smem), \
                                                (stream), __VA_ARGS__);     \
        cudaError_t _e = ::xm::launch_end(name, stream);                    \
        if (_l != cudaSuccess) _e = _l;                                     \
        if (_e != cudaSuccess) return ::xm::cuda_fail(_e, name);            \
    } while (0)

xm_status cuda_fail(cudaError_t e, const char* what);
xm_status set_error(xm_status s, const char* fmt, ...);

// The error status of a deferred index build from its error bits (host
// copy), XM_OK when clean.
xm_status index_build_status(int32_t bits);

// Device primitives (xm_sort.cu).
// Stable LSD radix sort of (keys, vals) on key bits [begin_bit, end_bit).
// Sorted data ends in (keys, vals); (tk, tv) are scratch of the same sizes.
// A look-back that timed out sets kErrTimeout in *err (device), which the
// caller reads at its next synchronisation.
xm_status radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n,
                         int begin_bit, int end_bit, int32_t* err, cudaStream_t s);

// Sets the sort kernels' shared-memory limits (done on first use; call it
// before capturing a stream that sorts).
void radix_sort_prepare();

// The index sort's plan, decided on the device from the keys themselves:
// the keys (zone << 32 | RA key) are sorted on the virtual key
// ((zone - zmin) << rb) | (RA key >> 8 & (2^rb - 1)), where the RA bits
// above rb are the same in every key, so its order is the key order and it
// needs only `active` 8-bit passes (trailing passes are skipped).
struct SortPlan {
    uint32_t zmin, zmax;      // zone range (atomicMin / atomicMax)
    uint32_t ra_and, ra_or;   // AND / OR of the 24-bit RA fields
    uint32_t rb, active;      // RA bits kept, passes needed
};

// Sets a plan to the empty ranges the key kernel narrows.
xm_status sort_plan_init(SortPlan* plan, cudaStream_t s);

// Sorts (keys, vals, pay) of an index build by the plan's virtual key with up
// to `max_passes` launches (each does nothing past plan->active); pay (a
// 64-bit payload per key, with scratch tp) may be NULL. The sorted data ends
// in (keys, vals, pay) when plan->active is even, else in (tk, tv, tp);
// sorted_in_scratch() tells which on the device.
xm_status index_sort(uint64_t* keys, uint32_t* vals, uint64_t* pay, uint64_t* tk, uint32_t* tv,
                     uint64_t* tp, int64_t n, SortPlan* plan, int max_passes, int32_t* err,
                     cudaStream_t s);

__device__ __forceinline__ bool sorted_in_scratch(const SortPlan* plan) { return plan->active & 1; }

// Sort keys file sources by zone, then by RA to 2^-24 of a turn (0.08
// arcsec): the low 8 bits of the RA key are dropped, so the sort starts at
// bit 8. Search windows are widened by one such quantum.
constexpr uint32_t kRaKeyMask = 0xFFFFFF00u;
constexpr int kSortBeginBit = 8;
// The index is ordered by zone and the top 16 bits of the RA key (2^-16 of a
// turn, 20 arcsec): its RA bucket tables never use finer buckets, and the
// scan compares every record's own (24-bit) key with the search window, so
// the order within one such bucket does not matter. A 16-bit RA field saves
// a counting pass over an all-sky index.
constexpr uint32_t kIndexRaMask = 0xFFFF0000u;
constexpr int kIndexSortBeginBit = 16;
// out[i] = sum of in[0..i) (int64); *total (device) = sum of all. One
// launch (single-pass, decoupled look-back); a look-back that timed out sets
// kErrTimeout in *err (device), which the caller reads at its next
// synchronisation.
xm_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                             int32_t* err, cudaStream_t s);
xm_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                             int32_t* err, cudaStream_t s);
// The same without allocating: ws holds 2 * ceil(n / 4096) int64 values and
// n is at most 4096 * 4096.
xm_status exclusive_scan_i32_ws(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                                int64_t* ws, cudaStream_t s);

// Host-side galactic -> equatorial rotation (row major, v_eq = m v_gal).
void gal_to_eq(double m[9]);

// Validation of one batch request (xm_batch.cu); names the request on error.
xm_status check_request(const xm_request& q, int64_t r);

void stats_add(const unsigned long long* host_counters);  // [0..4] as in xm_stats
// Per-device cumulative counters ([0..4] as in xm_stats) kernels add to.
unsigned long long* device_stats();

}  // namespace xm

// ------------------------------------------------------------ ABI objects

struct xm_index {
    int device;
    int32_t frame;
    int64_t n;
    double h_arcsec;  // zone height actually used (180 deg / nz)
    double h;         // rad
    int32_t nz;
    xm::BRec* rec;
    double2* pos;
    double *px, *py, *pz;
    int64_t* id;
    int64_t* zone_start;
    xm::ZoneInfo* zones;
    xm::ZoneHot* zhot;
    uint32_t* lut;
    int64_t lut_n;
    int64_t bytes;
    int32_t* build_err;  // error bits of a build whose check was deferred (else NULL)
    cudaStream_t stream;  // the stream it was built on (its memory is freed in its order)
    xm::IndexGeom geom() const {
        return xm::IndexGeom{rec, pos, px, py, pz, zones, zhot, lut, nz, h, (float)h};
    }
};

struct xm_result {
    int device;
    int32_t selection, precision, shape;
    int64_t n_a, n_b, n_pairs;
    int32_t* count;       // [n_a]
    int64_t* pair_off;    // [n_a] exclusive scan of count
    int64_t *a_row, *b_row;
    double* sep;
    int64_t* best_b;
    double* best_sep;
    // float64 description of the A sources (kept for float64 decisions after
    // the match; NULL in views of batch results): acold[slot], slot = a_slot[a]
    // (or a itself when a_slot is NULL)
    xm::ACold* acold;
    int32_t* a_slot;
    // the stream the result was computed on: its arrays are freed in that
    // stream's order, after the work the caller queued there to read them
    cudaStream_t stream;
};

struct xm_rows {
    int64_t n, n_unmatched_a, n_unmatched_b;
    int64_t *a_row, *b_row;
    double* sep;
    // a join whose counts are still on the device: [0] A-side rows,
    // [1] unmatched B, [2] unmatched A, [4] error bits; read (one
    // synchronisation of `stream`) by the first xm_rows_get
    int64_t* pending;
    cudaStream_t stream;
    int32_t with_un_b;
};

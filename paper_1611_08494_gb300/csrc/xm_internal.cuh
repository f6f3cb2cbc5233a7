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
// Sky partition (paper §2.3). Index frame latitudes are cut into zones of
// height h; zone z spans [-90 deg + z h, -90 deg + (z+1) h). Each zone is cut
// into `nbins` RA cells of equal width, nbins chosen so a cell is at most h
// wide on the zone's equator-side edge. B sources are sorted by
// (zone, ra_key) with ra_key = floor(RA / 2pi * 2^32). The cell of a source is
// bin = (ra_key * nbins) >> 32; its centre is ((bin + 1/2) 2pi/nbins, zone
// centre).
//
// Precision pattern. Each B source stores float32 orthographic offsets
// (xi, eta) = (p_B.e_c, p_B.n_c) in the tangent frame of its cell centre c.
// They are computed from float64 differences (RA - RA_c, Dec - Dec_c) followed
// by float32 trigonometry of those small angles, so they carry absolute
// errors of a few float32 ulps of the cell size. An A source re-expresses
// itself in the same cell frame once per (A, cell) and tests candidates with
// ~20 float32 operations; results within a guard band of the boundary are
// re-tested in float64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xm.h"

namespace xm {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kHalfPi = 1.570796326794896619231321691639751442;
constexpr double kDeg = kPi / 180.0;
constexpr double kArcsec = kPi / 648000.0;
constexpr double kRadToArcsec = 648000.0 / kPi;
constexpr double kKeyScale = 4294967296.0 / kTwoPi;  // ra_key per radian
constexpr float kEps32 = 5.9604645e-08f;              // 2^-24

// error bits set by kernels (device status word)
enum : int32_t {
    kErrCoord = 1,      // NaN / inf / |lat| > 90
    kErrSize = 2,       // negative or non-finite region size or angle
    kErrTimeout = 4,    // a bounded wait ran out
    kErrOverflow = 8,   // a fixed-capacity buffer would overflow
};

// Slots of the member list kept inline per A source during the count pass.
constexpr int kInlineSlots = 8;

struct ZoneInfo {
    double dec_c;          // zone centre latitude (rad)
    double sin_c, cos_c;   // of dec_c, float64
    double binw;           // RA cell width (rad)
    float sin_cf, cos_cf;  // of dec_c, float32
    uint32_t nbins;
    uint32_t pad;
};

// One B source in index order (16 bytes: one vector load per candidate).
struct __align__(16) BRec {
    float xi, eta;    // offsets in the tangent frame of the source's cell
    uint32_t ra_key;  // floor(RA / 2pi * 2^32)
    int32_t row;      // row in the caller's B catalogue
};

// One A source, prepared in (zone, RA) order.
struct APrep {
    double alpha, delta;  // index-frame RA / Dec (rad)
    double theta;         // position angle in the index frame (rad)
    double a, b;          // region sizes (rad); circle: a = b = radius
    float R;              // bounding radius (rad); 0 = empty region
    int32_t row;          // row in the caller's A catalogue
    float m00, m01, m10, m11;  // float32 map (x, y) -> (X/a, Y/b)
};

// A member kept inline during the count pass: B row and the separation
// (arcsec) that will be reported for the pair.
struct Slot {
    int32_t b_row;
    int32_t pad;
    double sep;
};

// Geometry of a built index, passed by value to kernels.
struct IndexGeom {
    const BRec* rec;
    const double2* pos;  // (RA, Dec) rad, float64, index order
    const double* px;    // float64 unit vectors, index order (nullable)
    const double* py;
    const double* pz;
    const int64_t* zone_start;  // [nz + 1]
    const ZoneInfo* zones;      // [nz]
    int32_t nz;
    double h;  // zone height (rad)
};

__host__ __device__ inline int32_t zone_of(double dec, double h, int32_t nz) {
    double t = floor((dec + kHalfPi) / h);
    int32_t z = t < 0 ? 0 : (t >= nz ? nz - 1 : (int32_t)t);
    return z;
}

__host__ __device__ inline uint32_t ra_key_of(double ra) {
    double k = floor(ra * kKeyScale);
    if (k < 0) k = 0;
    if (k > 4294967295.0) k = 4294967295.0;
    return (uint32_t)k;
}

__device__ __forceinline__ uint32_t bin_of(uint32_t ra_key, uint32_t nbins) {
    return (uint32_t)(((uint64_t)ra_key * (uint64_t)nbins) >> 32);
}

// Offsets of a position in the tangent frame of a cell:
//   xi   = cos(dec) sin(dRA)
//   eta  = sin(dDec) + cos(dec) sin(dec_c) (1 - cos dRA)
//   zeta = p.p_c - 1 = -[(1 - cos dDec) + cos(dec) cos(dec_c) (1 - cos dRA)]
// with dRA = RA - RA_c, dDec = Dec - Dec_c taken in float64 and everything
// after in float32; cos(dec) by angle addition from the zone centre.
struct CellOff {
    float xi, eta, zeta;
    float sd, cd;   // sin / cos of dec (float32)
    float sa, hav_a, sdd, hav_d;
};

__device__ __forceinline__ CellOff cell_offsets(double ra, double dec, const ZoneInfo& Z,
                                                uint32_t bin) {
    double ra_c = ((double)bin + 0.5) * Z.binw;
    double dra = ra - ra_c;
    if (dra > kPi) dra -= kTwoPi;
    else if (dra <= -kPi) dra += kTwoPi;
    double ddec = dec - Z.dec_c;
    float fa = (float)dra, fd = (float)ddec;
    CellOff o;
    float ca;
    sincosf(fa, &o.sa, &ca);
    float sh = sinf(0.5f * fa);
    o.hav_a = 2.0f * sh * sh;  // 1 - cos dRA without cancellation
    float cdd;
    sincosf(fd, &o.sdd, &cdd);
    float shd = sinf(0.5f * fd);
    o.hav_d = 2.0f * shd * shd;
    o.cd = Z.cos_cf * cdd - Z.sin_cf * o.sdd;
    o.sd = Z.sin_cf * cdd + Z.cos_cf * o.sdd;
    o.xi = o.cd * o.sa;
    o.eta = o.sdd + o.cd * Z.sin_cf * o.hav_a;
    o.zeta = -(o.hav_d + o.cd * Z.cos_cf * o.hav_a);
    return o;
}

// Per (A, cell) float32 transform taking B's cell offsets to (x, y) in A's
// east/north frame: (x, y) = J (dxi, deta) + dzeta t, d* = B - A offsets.
struct CellXf {
    float xa, ya, za;
    float j00, j01, j10, j11, t0, t1;
};

__device__ __forceinline__ CellXf cell_xf(double ra, double dec, const ZoneInfo& Z,
                                          uint32_t bin) {
    CellOff o = cell_offsets(ra, dec, Z, bin);
    CellXf x;
    x.xa = o.xi;
    x.ya = o.eta;
    x.za = o.zeta;
    // basis products (c = cell centre, A = the source)
    x.j00 = 1.0f - o.hav_a;            // e_c . e_A = cos dRA
    x.j01 = Z.sin_cf * o.sa;           // n_c . e_A
    x.t0 = -Z.cos_cf * o.sa;           // p_c . e_A
    x.j10 = -o.sd * o.sa;              // e_c . n_A
    x.j11 = (1.0f - o.hav_d) - o.sd * Z.sin_cf * o.hav_a;  // n_c . n_A
    x.t1 = -o.sdd + o.sd * Z.cos_cf * o.hav_a;              // p_c . n_A
    return x;
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

__device__ __forceinline__ A64 make_a64(const APrep& A) {
    A64 r;
    sincos(A.alpha, &r.sa, &r.ca);
    sincos(A.delta, &r.sd, &r.cd);
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

__device__ __forceinline__ void unit64(double ra, double dec, double* px, double* py,
                                       double* pz) {
    double sa, ca, sd, cd;
    sincos(ra, &sa, &ca);
    sincos(dec, &sd, &cd);
    *px = cd * ca;
    *py = cd * sa;
    *pz = sd;
}

// ---------------------------------------------------------------- host side

struct Ctx;  // per-call allocator / stream / launch bookkeeping (xm_api.cu)

void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Kernel launch bookkeeping: counts launches and, while profiling is on,
// brackets each launch with events on its stream.
void launch_begin(const char* name, cudaStream_t s);
cudaError_t launch_end(const char* name, cudaStream_t s);

#define XM_LAUNCH(name, grid, block, smem, stream, kernel, ...)             \
    do {                                                                    \
        ::xm::launch_begin(name, stream);                                   \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);         \
        cudaError_t _e = ::xm::launch_end(name, stream);                    \
        if (_e != cudaSuccess) return ::xm::cuda_fail(_e, name);            \
    } while (0)

xm_status cuda_fail(cudaError_t e, const char* what);
xm_status set_error(xm_status s, const char* fmt, ...);

// Device primitives (xm_sort.cu).
// Stable LSD radix sort of (keys, vals) on key bits [0, end_bit). Sorted data
// ends in (keys, vals); (tk, tv) are scratch of the same sizes.
xm_status radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n,
                         int end_bit, cudaStream_t s);
// out[i] = sum of in[0..i) (int64); *total (device) = sum of all. Works in
// place (out == in is not allowed).
xm_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                             cudaStream_t s);
xm_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                             cudaStream_t s);

// Host-side galactic -> equatorial rotation (row major, v_eq = m v_gal).
void gal_to_eq(double m[9]);

}  // namespace xm

// ------------------------------------------------------------ ABI objects

struct xm_index {
    int device;
    int32_t frame;
    int64_t n;
    double h_arcsec;
    double h;  // rad
    int32_t nz;
    xm::BRec* rec;
    double2* pos;
    double *px, *py, *pz;
    int64_t* id;
    int64_t* zone_start;
    xm::ZoneInfo* zones;
    int64_t bytes;
    xm::IndexGeom geom() const {
        return xm::IndexGeom{rec, pos, px, py, pz, zone_start, zones, nz, h};
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
};

struct xm_rows {
    int64_t n, n_unmatched_a, n_unmatched_b;
    int64_t *a_row, *b_row;
    double* sep;
};

namespace xm {
void stats_add(const unsigned long long* host_counters);  // [0..4] as in xm_stats
}

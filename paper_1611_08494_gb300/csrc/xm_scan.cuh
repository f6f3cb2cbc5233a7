// xm_scan.cuh -- device side of the Sky cross-match (paper §2.1) with the
// selections of §2.2, shared by the single-request and batched entry points.
//
//   k_ingest_a   validity, rotation into the index frame when the frames
//                differ, (zone, RA key) sort key per A source
//   k_prep_a     per A in (zone, RA) order: index-frame position (float64 and
//                fixed point), position angle (plus the frame rotation's
//                angle), sizes, bounding radius, float32 region map
//   k_scan       the candidate scan (below), in three modes: count (members,
//                best pair, member records), emit (re-scan straight into the
//                pair list), resolve (best pair decided in float64)
//   k_place, k_sort_small, k_seg_sort   member records into the canonical
//                pair list (ascending A row, then B row)
#pragma once

#include <math.h>

#include <mutex>
#include <new>

#include "xm_internal.cuh"

namespace xm {
namespace {

constexpr int kSegMax = 2048;  // largest member list sorted in shared memory
constexpr int kSmallSort = 16;  // largest member list sorted by one thread

enum { kPrecFP64 = 0, kPrecFP32 = 1 };
enum { kModeCount = 0, kModeEmit = 1, kModeResolve = 2 };

struct AIn {
    const double* lon;
    const double* lat;
    int64_t n;
    int32_t rotate;  // 1: rotate by rot (input frame -> index frame)
    double rot[9];
    int32_t shape, pa_dir;
    double a, b, pa;
    const double* a_col;
    const double* b_col;
    const double* pa_col;
    double size_k;   // radians per size unit (scale * unit * arcsec)
    double pa_zero;  // degrees
    float h_f;       // zone height of the index (rad)
    int32_t nz;
};

__device__ __noinline__ void rotate_position(double lon, double lat, const double* rot,
                                             double* lon_o, double* lat_o, double* gamma);

// Index-frame position of an A source given as (lon, lat) in its input
// frame, in degrees (lon in [0, 360)), and the angle gamma from the index
// frame's north to the input frame's north (east positive) at that point.
// rot (row major) maps input-frame vectors to the index frame when rotate.
__device__ __forceinline__ void a_position_of(double lon, double lat, int32_t rotate,
                                              const double* rot, double* lon_o, double* lat_o,
                                              double* gamma, bool* ok) {
    *ok = coord_ok(lon, lat);
    lon = keep_or_zero(lon, *ok);  // (an invalid position becomes (0, 0))
    lat = keep_or_zero(lat, *ok);
    lon = lon_mod360(lon);
    if (!rotate) {
        *lon_o = lon;
        *lat_o = lat;
        *gamma = 0.0;
        return;
    }
    rotate_position(lon, lat, rot, lon_o, lat_o, gamma);
}

// The rotation of a position into the index frame and the angle between the
// two frames' north directions there (out of line: its float64 trigonometry
// would otherwise hold registers in every kernel that prepares sources).
__device__ __noinline__ void rotate_position(double lon, double lat, const double* rot,
                                             double* lon_o, double* lat_o, double* gamma) {
    double sl, cl, sb, cb;
    sincos(lon * kDeg, &sl, &cl);
    sincos(lat * kDeg, &sb, &cb);
    const double p[3] = {cb * cl, cb * sl, sb};
    const double nn[3] = {-sb * cl, -sb * sl, cb};
    double q[3], m[3];
    for (int k = 0; k < 3; k++) {
        q[k] = rot[3 * k] * p[0] + rot[3 * k + 1] * p[1] + rot[3 * k + 2] * p[2];
        m[k] = rot[3 * k] * nn[0] + rot[3 * k + 1] * nn[1] + rot[3 * k + 2] * nn[2];
    }
    const double rxy = hypot(q[0], q[1]);
    double r = atan2(q[1], q[0]) / kDeg;
    if (r < 0) r += 360.0;
    if (r >= 360.0) r -= 360.0;
    *lon_o = r;
    *lat_o = atan2(q[2], rxy) / kDeg;
    const double ca = rxy > 0 ? q[0] / rxy : 1.0, sa = rxy > 0 ? q[1] / rxy : 0.0;
    const double sd = q[2], cd = rxy;
    // index-frame east / north at the rotated point
    const double me = -m[0] * sa + m[1] * ca;
    const double mn = -m[0] * sd * ca - m[1] * sd * sa + m[2] * cd;
    *gamma = atan2(me, mn);
}

__device__ __forceinline__ void a_position(const AIn& I, int64_t i, double* lon_o, double* lat_o,
                                           double* gamma, bool* ok) {
    a_position_of(I.lon[i], I.lat[i], I.rotate, I.rot, lon_o, lat_o, gamma, ok);
}

// Finite and not negative (-0 counts as 0), and finite, decided on the bit
// patterns (no float64 instruction).
__device__ __forceinline__ bool nonneg_finite(double x) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    return (u & 0x7FFFFFFFFFFFFFFFull) < 0x7FF0000000000000ull &&
           ((u >> 63) == 0 || (u << 1) == 0);
}

__device__ __forceinline__ bool finite_bits(double x) {
    return ((uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull) < 0x7FF0000000000000ull;
}

__device__ __forceinline__ bool size_ok(double a, double b, double pa) {
    return nonneg_finite(a) && nonneg_finite(b) && finite_bits(pa);
}

__global__ void k_ingest_a(AIn I, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           int32_t* err) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I.n) return;
    double lon, lat, gamma;
    bool ok;
    a_position(I, i, &lon, &lat, &gamma, &ok);
    if (!ok) atomicOr(err, kErrCoord);
    const double a = col_or(I.a_col, i, I.a);
    const double b = I.shape == XM_CIRCLE ? a : col_or(I.b_col, i, I.b);
    const double pa = col_or(I.pa_col, i, I.pa);
    if (!size_ok(a, b, pa)) atomicOr(err, kErrSize);
    const PosKey k = pos_key(lon, lat, I.nz);
    keys[i] = ((uint64_t)k.z << 32) | ((uint32_t)(k.key64 >> 32) & kRaKeyMask);
    vals[i] = (uint32_t)i;
}

// gamma as float32 (zero, and no conversion, when the frames agree).
__device__ __forceinline__ float gamma_f(double gamma) {
    return ((uint64_t)__double_as_longlong(gamma) << 1) == 0 ? 0.0f : (float)gamma;
}

// The prepared form of one A source (position already in the index frame),
// for an index of zone height h_f (rad): the float32 part P and the float64
// part C.
__device__ __forceinline__ void make_aprep(double lon, double lat, double gamma, bool ok, double a,
                                           double b, double pa, int32_t shape, int32_t pa_dir,
                                           double size_k, double pa_zero, int32_t nz, float h_f,
                                           int32_t row, APrep* P_out, ACold* C_out) {
    if (!size_ok(a, b, pa)) a = b = pa = 0.0;
    APrep P;
    ACold C;
    C.lon = lon;
    C.lat = lat;
    const PosKey k = pos_key(lon, lat, nz);
    P.key64 = k.key64;
    P.z = k.z;
    P.zfrac = k.zfrac;
    P.row = row;
    P.shape = shape;
    // (float64 operations are scarce on this GPU: a circle needs one size
    // and no angle)
    const bool circle = shape == XM_CIRCLE;
    C.a = a * size_k;
    C.b = circle ? C.a : b * size_k;
    // position angle east of north of the input frame, in degrees; gamma
    // turns it to the index frame's north. The float64 angle (for rechecks)
    // is one fused step; the float32 one is reduced to [0, 360) first so the
    // float32 rotation sees a small argument (in float64 only when large).
    double raw = circle ? 0.0 : pa_zero + (pa_dir > 0 ? pa : -pa);
    C.theta = circle ? 0.0 : fma(raw, kDeg, gamma);
    float af = (float)C.a, bf = (float)C.b;
    if (!ok || !(af > 0.0f || C.a > 0.0) || !(bf > 0.0f || C.b > 0.0)) {
        P.R = 0.0f;
        P.g = 0.0f;
        P.m00 = P.m01 = P.m10 = P.m11 = 0.0f;
    } else {
        // sizes below the float32 range stay regions (the float64 recheck
        // decides every candidate of so small a region)
        af = fmaxf(af, 1.17549435e-38f);
        bf = fmaxf(bf, 1.17549435e-38f);
        // bounding radius with a margin far above the float32 rounding here
        const float R = shape == XM_RECT ? sqrtf(fmaf(af, af, bf * bf)) : fmaxf(af, bf);
        P.R = R * (1.0f + 1e-6f);
        // the guard band: g bounds |q32 - q| with a 3x margin (rounding of
        // the offsets and of the map over a box of L_box), plus
        // (rho / s)^2 - 1 <= R^2 / 3 (planar against azimuthal distance)
        const float L_box = 1.42f * P.R + 2.0f * h_f;
        P.g = 128.0f * kEps32 * L_box / fminf(af, bf) + 0.34f * P.R * P.R + 16.0f * kEps32;
        float st = 0.0f, ct = 1.0f;
        if (!circle) {
            if (!(fabs(raw) < 720.0)) raw -= 360.0 * floor(raw * (1.0 / 360.0));
            float tf = (float)raw;
            tf -= 360.0f * floorf(tf * (1.0f / 360.0f));
            sincosf(fmaf(tf, 0.017453292519943295f, gamma_f(gamma)), &st, &ct);
        }
        const float ia = 1.0f / af, ib = 1.0f / bf;
        P.m00 = st * ia;
        P.m01 = ct * ia;
        P.m10 = ct * ib;
        P.m11 = -st * ib;
    }
    *P_out = P;
    *C_out = C;
}

// The prepared form of A row i from the caller's columns, its position
// (lon0, lat0) already read. Invalid positions and sizes set the error bits
// when err is given.
__device__ __forceinline__ void prep_at(const AIn& I, int64_t i, double lon0, double lat0,
                                        int32_t* err, APrep* P, ACold* C) {
    double lon, lat, gamma;
    bool ok;
    a_position_of(lon0, lat0, I.rotate, I.rot, &lon, &lat, &gamma, &ok);
    const double a = col_or(I.a_col, i, I.a);
    const double b = I.shape == XM_CIRCLE ? a : col_or(I.b_col, i, I.b);
    const double pa = col_or(I.pa_col, i, I.pa);
    if (err) {
        if (!ok) atomicOr(err, kErrCoord);
        if (!size_ok(a, b, pa)) atomicOr(err, kErrSize);
    }
    make_aprep(lon, lat, gamma, ok, a, b, pa, I.shape, I.pa_dir, I.size_k, I.pa_zero, I.nz, I.h_f,
               (int32_t)i, P, C);
}

__device__ __forceinline__ void prep_one(const AIn& I, int64_t i, int32_t* err, APrep* P,
                                         ACold* C) {
    prep_at(I, i, I.lon[i], I.lat[i], err, P, C);
}

// Prepared sources in scan order: vals[s] is the A row of position s (the
// sorted order), or NULL for input order. Invalid positions and sizes set
// the error bits (the sorted path found them already; setting them twice is
// harmless).
__global__ void k_prep_a(AIn I, const uint32_t* __restrict__ vals, APrep* __restrict__ out,
                         ACold* __restrict__ cold, int32_t* err) {
    pdl_wait();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= I.n) return;
    const int64_t i = vals ? (int64_t)vals[s] : s;
    APrep P;
    ACold C;
    prep_one(I, i, err, &P, &C);
    out[s] = P;
    cold[s] = C;
}

// One member found by the count pass: A row, its index among that row's
// members (scan order), B row, and the separation to report: float64 arcsec,
// or (flag 1) the float32 separation in radians, converted when placed.
struct MemberRec {
    int32_t a_row, k, b_row, f32;
    double sep;
};

struct ScanArgs {
    IndexGeom G;
    const APrep* A;
    const ACold* Ac;  // float64 part of A, same order
    // fused preparation (input order): the caller's columns, prepared by the
    // scan itself, and where the float64 part of sources with members goes
    AIn in;
    ACold* acold_out;
    int64_t nA;
    int32_t shape;
    int32_t want_best;
    const int32_t* list;  // sorted A indices to process (overflow / ties)
    int64_t nlist;
    const int32_t* nlist_dev;  // list length read on the device (overrides nlist)
    unsigned int* queue;       // work queue: warps claim 32-source chunks (persistent)
    // count mode: per A row
    int32_t* count;
    int64_t* best_b;
    double* best_sep;
    MemberRec* arena;             // member records (all-pairs selection), or NULL
    unsigned long long* arena_n;  // records claimed
    long long arena_cap;
    int32_t* ovf_list;  // sources with members that did not fit the arena
    int32_t* tie_list;  // sources whose best pair is decided in float64
    int32_t* big_list;  // rows with more than kSegMax members
    int32_t* list_n;    // [0] overflow, [1] ties, [2] big
    int32_t* max_count;  // (nullable) largest member count of any source
    // emit mode
    const int64_t* pair_off;
    int64_t* out_a;
    int64_t* out_b;
    double* out_sep;
    long long out_cap;          // slots of the pair list
    const int32_t* lrow;        // batch: batch-wide A row -> request row
    int32_t* err;               // status bits
    unsigned long long* stats;  // candidates, rechecked, flipped, members, tie_resolved
};

// Bounds of one A source's search: zones [z0, z1] and up to two ra_key
// segments (the RA window, split at 0/360). Float32 and integer arithmetic on
// the fixed-point position, widened so it contains every source within the
// bounding radius.
struct Window {
    int32_t z0, z1, nseg;
    uint32_t lo[2], hi[2];
};

__device__ __forceinline__ Window a_window(const APrep& A, const IndexGeom& G) {
    Window W;
    const float Rm = A.R * (1.0f + 1e-5f) + 1e-9f;
    const float dz = Rm / G.h_f * (1.0f + 1e-5f) + 1e-3f;  // zones, with margin
    const float t = A.zfrac + 0.5f;                       // position inside zone A.z
    const int32_t z0 = A.z + (int32_t)floorf(t - dz);
    const int32_t z1 = A.z + (int32_t)floorf(t + dz);
    bool full = z0 < 0 || z1 >= G.nz;  // the window reaches a pole
    W.z0 = max(z0, 0);
    W.z1 = min(z1, G.nz - 1);
    int64_t dk = 0;
    if (!full) {
        // half-width of the RA window: asin(sin R / cos dec), bounded by
        // asin(R / cos dec) and widened
        const ZoneHot Z = load_zone_hot(G.zhot + A.z);
        const LatTerms L = lat_terms(G.h_f * A.zfrac, Z.sin_cf, Z.cos_cf);
        const float ratio = Rm / L.cd;  // (sin Rm <= Rm: a window no narrower)
        if (!(L.cd > 0.0f && ratio < 0.9999f)) full = true;
        else dk = (int64_t)(int32_t)ceilf(asinf(ratio) * (1.0f + 2e-5f) * kKey32PerRadF) + 2;  // < 2^30
    }
    // stored B keys are rounded down to a multiple of 256: widen the low end
    const int64_t ka = (int64_t)(A.key64 >> 32);
    const int64_t lo = ka - dk - 256, hi = ka + dk;
    if (full || hi - lo >= 4294967295LL) {
        W.nseg = 1;
        W.lo[0] = 0;
        W.hi[0] = 0xFFFFFFFFu;
    } else if (lo < 0) {
        W.nseg = 2;
        W.lo[0] = 0;
        W.hi[0] = (uint32_t)hi;
        W.lo[1] = (uint32_t)(lo + 4294967296LL);
        W.hi[1] = 0xFFFFFFFFu;
    } else if (hi > 4294967295LL) {
        W.nseg = 2;
        W.lo[0] = 0;
        W.hi[0] = (uint32_t)(hi - 4294967296LL);
        W.lo[1] = (uint32_t)lo;
        W.hi[1] = 0xFFFFFFFFu;
    } else {
        W.nseg = 1;
        W.lo[0] = (uint32_t)lo;
        W.hi[0] = (uint32_t)hi;
    }
    return W;
}

// Rows [lo, hi) of a zone holding every row whose ra_key lies in
// [klo, khi]: the whole buckets of the zone's RA bucket table that the key
// window touches (about one source per bucket), from two table reads and no
// search; the candidates' own keys are compared with the window as they are
// read. Keys outside the zone's key range clamp to its first or last bucket.
// (Searching the bounds inside the buckets cut the rows read but measured
// slower: its dependent loads cost more than the extra candidate rounds.)
__device__ __forceinline__ void bucket_bounds(const IndexGeom& G, const ZoneHot& Z, uint32_t klo,
                                              uint32_t khi, int64_t* lo_out, int64_t* hi_out) {
    const int64_t start = Z.start;
    if (khi < Z.lut_kmin) {  // the whole window lies before the zone's first key
        *lo_out = *hi_out = start;
        return;
    }
    const uint32_t shift = Z.shift_lg & 0xFFu;
    const uint32_t last = (1u << (Z.shift_lg >> 8)) - 1u;
    const uint32_t* L = G.lut + (2 * start + Z.lut_rel);
    const uint32_t bl = klo <= Z.lut_kmin ? 0u : min((klo - Z.lut_kmin) >> shift, last);
    const uint32_t bh = min((khi - Z.lut_kmin) >> shift, last);
    *lo_out = start + __ldg(&L[bl]);
    *hi_out = start + __ldg(&L[bh + 1]);
}

// Float64 unit vector of B row `row` (exact positions are kept by row).
__device__ __forceinline__ void load_p64(const IndexGeom& G, int32_t row, double* x, double* y,
                                         double* z) {
    if (G.px) {
        *x = G.px[row];
        *y = G.py[row];
        *z = G.pz[row];
    } else {
        const double2 p = G.pos[row];
        unit64_deg(p.x, p.y, x, y, z);
    }
}

__device__ __forceinline__ void warp_add(unsigned long long* dst, uint32_t v) {
    const uint32_t s = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dst, (unsigned long long)s);
}

// Terms of one (A source, zone) item shared by all its candidates: A's
// latitude relative to the zone centre and A's RA key multiplied by the
// zone's cell count.
struct ItemTerms {
    float sdd, hav_d, cd, sd;  // LatTerms of A in this zone
    float sinc, cosc;          // zone centre
    float binw, ufrac;         // cell width; fractional cell of A, minus 1/2
    uint32_t binA, nbins;      // integer cell of A (exact product), cells
};

__device__ __forceinline__ ItemTerms item_terms(const APrep& A, const ZoneHot& Z, int32_t z,
                                                float h_f) {
    ItemTerms t;
    const LatTerms L = lat_terms(h_f * ((float)(A.z - z) + A.zfrac), Z.sin_cf, Z.cos_cf);
    t.sdd = L.sdd;
    t.hav_d = L.hav_d;
    t.cd = L.cd;
    t.sd = L.sd;
    t.sinc = Z.sin_cf;
    t.cosc = Z.cos_cf;
    t.binw = Z.binw_f;
    t.nbins = Z.nbins;
    t.binA = (uint32_t)__umul64hi(A.key64, (uint64_t)Z.nbins);
    t.ufrac = (float)(uint32_t)((A.key64 * (uint64_t)Z.nbins) >> 40) * 5.9604644775390625e-08f - 0.5f;
    return t;
}

// Float32 region test of candidate b against A (no float64 operation).
// Returns q (quadratic form; max form for rectangles) and the east/north
// components (x, y) of b in A's frame.
__device__ __forceinline__ float q32(const APrep& A, int shape, const ItemTerms& T, const BRec& b,
                                     float* xo, float* yo) {
    const uint32_t bin = bin_of(b.ra_key, T.nbins);
    int32_t d = (int32_t)(T.binA - bin);  // cells from B's cell to A's, wrapped at 0/360
    if (d > (int32_t)(T.nbins >> 1)) d -= (int32_t)T.nbins;
    else if (d < -(int32_t)(T.nbins >> 1)) d += (int32_t)T.nbins;
    const float dra = T.binw * ((float)d + T.ufrac);
    float sa, hav_a;
    sin_hav(dra, &sa, &hav_a);
    // A's offsets in the cell frame
    const float xa = T.cd * sa;
    const float ya = fmaf(T.cd * T.sinc, hav_a, T.sdd);
    const float za = -fmaf(T.cd * T.cosc, hav_a, T.hav_d);
    // cell frame -> A's east/north frame
    const float j00 = 1.0f - hav_a, j01 = T.sinc * sa, t0 = -T.cosc * sa;
    const float j10 = -T.sd * sa, j11 = (1.0f - T.hav_d) - T.sd * T.sinc * hav_a;
    const float t1 = fmaf(T.sd * T.cosc, hav_a, -T.sdd);
    const float dxi = b.xi - xa, deta = b.eta - ya;
    const float dz = zeta_of(b.xi, b.eta) - za;
    const float x = fmaf(j00, dxi, fmaf(j01, deta, t0 * dz));
    const float y = fmaf(j10, dxi, fmaf(j11, deta, t1 * dz));
    *xo = x;
    *yo = y;
    const float u0 = fmaf(A.m00, x, A.m01 * y);
    const float u1 = fmaf(A.m10, x, A.m11 * y);
    return shape == XM_RECT ? fmaxf(fabsf(u0), fabsf(u1)) : fmaf(u0, u0, u1 * u1);
}

// ---------------------------------------------------------------- the scan
//
// One warp owns a chunk of up to 32 A sources (consecutive in (zone, RA)
// order, or from a list). Work is flattened twice so all lanes stay busy
// whatever the region sizes: first the (source, zone, RA segment) items,
// whose window bounds lanes find in parallel, then the candidates of those
// items, 32 per round, loaded with consecutive lanes on consecutive rows.
// Members of a round are folded per source with a segmented warp reduction
// (lanes of one source are contiguous), so every per-source result is
// independent of timing; shared memory keeps the running state. In count
// mode every member is also streamed to a record arena (one atomic per round
// and warp) from which the pair list is placed without scanning again.
//
// Keys of the best-pair fold are the bit patterns of non-negative numbers,
// compared as integers: float32 separations for sources on the float32 path,
// float64 separations otherwise (one kind per source).

constexpr int kScanWarps = 4;
constexpr int kScanThreads = 32 * kScanWarps;
constexpr int kItemCap = 32;
constexpr long long kKeyInf = 0x7FF0000000000000LL;  // above every finite key of either kind

union ASlot {
    A64 a64;
    ACold cold;
};

// The prepared sources of a chunk and the terms of its items, laid out by
// field: lanes reading the fields of different sources or items hit
// different banks (a record per source or item, 48 or 40 bytes apart,
// would put several of them in one bank).
struct ASoA {
    uint64_t key64[32];
    int32_t z[32], row[32], shape[32];
    float zfrac[32], R[32], g[32];
    float m00[32], m01[32], m10[32], m11[32];
};

__device__ __forceinline__ void put_a(ASoA& S, int l, const APrep& A) {
    S.key64[l] = A.key64;
    S.z[l] = A.z;
    S.row[l] = A.row;
    S.shape[l] = A.shape;
    S.zfrac[l] = A.zfrac;
    S.R[l] = A.R;
    S.g[l] = A.g;
    S.m00[l] = A.m00;
    S.m01[l] = A.m01;
    S.m10[l] = A.m10;
    S.m11[l] = A.m11;
}

__device__ __forceinline__ APrep get_a(const ASoA& S, int l) {
    APrep A;
    A.key64 = S.key64[l];
    A.z = S.z[l];
    A.row = S.row[l];
    A.shape = S.shape[l];
    A.zfrac = S.zfrac[l];
    A.R = S.R[l];
    A.g = S.g[l];
    A.m00 = S.m00[l];
    A.m01 = S.m01[l];
    A.m10 = S.m10[l];
    A.m11 = S.m11[l];
    return A;
}

template <int N>
struct TSoA {
    float sdd[N], hav_d[N], cd[N], sd[N], sinc[N], cosc[N], binw[N], ufrac[N];
    uint32_t binA[N], nbins[N];
};

template <int N>
__device__ __forceinline__ void put_t(TSoA<N>& S, int k, const ItemTerms& T) {
    S.sdd[k] = T.sdd;
    S.hav_d[k] = T.hav_d;
    S.cd[k] = T.cd;
    S.sd[k] = T.sd;
    S.sinc[k] = T.sinc;
    S.cosc[k] = T.cosc;
    S.binw[k] = T.binw;
    S.ufrac[k] = T.ufrac;
    S.binA[k] = T.binA;
    S.nbins[k] = T.nbins;
}

template <int N>
__device__ __forceinline__ ItemTerms get_t(const TSoA<N>& S, int k) {
    ItemTerms T;
    T.sdd = S.sdd[k];
    T.hav_d = S.hav_d[k];
    T.cd = S.cd[k];
    T.sd = S.sd[k];
    T.sinc = S.sinc[k];
    T.cosc = S.cosc[k];
    T.binw = S.binw[k];
    T.ufrac = S.ufrac[k];
    T.binA = S.binA[k];
    T.nbins = S.nbins[k];
    return T;
}

struct ScanWarpSmem {
    ASoA A;
    int32_t sidx[32];          // index of each source in P.A / P.Ac
    ASlot ac[32];              // float64 basis of sources on float64 separations; with a
                               // fused preparation, the float64 part of the others
    long long m1[32], m2[32];  // best key, second key
    long long r1[32];          // reported separation of the best (bits)
    int32_t b1[32];
    int32_t cnt[32];
    int32_t cap[32];           // emit mode: count-pass members
    int32_t drop[32];          // count mode: a member did not fit the arena
    float g[32], esep[32];
    int32_t sep64[32];
    int32_t z0[32], nseg[32];
    uint32_t wlo[32][2], whi[32][2];
    int32_t ipref[33];         // first item of each source
    int32_t it_a[kItemCap];
    uint32_t it_klo[kItemCap], it_khi[kItemCap];  // the item's key window
    int64_t it_lo[kItemCap];
    int32_t it_start[kItemCap + 1];  // first candidate of each item
    TSoA<kItemCap> it_t;
};

// FUSED: the sources are the caller's A rows in input order (P.in), and the
// scan prepares each one itself instead of reading a prepared record; the
// count pass then also stores the float64 part of every source with members
// (P.acold_out), which later float64 decisions on the result read.
template <int PREC, int MODE, bool FUSED = false>
__global__ void __launch_bounds__(kScanThreads, 6) k_scan(ScanArgs P) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char scan_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ScanWarpSmem& W = reinterpret_cast<ScanWarpSmem*>(scan_smem)[warp];
    const IndexGeom& G = P.G;
    const int64_t n_units = P.list ? (P.nlist_dev ? (int64_t)*P.nlist_dev : P.nlist) : P.nA;
    const uint32_t lt_mask = (1u << lane) - 1u;
    A64 a_own;  // float64 basis for band rechecks of float32-path sources
    int a_own_for = -1;
    int max_cnt = 0;  // (count mode) the largest member count of this lane's sources
    uint32_t n_cand = 0, n_re = 0, n_flip = 0, n_mem = 0;
    int64_t chunk = (int64_t)blockIdx.x * kScanWarps + warp;
    // persistent mode: warps take 32-source chunks from the queue until it
    // runs dry; otherwise each warp does one chunk
    for (;;) {
    if (P.queue) {
        unsigned int c = 0;
        if (lane == 0) c = atomicAdd(P.queue, 1u);
        chunk = __shfl_sync(0xffffffffu, c, 0);
    }
    const int64_t first = chunk * 32;
    if (first >= n_units) break;  // whole warp
    const int nloc = (int)min((int64_t)32, n_units - first);
    a_own_for = -1;

    // ---- per-source setup (lane = source)
    int64_t s_me = -1;
    int n_items = 0;
    if (lane < nloc) {
        s_me = P.list ? P.list[first + lane] : first + lane;
        APrep A;
        ACold C;
        if (FUSED) prep_one(P.in, s_me, MODE == kModeCount ? P.err : nullptr, &A, &C);
        else A = P.A[s_me];
        put_a(W.A, lane, A);
        W.sidx[lane] = (int32_t)s_me;
        // float32 error bounds: g (from the preparation) bounds |q32 - q|;
        // esep bounds the float32 separation error (rad)
        const float L_mem = A.R + 2.0f * G.h_f;
        W.g[lane] = A.g;
        W.esep[lane] = 16.0f * kEps32 * L_mem;
        const bool s64 = PREC == kPrecFP64 || MODE == kModeResolve ||
                         W.esep[lane] * 206264.8f > 9e-5f;
        W.sep64[lane] = s64;
        if (s64 && A.R > 0.0f) W.ac[lane].a64 = make_a64(FUSED ? C : P.Ac[s_me]);
        else if (FUSED) W.ac[lane].cold = C;
        W.m1[lane] = kKeyInf;
        W.m2[lane] = kKeyInf;
        W.r1[lane] = 0;
        W.b1[lane] = 0x7fffffff;
        W.cnt[lane] = 0;
        W.drop[lane] = 0;
        W.cap[lane] = MODE == kModeEmit ? P.count[A.row] : 0;
        if (A.R > 0.0f) {
            const Window w = a_window(A, G);
            W.z0[lane] = w.z0;
            W.nseg[lane] = w.nseg;
            W.wlo[lane][0] = w.lo[0];
            W.whi[lane][0] = w.hi[0];
            W.wlo[lane][1] = w.lo[1];
            W.whi[lane][1] = w.hi[1];
            n_items = (w.z1 - w.z0 + 1) * w.nseg;
        } else {
            W.nseg[lane] = 1;
            W.z0[lane] = 0;
        }
    }
    // exclusive prefix of item counts over sources
    int incl = n_items;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    W.ipref[lane] = incl - n_items;
    const int total_items = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 31) W.ipref[32] = total_items;
    __syncwarp();

    for (int t0 = 0; t0 < total_items; t0 += kItemCap) {
        const int nb = min(kItemCap, total_items - t0);
        // ---- items: (source, zone, segment) -> candidate row range + terms
        for (int k = lane; k < nb; k += 32) {
            const int t = t0 + k;
            int al = 0;  // last source whose first item <= t
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (al + step < nloc && W.ipref[al + step] <= t) al += step;
            const int r = t - W.ipref[al];
            const int ns = W.nseg[al];
            const int z = W.z0[al] + (ns == 2 ? r >> 1 : r), sg = ns == 2 ? r & 1 : 0;
            const ZoneHot Z = load_zone_hot(G.zhot + z);
            const uint32_t klo = W.wlo[al][sg], khi = W.whi[al][sg];
            int64_t lo, hi;
            bucket_bounds(G, Z, klo, khi, &lo, &hi);
            W.it_a[k] = al;
            W.it_klo[k] = klo;
            W.it_khi[k] = khi;
            W.it_lo[k] = lo;
            W.it_start[k] = (int32_t)(hi - lo);  // count, scanned below
            if (PREC == kPrecFP32 && hi > lo) put_t(W.it_t, k, item_terms(get_a(W.A, al), Z, z, G.h_f));
        }
        __syncwarp();
        // exclusive scan of item candidate counts (nb <= 64: 2 per lane)
        {
            int v[kItemCap / 32];
            int sum = 0;
#pragma unroll
            for (int q = 0; q < kItemCap / 32; q++) {
                const int k = lane * (kItemCap / 32) + q;
                v[q] = k < nb ? W.it_start[k] : 0;
                sum += v[q];
            }
            int inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            int run = inc - sum;
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kItemCap / 32; q++) {
                const int k = lane * (kItemCap / 32) + q;
                if (k < nb) W.it_start[k] = run;
                run += v[q];
            }
            if (lane == 31) W.it_start[nb] = inc;
        }
        __syncwarp();
        const int total_cand = W.it_start[nb];

        // ---- candidates, 32 per round. The records of the next round are
        // loaded before this round is tested, so consecutive rounds' loads
        // overlap the tests. A lane's record belongs to its item's bucket
        // range; it is a candidate when its own key lies in the item's window.
        int kp = 0;  // item of the prefetched candidate; only moves forward
        int nxt_k = 0;
        BRec nxt;
        auto fetch = [&](int c) {
            const int cc = c < total_cand ? c : total_cand - 1;
            while (W.it_start[kp + 1] <= cc) kp++;  // last item with start <= c
            nxt_k = kp;
            if (c < total_cand) nxt = load_brec(G.rec + W.it_lo[kp] + (c - W.it_start[kp]));
        };
        if (total_cand > 0) fetch(lane);
        for (int c0 = 0; c0 < total_cand; c0 += 32) {
            const int c = c0 + lane;
            const bool active = c < total_cand;
            const int k = nxt_k;
            const BRec b = nxt;
            if (c0 + 32 < total_cand) fetch(c0 + 32 + lane);
            const int al = W.it_a[k];
            bool is_mem = false;
            long long key = kKeyInf, rep = 0;
            int32_t brow = 0x7fffffff;
            bool rep32 = false;
            if (active && b.ra_key >= W.it_klo[k] && b.ra_key <= W.it_khi[k]) {
                const APrep A = get_a(W.A, al);
                brow = b.row;
                n_cand++;
                const bool s64 = W.sep64[al];
                bool need64 = PREC == kPrecFP64;
                float x = 0.f, y = 0.f;
                bool maybe = true, band = false, in32 = false;
                if (PREC == kPrecFP32) {
                    // q <= 1 - g: inside; q > 1 + g: outside; between: float64
                    const float q = q32(A, A.shape, get_t(W.it_t, k), b, &x, &y);
                    const float g = W.g[al];
                    maybe = q <= 1.0f + g;
                    if (maybe) {
                        band = q >= 1.0f - g;
                        in32 = q <= 1.0f;
                        need64 = band || s64;
                        n_re += band;
                        is_mem = !need64;
                    }
                }
                double exact = 0.0;
                if (maybe && need64) {
                    const A64* a64 = &W.ac[al].a64;
                    if (!s64) {  // band recheck of a float32-path source
                        if (a_own_for != al) {
                            a_own = make_a64(FUSED ? W.ac[al].cold : P.Ac[W.sidx[al]]);
                            a_own_for = al;
                        }
                        a64 = &a_own;
                    }
                    double px, py, pz, rho;
                    load_p64(G, b.row, &px, &py, &pz);
                    const bool in = test64(*a64, A.shape, px, py, pz, &rho);
                    n_flip += band && in != in32;
                    is_mem = in;
                    exact = rho * kRadToArcsec;
                }
                if (is_mem) {
                    n_mem++;
                    if (s64 && MODE != kModeResolve) {
                        rep = __double_as_longlong(exact);
                        key = rep;
                    } else {
                        const float s2 = fmaf(x, x, y * y);
                        const float rho32 = s2 < 1e-6f ? sqrtf(s2) * fmaf(s2, 1.0f / 6.0f, 1.0f)
                                                       : asinf(sqrtf(s2));
                        rep = (long long)__float_as_int(rho32);
                        rep32 = true;
                        // resolve mode ranks by the float64 separation but
                        // reports the float32 one, as the count pass did
                        key = MODE == kModeResolve ? __double_as_longlong(exact) : rep;
                    }
                }
            }
            const uint32_t mem_mask = __ballot_sync(0xffffffffu, is_mem);
            if (mem_mask == 0) continue;  // nothing to fold this round
            // ---- fold this round's members per source (segmented over lanes)
            const uint32_t same = __match_any_sync(0xffffffffu, active ? al : -1);
            const int rank = __popc(mem_mask & same & lt_mask);
            const int seg_mem = __popc(mem_mask & same);
            long long m1 = key, m2 = kKeyInf, r1 = rep;
            int32_t b1 = is_mem ? brow : 0x7fffffff;
            // the lane that folds a source's members into shared memory: its
            // only member lane, or the segment head after a reduction
            bool leader = is_mem && rank == 0;
            if (__any_sync(0xffffffffu, seg_mem > 1)) {
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long om1 = __shfl_down_sync(0xffffffffu, m1, o);
                    const long long om2 = __shfl_down_sync(0xffffffffu, m2, o);
                    const long long or1 = __shfl_down_sync(0xffffffffu, r1, o);
                    const int32_t ob1 = __shfl_down_sync(0xffffffffu, b1, o);
                    const bool same_seg = lane + o < 32 && ((same >> (lane + o)) & 1u);
                    if (same_seg) {
                        if (om1 < m1 || (om1 == m1 && ob1 < b1)) {
                            m2 = min(m1, om2);
                            m1 = om1;
                            b1 = ob1;
                            r1 = or1;
                        } else {
                            m2 = min(m2, om1);
                        }
                    }
                }
                leader = active && (same & lt_mask) == 0 && seg_mem > 0;
            }
            const int base = active ? W.cnt[al] : 0;
            // arena space for this round's members (count mode, all pairs)
            long long abase = 0;
            if (MODE == kModeCount && P.arena) {
                if (lane == 0)
                    abase = (long long)atomicAdd(P.arena_n, (unsigned long long)__popc(mem_mask));
                abase = __shfl_sync(0xffffffffu, abase, 0);
            }
            __syncwarp();
            if (is_mem) {
                const int idx = base + rank;
                const int32_t a_row = W.A.row[al];
                if (MODE == kModeCount) {
                    if (P.arena) {
                        const long long slot = abase + __popc(mem_mask & lt_mask);
                        if (slot < P.arena_cap) {
                            MemberRec r;
                            r.a_row = a_row;
                            r.k = idx;
                            r.b_row = brow;
                            r.f32 = rep32;
                            r.sep = __longlong_as_double(rep);
                            P.arena[slot] = r;
                        } else {
                            W.drop[al] = 1;
                        }
                    }
                } else if (MODE == kModeEmit) {
                    if (idx < W.cap[al] && P.pair_off[a_row] + idx < P.out_cap) {
                        const int64_t o = P.pair_off[a_row] + idx;
                        P.out_a[o] = P.lrow ? P.lrow[a_row] : a_row;
                        P.out_b[o] = brow;
                        P.out_sep[o] = rep32 ? (double)__int_as_float((int)rep) * kRadToArcsec
                                             : __longlong_as_double(rep);
                    }
                }
            }
            if (leader) {
                W.cnt[al] = base + seg_mem;
                const long long c1 = W.m1[al];
                const int32_t cb = W.b1[al];
                if (m1 < c1 || (m1 == c1 && b1 < cb)) {
                    W.m2[al] = min(c1, min(m2, W.m2[al]));
                    W.m1[al] = m1;
                    W.b1[al] = b1;
                    W.r1[al] = r1;
                } else {
                    W.m2[al] = min(W.m2[al], m1);
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }

    // ---- per-source results (lane = source)
    if (lane < nloc) {
        const APrep A = get_a(W.A, lane);
        const int cnt = W.cnt[lane];
        const bool s64 = W.sep64[lane] && MODE != kModeResolve;
        const double best_sep = cnt == 0 ? NAN
                                : s64    ? __longlong_as_double(W.r1[lane])
                                         : (double)__int_as_float((int)W.r1[lane]) * kRadToArcsec;
        if (MODE == kModeCount) {
            P.count[A.row] = cnt;
            max_cnt = max(max_cnt, cnt);
            if (FUSED && P.acold_out && cnt > 0) {
                ACold C = W.ac[lane].cold;
                if (W.sep64[lane]) {  // (its slot holds the float64 basis)
                    APrep Q;
                    prep_one(P.in, s_me, nullptr, &Q, &C);
                }
                P.acold_out[A.row] = C;
            }
            if (P.want_best) {
                P.best_b[A.row] = cnt ? (int64_t)W.b1[lane] : -1;
                P.best_sep[A.row] = best_sep;
                // float32 separations within twice their error bound of the
                // smallest: decide the best pair in float64
                if (PREC == kPrecFP32 && !s64 && cnt > 1 &&
                    __int_as_float((int)W.m2[lane]) - __int_as_float((int)W.m1[lane]) <=
                        2.0f * W.esep[lane])
                    P.tie_list[atomicAdd(&P.list_n[1], 1)] = (int32_t)s_me;
            }
            if (W.drop[lane]) P.ovf_list[atomicAdd(&P.list_n[0], 1)] = (int32_t)s_me;
            if (P.arena && cnt > kSegMax) P.big_list[atomicAdd(&P.list_n[2], 1)] = A.row;
        } else if (MODE == kModeEmit) {
            if (cnt != W.cap[lane]) atomicOr(P.err, kErrOverflow);  // passes disagree
        } else {
            // resolve: the float64 best pair, with its float32 separation as
            // the count pass reports it, so the pair list and best row agree
            P.best_b[A.row] = W.b1[lane];
            P.best_sep[A.row] = best_sep;
            atomicAdd(&P.stats[4], 1ull);
        }
    }
    __syncwarp();
    if (!P.queue) break;
    }  // chunks
    if (MODE == kModeCount) {
        warp_add(&P.stats[0], n_cand);
        warp_add(&P.stats[1], n_re);
        warp_add(&P.stats[2], n_flip);
        warp_add(&P.stats[3], n_mem);
        const int wm = __reduce_max_sync(0xffffffffu, max_cnt);
        if (P.max_count && lane == 0 && wm > 0) atomicMax(P.max_count, wm);
    }
}

constexpr size_t kScanSmem = sizeof(ScanWarpSmem) * kScanWarps;

// ------------------------------------------------ the sparse count pass
//
// The count pass for regions that are small against the zone height, where a
// source meets one or two zone items and a few records (the all-sky case):
// one lane per source from its preparation to its results, with the running
// state in registers instead of the flattened item and candidate rounds of
// k_scan. A lane finds its items' bucket ranges at once; then the warp steps
// through the lanes' records together, one record per lane and step (the next
// one loaded while this one is tested), so the step's members can be staged
// in shared memory and written to the record arena with one atomic per warp
// and stage. The best-pair fold and the member indices are the count pass's
// (sequential per source, the same minimum, second minimum and lowest-row
// tie). Sources outside this shape -- more than two items, more than
// kSrcMaxRec records in their ranges, or float64 separations -- are listed
// (`defer`) and counted by k_scan over the list afterwards, in the same
// outputs.

constexpr int kSrcMaxRec = 48;  // records a lane takes on; more go to k_scan
constexpr int kSrcStage = 64;   // member records staged per warp

constexpr int kSrcBuf = 128;    // records of a chunk loaded together

struct SrcWarpSmem {
    BRec buf[kSrcBuf];  // the chunk's records, lane after lane
    MemberRec rec[kSrcStage];
    ACold cold[32];  // float64 part of each lane's source
    int32_t first[33];       // first record of each lane in buf (prefix)
    int32_t lo0[32], lo1[32], n0[32];  // each lane's rows
    uint8_t who[kSrcStage];  // lane of each staged record
    int32_t drop[32];        // a member of the lane's source did not fit the arena
};

constexpr size_t kSrcSmem = sizeof(SrcWarpSmem) * kScanWarps;

// The float64 decision of a candidate in the guard band (rare), out of line
// so its registers are not held across the record loop.
__device__ __noinline__ bool recheck64(const ACold* C, int shape, const double2* pos,
                                       const double* ux, const double* uy, const double* uz,
                                       int32_t row) {
    const A64 a64 = make_a64(*C);
    double px, py, pz, rho;
    if (ux) {
        px = ux[row];
        py = uy[row];
        pz = uz[row];
    } else {
        const double2 p = pos[row];
        unit64_deg(p.x, p.y, &px, &py, &pz);
    }
    return test64(a64, shape, px, py, pz, &rho);
}

__global__ void __launch_bounds__(kScanThreads, 6) k_scan_src(ScanArgs P, int32_t* defer,
                                                              int32_t* n_defer) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char src_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SrcWarpSmem& W = reinterpret_cast<SrcWarpSmem*>(src_smem)[warp];
    const IndexGeom& G = P.G;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t n_cand = 0, n_mem = 0;
    int max_cnt = 0;
    // The region has a fixed size: its prepared terms are the same for every
    // source, except when a frame rotation turns a region that is not a
    // circle (the position angle then varies with the position). They are
    // prepared once per block; each source adds its position.
    const AIn& I = P.in;
    const bool same_region = !I.rotate || I.shape == XM_CIRCLE;
    __shared__ APrep s_at;
    __shared__ ACold s_ct;
    if (threadIdx.x == 0) {
        const double b = I.shape == XM_CIRCLE ? I.a : I.b;
        APrep at;
        ACold ct;
        make_aprep(0.0, 0.0, 0.0, true, I.a, b, I.pa, I.shape, I.pa_dir, I.size_k, I.pa_zero, I.nz,
                   I.h_f, 0, &at, &ct);
        s_at = at;
        s_ct = ct;
        if (blockIdx.x == 0 && P.nA > 0 && !size_ok(I.a, b, I.pa)) atomicOr(P.err, kErrSize);
    }
    __syncthreads();
    // chunks from the queue, the next one claimed while this one runs
    unsigned int next = 0;
    if (lane == 0) next = atomicAdd(P.queue, 1u);
    for (;;) {
        const int64_t this_first = (int64_t)__shfl_sync(0xffffffffu, next, 0) * 32;
        if (this_first >= P.nA) break;  // whole warp
        if (lane == 0) next = atomicAdd(P.queue, 1u);
        W.drop[lane] = 0;

        // ---- preparation, window and bucket ranges (lane = source)
        APrep A;
        bool mine = false;  // this lane's source is counted here
        int n0 = 0, nrec = 0;  // records of item 0, of both items
        int32_t lo0 = 0, lo1 = 0;  // first rows (rows fit 31 bits)
        uint32_t klo0 = 0, khi0 = 0, klo1 = 0, khi1 = 0;
        int32_t z0 = 0, z1 = 0;
        if (this_first + lane < P.nA) {
            const int64_t s = this_first + lane;
            ACold C;
            if (same_region) {
                double lon, lat, gamma;
                bool ok;
                a_position_of(I.lon[s], I.lat[s], I.rotate, I.rot, &lon, &lat, &gamma, &ok);
                if (!ok) atomicOr(P.err, kErrCoord);
                const PosKey k = pos_key(lon, lat, I.nz);
                A = s_at;
                A.key64 = k.key64;
                A.z = k.z;
                A.zfrac = k.zfrac;
                A.row = (int32_t)s;
                if (!ok) {  // (an invalid position matches nothing)
                    A.R = 0.0f;
                    A.g = 0.0f;
                    A.m00 = A.m01 = A.m10 = A.m11 = 0.0f;
                }
                C = s_ct;
                C.lon = lon;
                C.lat = lat;
            } else {
                prep_one(I, s, P.err, &A, &C);
            }
            W.cold[lane] = C;
            mine = 16.0f * kEps32 * (A.R + 2.0f * G.h_f) * 206264.8f <= 9e-5f;  // float32 separations
            if (mine && A.R > 0.0f) {
                const Window w = a_window(A, G);
                const int items = (w.z1 - w.z0 + 1) * w.nseg;
                if (items > 2) {
                    mine = false;
                } else {
                    // item 0: (z0, segment 0); item 1: the next zone, or the
                    // second segment of the same zone
                    z0 = w.z0;
                    z1 = w.nseg == 2 ? w.z0 : w.z0 + 1;
                    klo0 = w.lo[0];
                    khi0 = w.hi[0];
                    klo1 = w.lo[w.nseg - 1];
                    khi1 = w.hi[w.nseg - 1];
                    int64_t l0, h0, l1 = 0, h1 = 0;
                    if (items == 2) bucket_bounds(G, load_zone_hot(G.zhot + z1), klo1, khi1, &l1, &h1);
                    bucket_bounds(G, load_zone_hot(G.zhot + z0), klo0, khi0, &l0, &h0);
                    if ((h0 - l0) + (h1 - l1) > kSrcMaxRec) {
                        mine = false;
                    } else {
                        lo0 = (int32_t)l0;
                        lo1 = (int32_t)l1;
                        n0 = (int)(h0 - l0);
                        nrec = n0 + (int)(h1 - l1);
                    }
                }
            }
            if (!mine) defer[atomicAdd(n_defer, 1)] = (int32_t)s;
        }

        // ---- records: the warp loads the chunk's records together (32 per
        // round, flattened over the lanes, so their loads are in flight at
        // once) into shared memory, kSrcBuf at most; then every lane tests
        // its own, a step per record (records past the buffer are read from
        // memory). Keys are the bit patterns of the float32 separations
        // (non-negative, so ordered as integers).
        if (!mine) nrec = 0;
        int incl = nrec;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int my_first = incl - nrec;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        W.first[lane] = my_first;
        if (lane == 31) W.first[32] = total;
        W.lo0[lane] = lo0;
        W.lo1[lane] = lo1;
        W.n0[lane] = n0;
        __syncwarp();
        const int nbuf = min(total, kSrcBuf);
        for (int c = lane; c < nbuf; c += 32) {
            int ol = 0;  // last lane whose first record is <= c
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (W.first[ol + step] <= c) ol += step;
            const int jj = c - W.first[ol];
            const int32_t row = jj < W.n0[ol] ? W.lo0[ol] + jj : W.lo1[ol] + (jj - W.n0[ol]);
            W.buf[c] = load_brec(G.rec + row);
        }
        __syncwarp();
        int cnt = 0;
        int32_t m1 = 0x7F800000, m2 = 0x7F800000;  // smallest and second smallest key
        int32_t b1 = 0x7fffffff;
        int j = 0, cur = -1;
        ItemTerms T;
        int staged = 0;  // (warp-uniform)
        auto flush = [&]() {
            __syncwarp();
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.arena_n, (unsigned long long)staged);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int i = lane; i < staged; i += 32) {
                if ((long long)(base + i) < P.arena_cap) P.arena[base + i] = W.rec[i];
                else W.drop[W.who[i]] = 1;
            }
            staged = 0;
            __syncwarp();
        };
        while (__any_sync(0xffffffffu, j < nrec)) {
            int32_t key = -1, brow = 0;  // key >= 0: the record is a member
            if (j < nrec) {
                const int it = j < n0 ? 0 : 1;
                const BRec b = my_first + j < kSrcBuf ? W.buf[my_first + j]
                                                      : load_brec(G.rec + (it ? lo1 + (j - n0) : lo0 + j));
                j++;
                if (b.ra_key >= (it ? klo1 : klo0) && b.ra_key <= (it ? khi1 : khi0)) {
                    if (it != cur) {
                        cur = it;
                        const int32_t z = it ? z1 : z0;
                        T = item_terms(A, load_zone_hot(G.zhot + z), z, G.h_f);
                    }
                    n_cand++;
                    float x, y;
                    const float q = q32(A, A.shape, T, b, &x, &y);
                    if (q <= 1.0f + A.g) {
                        bool in = true;
                        if (q >= 1.0f - A.g) {  // the guard band: decided in float64
                            in = recheck64(&W.cold[lane], A.shape, G.pos, G.px, G.py, G.pz, b.row);
                            atomicAdd(&P.stats[1], 1ull);
                            if (in != (q <= 1.0f)) atomicAdd(&P.stats[2], 1ull);
                        }
                        if (in) {
                            const float s2 = fmaf(x, x, y * y);
                            const float rho32 = s2 < 1e-6f ? sqrtf(s2) * fmaf(s2, 1.0f / 6.0f, 1.0f)
                                                           : asinf(sqrtf(s2));
                            key = __float_as_int(rho32);
                            brow = b.row;
                            n_mem++;
                            cnt++;
                            if (key < m1 || (key == m1 && brow < b1)) {
                                m2 = m1;
                                m1 = key;
                                b1 = brow;
                            } else {
                                m2 = min(m2, key);
                            }
                        }
                    }
                }
            }
            if (P.arena) {
                const uint32_t mm = __ballot_sync(0xffffffffu, key >= 0);
                if (mm) {
                    if (staged + __popc(mm) > kSrcStage) flush();
                    if (key >= 0) {
                        const int slot = staged + __popc(mm & lt_mask);
                        MemberRec r;
                        r.a_row = A.row;
                        r.k = cnt - 1;
                        r.b_row = brow;
                        r.f32 = 1;
                        r.sep = __longlong_as_double((long long)key);
                        W.rec[slot] = r;
                        W.who[slot] = (uint8_t)lane;
                    }
                    staged += __popc(mm);
                }
            }
        }
        if (P.arena && staged > 0) flush();
        __syncwarp();

        // ---- results (lane = source)
        if (mine) {
            P.count[A.row] = cnt;
            max_cnt = max(max_cnt, cnt);
            if (P.acold_out && cnt > 0) P.acold_out[A.row] = W.cold[lane];
            if (P.want_best) {
                P.best_b[A.row] = cnt ? (int64_t)b1 : -1;
                P.best_sep[A.row] = cnt ? (double)__int_as_float(m1) * kRadToArcsec : NAN;
                // float32 separations within twice their error bound of the
                // smallest: the best pair is decided in float64
                const float esep = 16.0f * kEps32 * (A.R + 2.0f * G.h_f);
                if (cnt > 1 && __int_as_float(m2) - __int_as_float(m1) <= 2.0f * esep)
                    P.tie_list[atomicAdd(&P.list_n[1], 1)] = A.row;
            }
            if (W.drop[lane]) P.ovf_list[atomicAdd(&P.list_n[0], 1)] = A.row;
        }
        __syncwarp();
    }
    warp_add(&P.stats[0], n_cand);
    warp_add(&P.stats[3], n_mem);
    const int wm = __reduce_max_sync(0xffffffffu, max_cnt);
    if (P.max_count && lane == 0 && wm > 0) atomicMax(P.max_count, wm);
}

// Pair records from the arena to their canonical slots: row a_row, member k.
// In a batch, a_row is batch-wide and lrow maps it to the request's row.
__global__ void k_place(const MemberRec* __restrict__ arena, const unsigned long long* n_rec,
                        long long cap, const int64_t* __restrict__ pair_off,
                        const int32_t* __restrict__ lrow, long long out_cap,
                        int64_t* __restrict__ out_a, int64_t* __restrict__ out_b,
                        double* __restrict__ out_sep) {
    pdl_wait();
    const long long n = min((long long)*n_rec, cap);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const MemberRec r = arena[i];
        const int64_t o = pair_off[r.a_row] + r.k;
        if (o >= out_cap) continue;  // the batch's pair arena is short: rerun
        out_a[o] = lrow ? lrow[r.a_row] : r.a_row;
        out_b[o] = r.b_row;
        out_sep[o] = r.f32 ? (double)__int_as_float((int)__double_as_longlong(r.sep)) * kRadToArcsec
                           : r.sep;
    }
}

// Members of A rows with 2 <= count <= kSmallSort (16) into ascending B row.
// Each warp takes 32 consecutive rows and sorts the qualifying ones two at a
// time, one per half-warp: lane l of the half loads member l (coalesced),
// counts the members of its row with a smaller B row by shuffles across the
// half (B rows of a row are distinct), and stores itself at that rank. Launch
// with 256 threads per block and at least nA / 256 blocks.
__global__ void __launch_bounds__(256) k_sort_small(const int32_t* __restrict__ count,
                                                    const int64_t* __restrict__ pair_off,
                                                    int64_t nA, long long out_cap,
                                                    int64_t* __restrict__ out_b,
                                                    double* __restrict__ out_sep,
                                                    const int32_t* max_count) {
    pdl_wait();
    if (max_count && *max_count < 2) return;  // no row to sort
    static_assert(kSmallSort == 16, "one row per half-warp");
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         base < nA; base += warps * 32) {
        const int64_t mine = base + lane;
        const int32_t cm = mine < nA ? count[mine] : 0;
        unsigned todo = __ballot_sync(0xffffffffu, cm >= 2 && cm <= kSmallSort);
        while (todo) {  // uniform over the warp
            const int r0 = __ffs(todo) - 1;
            todo &= todo - 1;
            const int r1 = todo ? __ffs(todo) - 1 : -1;
            if (todo) todo &= todo - 1;
            const int32_t c0 = __shfl_sync(0xffffffffu, cm, r0);
            const int32_t c1 = __shfl_sync(0xffffffffu, cm, r1 < 0 ? 0 : r1);
            const int r = half ? r1 : r0;
            const int32_t c = r < 0 ? 0 : (half ? c1 : c0);
            const int64_t o = r < 0 ? 0 : pair_off[base + r];
            const bool valid = hl < c && o + c <= out_cap;
            const int64_t kb = valid ? out_b[o + hl] : INT64_MAX;
            const double ks = valid ? out_sep[o + hl] : 0.0;
            int rank = 0;
#pragma unroll
            for (int j = 0; j < 16; j++) rank += __shfl_sync(0xffffffffu, kb, (half << 4) | j) < kb;
            __syncwarp();  // every load of the rows is done before any store
            if (valid) {
                out_b[o + rank] = kb;
                out_sep[o + rank] = ks;
            }
        }
    }
}

// Members of A rows with kSmallSort < count <= kWarpSort into ascending B row,
// one warp per row: every entry's final place is the number of entries with a
// smaller B row (all distinct within a row), counted against a copy in shared
// memory. Warps stride over the rows 32 at a time: one coalesced load of 32
// counts and a ballot find the rows of this size class, so rows of other
// classes cost no dependent load.
constexpr int kWarpSort = 512;
constexpr int kWarpSortWarps = 4;

__global__ void __launch_bounds__(32 * kWarpSortWarps) k_sort_warp(
    const int32_t* __restrict__ count, const int64_t* __restrict__ pair_off, int64_t nA,
    long long out_cap, int64_t* __restrict__ out_b, double* __restrict__ out_sep,
    const int32_t* max_count) {
    pdl_wait();
    if (max_count && *max_count <= kSmallSort) return;  // no row of this size class
    __shared__ int64_t sb[kWarpSortWarps][kWarpSort];
    __shared__ double ss[kWarpSortWarps][kWarpSort];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kWarpSortWarps * 32;
    for (int64_t base = ((int64_t)blockIdx.x * kWarpSortWarps + w) * 32; base < nA; base += stride) {
        const int64_t mine = base + lane;
        const int32_t cm = mine < nA ? count[mine] : 0;
        unsigned todo = __ballot_sync(0xffffffffu, cm > kSmallSort && cm <= kWarpSort);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t row = base + l;
            const int32_t c = __shfl_sync(0xffffffffu, cm, l);
            const int64_t o = pair_off[row];
            if (o + c > out_cap) continue;  // uniform over the warp
            for (int k = lane; k < c; k += 32) {
                sb[w][k] = out_b[o + k];
                ss[w][k] = out_sep[o + k];
            }
            __syncwarp();
            for (int k = lane; k < c; k += 32) {
                const int64_t key = sb[w][k];
                int rank = 0;
                for (int j = 0; j < c; j++) rank += sb[w][j] < key;
                out_b[o + rank] = key;
                out_sep[o + rank] = ss[w][k];
            }
            __syncwarp();
        }
    }
}

// Members of A rows with kWarpSort < count <= kSegMax into ascending B row:
// a bitonic network in shared memory, one block per row. Blocks stride over
// the rows a block's width at a time, each thread checking one count, and sort the rows
// of this size class found in the chunk (no list, so no host
// synchronisation is needed to launch it).
__global__ void __launch_bounds__(256) k_seg_sort(const int32_t* __restrict__ count,
                                                  const int64_t* __restrict__ pair_off, int64_t nA,
                                                  long long out_cap, int64_t* __restrict__ out_b,
                                                  double* __restrict__ out_sep,
                                                  const int32_t* max_count) {
    pdl_wait();
    if (max_count && *max_count <= kWarpSort) return;  // no row of this size class
    __shared__ int64_t kb[kSegMax];
    __shared__ double ks[kSegMax];
    __shared__ int32_t found[256];
    __shared__ int n_found;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nA;
         base += (int64_t)gridDim.x * blockDim.x) {
        if (threadIdx.x == 0) n_found = 0;
        __syncthreads();
        const int64_t mine = base + threadIdx.x;
        if (mine < nA) {
            const int32_t cm = count[mine];
            if (cm > kWarpSort && cm <= kSegMax) found[atomicAdd(&n_found, 1)] = (int32_t)threadIdx.x;
        }
        __syncthreads();
        const int nf = n_found;
        for (int f = 0; f < nf; f++) {
            const int64_t row = base + found[f];
            const int32_t c = count[row];
            const int64_t o = pair_off[row];
            if (o + c > out_cap) continue;  // uniform over the block
            int np = 1;
            while (np < c) np <<= 1;
            for (int k = threadIdx.x; k < np; k += blockDim.x) {
                kb[k] = k < c ? out_b[o + k] : INT64_MAX;
                ks[k] = k < c ? out_sep[o + k] : 0.0;
            }
            __syncthreads();
            for (int size = 2; size <= np; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int k = threadIdx.x; k < np; k += blockDim.x) {
                        const int partner = k ^ stride;
                        if (partner > k) {
                            const bool up = (k & size) == 0;
                            if ((kb[k] > kb[partner]) == up) {
                                const int64_t tb = kb[k];
                                kb[k] = kb[partner];
                                kb[partner] = tb;
                                const double ts = ks[k];
                                ks[k] = ks[partner];
                                ks[partner] = ts;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int k = threadIdx.x; k < c; k += blockDim.x) {
                out_b[o + k] = kb[k];
                out_sep[o + k] = ks[k];
            }
            __syncthreads();
        }
        __syncthreads();  // n_found is reset for the next chunk
    }
}

// Long segments: sort (b_row, position) pairs with the radix sort, then
// permute the segment through a scratch copy.
__global__ void k_seg_keys(const int64_t* __restrict__ b, int64_t n, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint64_t)b[i];
    vals[i] = (uint32_t)i;
}

__global__ void k_seg_permute(const uint32_t* __restrict__ vals, int64_t n,
                              const int64_t* __restrict__ b_in, const double* __restrict__ s_in,
                              int64_t* __restrict__ b_out, double* __restrict__ s_out) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b_out[i] = b_in[vals[i]];
    s_out[i] = s_in[vals[i]];
}

// Shared-memory limits of this translation unit's scan kernels and of the
// sort, set once per device (thread-safe; before any capture that scans).
void prepare_kernels() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    const int sm = (int)kScanSmem;
    cudaFuncSetAttribute(k_scan<kPrecFP32, kModeCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP32, kModeEmit>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP32, kModeResolve>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP64, kModeCount>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP64, kModeEmit>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP32, kModeCount, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP32, kModeEmit, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP32, kModeResolve, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP64, kModeCount, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan<kPrecFP64, kModeEmit, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_scan_src, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSrcSmem);
    radix_sort_prepare();
    done[dev] = true;
}

// Segments of more than kSegMax members (rows listed on the device): radix
// sort of (B row, position) pairs, then a permutation through a scratch copy.
// Rare (regions holding thousands of sources); synchronises the stream.
xm_status sort_long_segments(const int32_t* d_rows, int64_t n_big, xm_result* R, int32_t* err,
                             cudaStream_t s) {
    int32_t* h_big = new (std::nothrow) int32_t[n_big];
    if (!h_big) return set_error(XM_ENOMEM, "host list");
    cudaError_t e = cudaMemcpyAsync(h_big, d_rows, n_big * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    xm_status r = XM_OK;
    for (int64_t k = 0; k < n_big && e == cudaSuccess && r == XM_OK; k++) {
        const int32_t row = h_big[k];
        int32_t c = 0;
        int64_t off = 0;
        e = cudaMemcpyAsync(&c, R->count + row, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&off, R->pair_off + row, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        uint64_t* sk = (uint64_t*)dev_alloc(2 * (size_t)c * sizeof(uint64_t), s);
        uint32_t* sv = (uint32_t*)dev_alloc(2 * (size_t)c * sizeof(uint32_t), s);
        int64_t* cb = (int64_t*)dev_alloc((size_t)c * (sizeof(int64_t) + sizeof(double)), s);
        if (!sk || !sv || !cb) {
            r = set_error(XM_ENOMEM, "segment sort");
        } else {
            double* cs = (double*)(cb + c);
            launch_begin("k_seg_keys", s);
            k_seg_keys<<<(unsigned)((c + 255) / 256), 256, 0, s>>>(R->b_row + off, c, sk, sv);
            e = launch_end("k_seg_keys", s);
            if (e == cudaSuccess) r = radix_sort_u64(sk, sv, sk + c, sv + c, c, 0, 32, err, s);
            if (e == cudaSuccess && r == XM_OK)
                e = cudaMemcpyAsync(cb, R->b_row + off, c * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && r == XM_OK)
                e = cudaMemcpyAsync(cs, R->sep + off, c * sizeof(double), cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && r == XM_OK) {
                launch_begin("k_seg_permute", s);
                k_seg_permute<<<(unsigned)((c + 255) / 256), 256, 0, s>>>(sv, c, cb, cs, R->b_row + off, R->sep + off);
                e = launch_end("k_seg_permute", s);
            }
        }
        dev_free(sk, s);
        dev_free(sv, s);
        dev_free(cb, s);
    }
    delete[] h_big;
    if (e != cudaSuccess) return cuda_fail(e, "segment sort");
    return r;
}

}  // namespace
}  // namespace xm

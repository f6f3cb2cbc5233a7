// xm_match.cu -- the Sky cross-match of paper §2.1 with the selections of
// §2.2, against a resident index of the second catalogue (§2.3).
//
// Pipeline of one xm_match call (A = the first catalogue):
//   k_ingest_a   validity, rotation into the index frame when the frames
//                differ, (zone, ra_key) sort key per A source
//   radix sort   A in (zone, RA) order, so neighbouring threads search
//                neighbouring B ranges
//   k_prep_a     per sorted A: index-frame position, position angle (plus the
//                frame rotation's angle), sizes, bounding radius, float32
//                region map
//   k_scan       per A: zone span and RA window (cos(dec) widening, RA wrap,
//                full ring at the poles), binary search of each zone's
//                RA-sorted run, region test of every candidate, and in one
//                pass: member count, best pair, first 8 members kept inline
//   scan counts  pair offsets in A-row order (deterministic, no atomics on
//                the output)
//   k_emit       inline members sorted by B row into the pair list; A
//                sources with more members are re-scanned in emit mode and
//                their segments sorted
//   k_scan<RESOLVE>  float32 path only: A sources whose two smallest
//                float32 separations lie within their error bound get their
//                best pair decided in float64
#include <math.h>

#include <new>

#include "xm_internal.cuh"

namespace xm {

namespace {

constexpr int kBlock = 256;
constexpr int kSegMax = 2048;  // largest member list sorted in shared memory

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
    double h;        // index zone height (rad)
    int32_t nz;
};

__device__ __forceinline__ bool coord_ok(double lon, double lat) {
    return isfinite(lon) && isfinite(lat) && lat >= -90.0 && lat <= 90.0;
}

// Index-frame (RA, Dec) of A source i and the angle gamma from the index
// frame's north to the input frame's north (east positive) at that point.
__device__ void a_position(const AIn& I, int64_t i, double* ra, double* dec, double* gamma,
                           bool* ok) {
    double lon = I.lon[i], lat = I.lat[i];
    *ok = coord_ok(lon, lat);
    if (!*ok) { lon = 0.0; lat = 0.0; }
    double l = fmod(lon, 360.0);
    if (l < 0) l += 360.0;
    double lam = l * kDeg, bet = lat * kDeg;
    if (!I.rotate) {
        *ra = lam;
        *dec = bet;
        *gamma = 0.0;
        return;
    }
    double sl, cl, sb, cb;
    sincos(lam, &sl, &cl);
    sincos(bet, &sb, &cb);
    const double p[3] = {cb * cl, cb * sl, sb};
    const double nn[3] = {-sb * cl, -sb * sl, cb};
    double q[3], m[3];
    for (int k = 0; k < 3; k++) {
        q[k] = I.rot[3 * k] * p[0] + I.rot[3 * k + 1] * p[1] + I.rot[3 * k + 2] * p[2];
        m[k] = I.rot[3 * k] * nn[0] + I.rot[3 * k + 1] * nn[1] + I.rot[3 * k + 2] * nn[2];
    }
    double rxy = hypot(q[0], q[1]);
    double r = atan2(q[1], q[0]);
    if (r < 0) r += kTwoPi;
    if (r >= kTwoPi) r -= kTwoPi;
    *ra = r;
    *dec = atan2(q[2], rxy);
    double ca = rxy > 0 ? q[0] / rxy : 1.0, sa = rxy > 0 ? q[1] / rxy : 0.0;
    double sd = q[2], cd = rxy;
    // index-frame east / north at the rotated point
    double me = -m[0] * sa + m[1] * ca;
    double mn = -m[0] * sd * ca - m[1] * sd * sa + m[2] * cd;
    *gamma = atan2(me, mn);
}

__global__ void k_ingest_a(AIn I, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           int32_t* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I.n) return;
    double ra, dec, gamma;
    bool ok;
    a_position(I, i, &ra, &dec, &gamma, &ok);
    if (!ok) atomicOr(err, kErrCoord);
    double a = I.a_col ? I.a_col[i] : I.a;
    double b = I.shape == XM_CIRCLE ? a : (I.b_col ? I.b_col[i] : I.b);
    double pa = I.pa_col ? I.pa_col[i] : I.pa;
    if (!(isfinite(a) && isfinite(b) && isfinite(pa) && a >= 0.0 && b >= 0.0))
        atomicOr(err, kErrSize);
    keys[i] = ((uint64_t)zone_of(dec, I.h, I.nz) << 32) | ra_key_of(ra);
    vals[i] = (uint32_t)i;
}

__global__ void k_prep_a(AIn I, const uint32_t* __restrict__ vals, APrep* __restrict__ out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= I.n) return;
    int64_t i = vals[s];
    double ra, dec, gamma;
    bool ok;
    a_position(I, i, &ra, &dec, &gamma, &ok);
    double a = I.a_col ? I.a_col[i] : I.a;
    double b = I.shape == XM_CIRCLE ? a : (I.b_col ? I.b_col[i] : I.b);
    double pa = I.pa_col ? I.pa_col[i] : I.pa;
    if (!(isfinite(a) && isfinite(b) && isfinite(pa) && a >= 0.0 && b >= 0.0)) a = b = pa = 0.0;
    APrep P;
    P.alpha = ra;
    P.delta = dec;
    P.row = (int32_t)i;
    P.a = a * I.size_k;
    P.b = b * I.size_k;
    double th = (I.pa_zero + I.pa_dir * pa) * kDeg + gamma;
    th = remainder(th, kTwoPi);
    P.theta = th;
    if (P.a <= 0.0 || P.b <= 0.0 || !ok) {
        P.R = 0.0f;
        P.m00 = P.m01 = P.m10 = P.m11 = 0.0f;
    } else {
        double R = I.shape == XM_RECT ? hypot(P.a, P.b) : fmax(P.a, P.b);
        P.R = (float)(R * (1.0 + 1e-6));
        float st, ct;
        sincosf((float)th, &st, &ct);
        float ia = (float)(1.0 / P.a), ib = (float)(1.0 / P.b);
        P.m00 = st * ia;
        P.m01 = ct * ia;
        P.m10 = ct * ib;
        P.m11 = -st * ib;
    }
    out[s] = P;
}

struct ScanArgs {
    IndexGeom G;
    const APrep* A;
    int64_t nA;
    int32_t shape;
    int32_t want_best;
    const int32_t* list;  // sorted A indices to process (overflow / ties)
    int64_t nlist;
    // count mode, indexed by A row (count, best, spos) or sorted index (slots)
    int32_t* count;
    int32_t* spos;
    int64_t* best_b;
    double* best_sep;
    Slot* slots;
    int32_t* ovf_list;
    int32_t* tie_list;
    int32_t* list_n;  // [0] overflow, [1] ties
    // emit mode
    const int64_t* pair_off;
    int64_t* out_a;
    int64_t* out_b;
    double* out_sep;
    int32_t* big_list;  // overflow segments too long for the shared-memory sort
    int32_t* err;       // status bits
    unsigned long long* stats;  // candidates, rechecked, flipped, members, tie_resolved
};

// Bounds of one A source's search: zones [z0, z1] and up to two ra_key
// segments (the RA window, split at 0/360).
struct Window {
    int32_t z0, z1, nseg;
    uint32_t lo[2], hi[2];
};

__device__ __forceinline__ Window a_window(const APrep& A, const IndexGeom& G) {
    Window W;
    double Rm = (double)A.R * (1.0 + 1e-6) + 1e-12;
    double dlo = A.delta - Rm, dhi = A.delta + Rm;
    W.z0 = zone_of(fmax(dlo, -kHalfPi), G.h, G.nz);
    W.z1 = zone_of(fmin(dhi, kHalfPi), G.h, G.nz);
    bool full = dhi >= kHalfPi || dlo <= -kHalfPi;
    double dra = 0.0;
    if (!full) {
        // half-width of the RA window: asin(sin R / cos dec), widened
        float cd = sinf((float)(kHalfPi - fabs(A.delta)));  // cos(dec), accurate near poles
        float ratio = sinf((float)Rm) / cd;
        if (!(ratio < 0.9999f)) full = true;
        else dra = (double)asinf(ratio) * (1.0 + 2e-5) + 1e-12;
    }
    if (!full) {
        double lo = floor((A.alpha - dra) * kKeyScale);
        double hi = floor((A.alpha + dra) * kKeyScale);
        if (hi - lo >= 4294967295.0) {
            full = true;
        } else if (lo < 0) {
            W.nseg = 2;
            W.lo[0] = 0;
            W.hi[0] = (uint32_t)hi;
            W.lo[1] = (uint32_t)(lo + 4294967296.0);
            W.hi[1] = 0xFFFFFFFFu;
        } else if (hi > 4294967295.0) {
            W.nseg = 2;
            W.lo[0] = 0;
            W.hi[0] = (uint32_t)(hi - 4294967296.0);
            W.lo[1] = (uint32_t)lo;
            W.hi[1] = 0xFFFFFFFFu;
        } else {
            W.nseg = 1;
            W.lo[0] = (uint32_t)lo;
            W.hi[0] = (uint32_t)hi;
        }
    }
    if (full) {
        W.nseg = 1;
        W.lo[0] = 0;
        W.hi[0] = 0xFFFFFFFFu;
    }
    return W;
}

// first index in [lo, hi) whose ra_key >= key (hi if none)
__device__ __forceinline__ int64_t lower_key(const BRec* __restrict__ rec, int64_t lo, int64_t hi,
                                             uint32_t key) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&rec[mid].ra_key) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// first index in [lo, hi) whose ra_key > key
__device__ __forceinline__ int64_t upper_key(const BRec* __restrict__ rec, int64_t lo, int64_t hi,
                                             uint32_t key) {
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&rec[mid].ra_key) <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void load_p64(const IndexGeom& G, int64_t j, double* x, double* y,
                                         double* z) {
    if (G.px) {
        *x = G.px[j];
        *y = G.py[j];
        *z = G.pz[j];
    } else {
        double2 p = G.pos[j];
        unit64(p.x, p.y, x, y, z);
    }
}

__device__ __forceinline__ void warp_add(unsigned long long* dst, uint32_t v) {
    uint32_t mask = __activemask();
    uint32_t s = __reduce_add_sync(mask, v);
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && s) atomicAdd(dst, (unsigned long long)s);
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(kBlock) k_scan(ScanArgs P) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s;
    if (P.list) {
        if (t >= P.nlist) return;
        s = P.list[t];
    } else {
        if (t >= P.nA) return;
        s = t;
    }
    const APrep A = P.A[s];
    const IndexGeom& G = P.G;
    const int shape = P.shape;
    uint32_t n_cand = 0, n_re = 0, n_flip = 0, n_mem = 0;
    int32_t cnt = 0;
    // best pair: by (sep, b_row); m2 = second smallest separation
    double m1 = INFINITY, m2 = INFINITY, r64 = INFINITY;
    int32_t b1 = 0x7fffffff, r_b = 0x7fffffff;
    double r_rep = NAN;
    int64_t out_base = 0;
    int32_t out_cap = 0;  // emit mode writes at most the count-pass members
    if (MODE == kModeEmit) {
        out_base = P.pair_off[A.row];
        out_cap = P.count[A.row];
    }

    // float32 error bounds of this A source. The float32 offsets of A and of
    // B in a cell frame carry absolute errors below ~7 ulp of the larger of
    // their distance to the cell centre and the zone height, so (x, y) is off
    // by at most ~14 eps L, L the largest such distance: 1.42 R + 2h over the
    // candidate box, R + 2h for members. g bounds the error of q (x 3 margin)
    // plus the azimuthal-equidistant factor (rho/s)^2 - 1 <= R^2/3; esep
    // bounds the error of the float32 separation. When esep could exceed
    // 9e-5 arcsec, members get float64 separations instead.
    const float L_box = 1.42f * A.R + 2.0f * (float)G.h;
    const float L_mem = A.R + 2.0f * (float)G.h;
    const float bmin = (float)fmin(A.a, A.b);
    const float g = 128.0f * kEps32 * L_box / bmin + 0.34f * A.R * A.R + 16.0f * kEps32;
    const float esep = 16.0f * kEps32 * L_mem;
    const bool sep64 = PREC == kPrecFP64 || (double)esep * kRadToArcsec > 9e-5;
    A64 a64;
    bool have64 = false;
    if (PREC == kPrecFP64 || MODE == kModeResolve) {
        a64 = make_a64(A);
        have64 = true;
    }

    if (A.R > 0.0f) {
        const Window W = a_window(A, G);
        for (int32_t z = W.z0; z <= W.z1; z++) {
            const int64_t zs = G.zone_start[z], ze = G.zone_start[z + 1];
            if (zs >= ze) continue;
            const ZoneInfo Z = G.zones[z];
            for (int sg = 0; sg < W.nseg; sg++) {
                const int64_t lo = lower_key(G.rec, zs, ze, W.lo[sg]);
                const int64_t hi = upper_key(G.rec, lo, ze, W.hi[sg]);
                uint32_t cur = 0xFFFFFFFFu;
                CellXf X;
                for (int64_t j = lo; j < hi; j++) {
                    const BRec b = G.rec[j];
                    n_cand++;
                    double rep;       // separation reported for the pair (arcsec)
                    double exact = NAN;  // float64 separation (arcsec), when computed
                    if (PREC == kPrecFP32) {
                        uint32_t bin = bin_of(b.ra_key, Z.nbins);
                        if (bin != cur) {
                            X = cell_xf(A.alpha, A.delta, Z, bin);
                            cur = bin;
                        }
                        float dxi = b.xi - X.xa, deta = b.eta - X.ya;
                        float dz = zeta_of(b.xi, b.eta) - X.za;
                        float x = fmaf(X.j00, dxi, fmaf(X.j01, deta, X.t0 * dz));
                        float y = fmaf(X.j10, dxi, fmaf(X.j11, deta, X.t1 * dz));
                        float u0 = fmaf(A.m00, x, A.m01 * y);
                        float u1 = fmaf(A.m10, x, A.m11 * y);
                        float q = shape == XM_RECT ? fmaxf(fabsf(u0), fabsf(u1))
                                                   : fmaf(u0, u0, u1 * u1);
                        if (q > 1.0f + g) continue;
                        if (q >= 1.0f - g || sep64) {
                            if (!have64) {
                                a64 = make_a64(A);
                                have64 = true;
                            }
                            double px, py, pz, rho;
                            load_p64(G, j, &px, &py, &pz);
                            bool in = test64(a64, shape, px, py, pz, &rho);
                            if (q >= 1.0f - g) {
                                n_re++;
                                if (in != (q <= 1.0f)) n_flip++;
                            }
                            if (!in) continue;
                            exact = rho * kRadToArcsec;
                        }
                        float s2 = fmaf(x, x, y * y);
                        float rho32 = s2 < 1e-6f ? sqrtf(s2) * fmaf(s2, 1.0f / 6.0f, 1.0f)
                                                 : asinf(sqrtf(s2));
                        rep = sep64 ? exact : (double)rho32 * kRadToArcsec;
                        if (MODE == kModeResolve && isnan(exact)) {
                            double px, py, pz, rho;
                            load_p64(G, j, &px, &py, &pz);
                            test64(a64, shape, px, py, pz, &rho);
                            exact = rho * kRadToArcsec;
                        }
                    } else {
                        double px, py, pz, rho;
                        load_p64(G, j, &px, &py, &pz);
                        if (!test64(a64, shape, px, py, pz, &rho)) continue;
                        exact = rho * kRadToArcsec;
                        rep = exact;
                    }
                    // a member
                    n_mem++;
                    if (MODE == kModeCount) {
                        if (cnt < kInlineSlots) {
                            Slot sl;
                            sl.b_row = b.row;
                            sl.pad = 0;
                            sl.sep = rep;
                            P.slots[s * kInlineSlots + cnt] = sl;
                        }
                        if (rep < m1 || (rep == m1 && b.row < b1)) {
                            m2 = fmin(m2, m1);
                            m1 = rep;
                            b1 = b.row;
                        } else {
                            m2 = fmin(m2, rep);
                        }
                    } else if (MODE == kModeEmit) {
                        if (cnt < out_cap) {
                            P.out_a[out_base + cnt] = A.row;
                            P.out_b[out_base + cnt] = b.row;
                            P.out_sep[out_base + cnt] = rep;
                        }
                    } else {  // resolve: best by float64 separation
                        if (exact < r64 || (exact == r64 && b.row < r_b)) {
                            r64 = exact;
                            r_b = b.row;
                            r_rep = rep;
                        }
                    }
                    cnt++;
                }
            }
        }
    }

    if (MODE == kModeCount) {
        P.count[A.row] = cnt;
        P.spos[A.row] = (int32_t)s;
        if (P.want_best) {
            P.best_b[A.row] = cnt ? (int64_t)b1 : -1;
            P.best_sep[A.row] = cnt ? m1 : NAN;
            // float32 separations within twice their error bound of the
            // smallest: decide the best pair in float64
            if (!sep64 && cnt > 1 && m2 - m1 <= 2.0 * (double)esep * kRadToArcsec)
                P.tie_list[atomicAdd(&P.list_n[1], 1)] = (int32_t)s;
        }
        if (cnt > kInlineSlots) P.ovf_list[atomicAdd(&P.list_n[0], 1)] = (int32_t)s;
    } else if (MODE == kModeEmit) {
        if (cnt != out_cap) atomicOr(P.err, kErrOverflow);  // passes disagree: report
        else if (cnt > kSegMax) P.big_list[atomicAdd(&P.list_n[2], 1)] = A.row;
    } else {
        P.best_b[A.row] = r_b;
        P.best_sep[A.row] = r_rep;
    }
    if (MODE == kModeCount) {
        warp_add(&P.stats[0], n_cand);
        warp_add(&P.stats[1], n_re);
        warp_add(&P.stats[2], n_flip);
        warp_add(&P.stats[3], n_mem);
    } else if (MODE == kModeResolve) {
        warp_add(&P.stats[4], 1u);
    }
}

// Inline members (count <= 8) into the pair list, sorted by B row.
__global__ void k_emit(const int32_t* __restrict__ count, const int32_t* __restrict__ spos,
                       const Slot* __restrict__ slots, const int64_t* __restrict__ pair_off,
                       int64_t nA, int64_t* __restrict__ out_a, int64_t* __restrict__ out_b,
                       double* __restrict__ out_sep) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nA) return;
    int32_t c = count[i];
    if (c == 0 || c > kInlineSlots) return;
    const Slot* sl = slots + (int64_t)spos[i] * kInlineSlots;
    int32_t br[kInlineSlots];
    double sp[kInlineSlots];
#pragma unroll
    for (int k = 0; k < kInlineSlots; k++) {
        if (k < c) {
            Slot v = sl[k];
            br[k] = v.b_row;
            sp[k] = v.sep;
        }
    }
    // insertion sort by B row (at most 8 entries, all distinct)
    for (int k = 1; k < c; k++) {
        int32_t kb = br[k];
        double ks = sp[k];
        int m = k - 1;
        while (m >= 0 && br[m] > kb) {
            br[m + 1] = br[m];
            sp[m + 1] = sp[m];
            m--;
        }
        br[m + 1] = kb;
        sp[m + 1] = ks;
    }
    int64_t o = pair_off[i];
    for (int k = 0; k < c; k++) {
        out_a[o + k] = i;
        out_b[o + k] = br[k];
        out_sep[o + k] = sp[k];
    }
}

// Sorts the pair segments of overflow A sources (<= kSegMax members) by B
// row with a bitonic network in shared memory, one block per segment.
__global__ void __launch_bounds__(kBlock) k_seg_sort(const int32_t* __restrict__ list,
                                                     const APrep* __restrict__ A,
                                                     const int32_t* __restrict__ count,
                                                     const int64_t* __restrict__ pair_off,
                                                     int64_t* __restrict__ out_b,
                                                     double* __restrict__ out_sep) {
    __shared__ int64_t kb[kSegMax];
    __shared__ double ks[kSegMax];
    int32_t row = A[list[blockIdx.x]].row;
    int32_t c = count[row];
    if (c > kSegMax) return;
    int64_t o = pair_off[row];
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
                int partner = k ^ stride;
                if (partner > k) {
                    bool up = (k & size) == 0;
                    if ((kb[k] > kb[partner]) == up) {
                        int64_t tb = kb[k]; kb[k] = kb[partner]; kb[partner] = tb;
                        double ts = ks[k]; ks[k] = ks[partner]; ks[partner] = ts;
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
}

// Long segments: sort (b_row, position) pairs with the radix sort, then
// permute the segment through a scratch copy.
__global__ void k_seg_keys(const int64_t* __restrict__ b, int64_t n, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint64_t)b[i];
    vals[i] = (uint32_t)i;
}

__global__ void k_seg_permute(const uint32_t* __restrict__ vals, int64_t n,
                              const int64_t* __restrict__ b_in, const double* __restrict__ s_in,
                              int64_t* __restrict__ b_out, double* __restrict__ s_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    b_out[i] = b_in[vals[i]];
    s_out[i] = s_in[vals[i]];
}

unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

template <int PREC>
xm_status launch_scan(const ScanArgs& a, int mode, int64_t nthreads, int block, cudaStream_t s) {
    if (nthreads <= 0) return XM_OK;
    unsigned g = (unsigned)((nthreads + block - 1) / block);
    if (mode == kModeCount) {
        XM_LAUNCH(PREC == kPrecFP32 ? "k_scan_fp32_count" : "k_scan_fp64_count", g, block, 0, s,
                  (k_scan<PREC, kModeCount>), a);
    } else if (mode == kModeEmit) {
        XM_LAUNCH(PREC == kPrecFP32 ? "k_scan_fp32_emit" : "k_scan_fp64_emit", g, block, 0, s,
                  (k_scan<PREC, kModeEmit>), a);
    } else {
        XM_LAUNCH("k_scan_fp32_resolve", g, block, 0, s, (k_scan<kPrecFP32, kModeResolve>), a);
    }
    return XM_OK;
}

xm_status launch_scan_any(int prec, const ScanArgs& a, int mode, int64_t nthreads, int block,
                          cudaStream_t s) {
    if (prec == XM_PREC_FP32_RECHECK) return launch_scan<kPrecFP32>(a, mode, nthreads, block, s);
    return launch_scan<kPrecFP64>(a, mode, nthreads, block, s);
}

int bits_for(int64_t v) {
    int b = 0;
    while (v > 0) { b++; v >>= 1; }
    return b;
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

}  // namespace

}  // namespace xm

using namespace xm;

static void free_result(xm_result* R) {
    if (!R) return;
    cudaStream_t s = nullptr;
    dev_free(R->count, s);
    dev_free(R->pair_off, s);
    dev_free(R->a_row, s);
    dev_free(R->best_b, s);
    delete R;
}

extern "C" xm_status xm_match(const xm_index* X, const xm_columns* Acols, const xm_region* region,
                              const xm_match_opts* opts, void* stream, xm_result** out) {
    if (!out) return set_error(XM_EINVAL, "xm_match: out is NULL");
    *out = nullptr;
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
    int block = opts->block ? opts->block : 128;
    if (block < 32 || block > 256 || (block & 31))
        return set_error(XM_EINVAL, "xm_match: block must be a multiple of 32 in [32, 256]");

    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    xm_result* R = new (std::nothrow) xm_result();
    if (!R) return set_error(XM_ENOMEM, "xm_match: host allocation");
    cudaGetDevice(&R->device);
    R->selection = sel;
    R->precision = prec;
    R->shape = region->shape;
    R->n_a = nA;
    R->n_b = X->n;
    const int64_t nn = nA > 0 ? nA : 1;
    xm_status st = XM_OK;
    {
        Temps T(s);
        // per-A outputs
        R->count = (int32_t*)dev_alloc(nn * sizeof(int32_t), s);
        R->pair_off = (int64_t*)dev_alloc(nn * sizeof(int64_t), s);
        if (sel & XM_SEL_BEST) {
            R->best_b = (int64_t*)dev_alloc(nn * (sizeof(int64_t) + sizeof(double)), s);
            R->best_sep = R->best_b ? (double*)(R->best_b + nn) : nullptr;
        }
        if (!R->count || !R->pair_off || ((sel & XM_SEL_BEST) && !R->best_b)) {
            free_result(R);
            return set_error(XM_ENOMEM, "xm_match: result arrays");
        }

        auto body = [&]() -> xm_status {
            // A columns on the device
            const double *lon = Acols->lon_deg, *lat = Acols->lat_deg;
            const double *ac = region->a_col, *bc = region->b_col, *pc = region->pa_col;
            if (!Acols->on_device && nA > 0) {
                double* buf = T.get<double>(5 * nA);
                if (!buf) return set_error(XM_ENOMEM, "A input copy");
                const double* src[5] = {lon, lat, ac, bc, pc};
                const double** dst[5] = {&lon, &lat, &ac, &bc, &pc};
                for (int k = 0; k < 5; k++) {
                    if (!src[k]) continue;
                    e = cudaMemcpyAsync(buf + k * nA, src[k], nA * sizeof(double),
                                        cudaMemcpyHostToDevice, s);
                    if (e != cudaSuccess) return cuda_fail(e, "A input copy");
                    *dst[k] = buf + k * nA;
                }
            }
            AIn I;
            I.lon = lon;
            I.lat = lat;
            I.n = nA;
            I.rotate = Acols->frame != X->frame;
            double m[9];
            gal_to_eq(m);
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++)
                    I.rot[3 * r + c] = (Acols->frame == XM_FRAME_GAL) ? m[3 * r + c] : m[3 * c + r];
            I.shape = region->shape;
            I.pa_dir = region->pa_dir;
            I.a = region->a;
            I.b = region->b;
            I.pa = region->pa_deg;
            I.a_col = ac;
            I.b_col = bc;
            I.pa_col = pc;
            I.size_k = region->size_scale * region->size_unit_arcsec * kArcsec;
            I.pa_zero = region->pa_zero_deg;
            I.h = X->h;
            I.nz = X->nz;

            uint64_t* keys = T.get<uint64_t>(2 * nn);
            uint32_t* vals = T.get<uint32_t>(2 * nn);
            APrep* prep = T.get<APrep>(nn);
            int32_t* spos = T.get<int32_t>(nn);
            Slot* slots = T.get<Slot>(nn * kInlineSlots);
            int32_t* lists = T.get<int32_t>(2 * nn);
            int32_t* small = T.get<int32_t>(8);  // [0] err, [1..3] list counts, [4] pad
            int64_t* total = T.get<int64_t>(1);
            unsigned long long* stats = T.get<unsigned long long>(8);
            if (!keys || !vals || !prep || !spos || !slots || !lists || !small || !total || !stats)
                return set_error(XM_ENOMEM, "xm_match: work buffers");
            e = cudaMemsetAsync(small, 0, 8 * sizeof(int32_t), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(stats, 0, 8 * sizeof(unsigned long long), s);
            if (e != cudaSuccess) return cuda_fail(e, "memset");
            int32_t* err = small;
            if (nA > 0) {
                XM_LAUNCH("k_ingest_a", grid_for(nA), kBlock, 0, s, k_ingest_a, I, keys, vals, err);
                xm_status r = radix_sort_u64(keys, vals, keys + nn, vals + nn, nA,
                                             32 + bits_for(X->nz - 1), s);
                if (r != XM_OK) return r;
                XM_LAUNCH("k_prep_a", grid_for(nA), kBlock, 0, s, k_prep_a, I, vals, prep);
            }
            ScanArgs a{};
            a.G = X->geom();
            a.A = prep;
            a.nA = nA;
            a.shape = region->shape;
            a.want_best = (sel & XM_SEL_BEST) != 0;
            a.count = R->count;
            a.spos = spos;
            a.best_b = R->best_b;
            a.best_sep = R->best_sep;
            a.slots = slots;
            a.ovf_list = lists;
            a.tie_list = lists + nn;
            a.list_n = small + 1;
            a.stats = stats;
            a.err = err;
            xm_status r = launch_scan_any(prec, a, kModeCount, nA, block, s);
            if (r != XM_OK) return r;
            r = exclusive_scan_i32(R->count, R->pair_off, nA, total, s);
            if (r != XM_OK) return r;
            // one synchronisation: total pairs, list lengths, error bits
            int32_t h_small[8];
            int64_t h_total = 0;
            e = cudaMemcpyAsync(h_small, small, sizeof(h_small), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&h_total, total, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "xm_match sync");
            if (h_small[0] & kErrCoord) return set_error(XM_EINVAL, "A: NaN/inf or |lat| > 90");
            if (h_small[0] & kErrSize)
                return set_error(XM_EINVAL, "A: negative or non-finite region size or angle");
            const int64_t n_ovf = h_small[1], n_tie = h_small[2];
            R->n_pairs = (sel & XM_SEL_ALL) ? h_total : 0;

            if (sel & XM_SEL_ALL) {
                int64_t np = h_total > 0 ? h_total : 1;
                R->a_row = (int64_t*)dev_alloc(np * (2 * sizeof(int64_t) + sizeof(double)), s);
                if (!R->a_row) return set_error(XM_ENOMEM, "xm_match: %lld pairs", (long long)h_total);
                R->b_row = R->a_row + np;
                R->sep = (double*)(R->b_row + np);
                if (nA > 0)
                    XM_LAUNCH("k_emit", grid_for(nA), kBlock, 0, s, k_emit, R->count, spos, slots,
                              R->pair_off, nA, R->a_row, R->b_row, R->sep);
                if (n_ovf > 0) {
                    ScanArgs b = a;
                    b.list = lists;
                    b.nlist = n_ovf;
                    b.pair_off = R->pair_off;
                    b.out_a = R->a_row;
                    b.out_b = R->b_row;
                    b.out_sep = R->sep;
                    int32_t* big = T.get<int32_t>(n_ovf);
                    if (!big) return set_error(XM_ENOMEM, "overflow list");
                    b.big_list = big;
                    r = launch_scan_any(prec, b, kModeEmit, n_ovf, block, s);
                    if (r != XM_OK) return r;
                    XM_LAUNCH("k_seg_sort", (unsigned)n_ovf, kBlock, 0, s, k_seg_sort, lists, prep,
                              R->count, R->pair_off, R->b_row, R->sep);
                    int32_t h2[4];
                    e = cudaMemcpyAsync(h2, small, sizeof(h2), cudaMemcpyDeviceToHost, s);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                    if (e != cudaSuccess) return cuda_fail(e, "xm_match sync");
                    if (h2[0] & kErrOverflow)
                        return set_error(XM_ECUDA, "xm_match: emit pass disagreed with count pass");
                    const int32_t n_big = h2[3];
                    if (n_big > 0) {
                        // rare: regions holding more than kSegMax sources
                        int32_t* h_big = new (std::nothrow) int32_t[n_big];
                        if (!h_big) return set_error(XM_ENOMEM, "host list");
                        e = cudaMemcpy(h_big, big, n_big * sizeof(int32_t), cudaMemcpyDeviceToHost);
                        for (int32_t k = 0; k < n_big && e == cudaSuccess && r == XM_OK; k++) {
                            int32_t row = h_big[k], c = 0;
                            int64_t off = 0;
                            e = cudaMemcpy(&c, R->count + row, sizeof(int32_t), cudaMemcpyDeviceToHost);
                            if (e == cudaSuccess)
                                e = cudaMemcpy(&off, R->pair_off + row, sizeof(int64_t),
                                               cudaMemcpyDeviceToHost);
                            if (e != cudaSuccess) break;
                            uint64_t* sk = (uint64_t*)dev_alloc(2 * c * sizeof(uint64_t), s);
                            uint32_t* sv = (uint32_t*)dev_alloc(2 * c * sizeof(uint32_t), s);
                            int64_t* cb = (int64_t*)dev_alloc(c * (sizeof(int64_t) + sizeof(double)), s);
                            if (!sk || !sv || !cb) {
                                r = set_error(XM_ENOMEM, "segment sort");
                            } else {
                                double* cs = (double*)(cb + c);
                                launch_begin("k_seg_keys", s);
                                k_seg_keys<<<grid_for(c), kBlock, 0, s>>>(R->b_row + off, c, sk, sv);
                                e = launch_end("k_seg_keys", s);
                                if (e == cudaSuccess)
                                    r = radix_sort_u64(sk, sv, sk + c, sv + c, c, 32, s);
                                if (e == cudaSuccess && r == XM_OK)
                                    e = cudaMemcpyAsync(cb, R->b_row + off, c * sizeof(int64_t),
                                                        cudaMemcpyDeviceToDevice, s);
                                if (e == cudaSuccess && r == XM_OK)
                                    e = cudaMemcpyAsync(cs, R->sep + off, c * sizeof(double),
                                                        cudaMemcpyDeviceToDevice, s);
                                if (e == cudaSuccess && r == XM_OK) {
                                    launch_begin("k_seg_permute", s);
                                    k_seg_permute<<<grid_for(c), kBlock, 0, s>>>(
                                        sv, c, cb, cs, R->b_row + off, R->sep + off);
                                    e = launch_end("k_seg_permute", s);
                                }
                            }
                            dev_free(sk, s);
                            dev_free(sv, s);
                            dev_free(cb, s);
                        }
                        delete[] h_big;
                        if (e != cudaSuccess) return cuda_fail(e, "segment sort");
                        if (r != XM_OK) return r;
                    }
                }
            }
            if ((sel & XM_SEL_BEST) && n_tie > 0 && prec == XM_PREC_FP32_RECHECK) {
                ScanArgs b = a;
                b.list = lists + nn;
                b.nlist = n_tie;
                r = launch_scan_any(prec, b, kModeResolve, n_tie, block, s);
                if (r != XM_OK) return r;
            }
            unsigned long long h_stats[8];
            e = cudaMemcpyAsync(h_stats, stats, sizeof(h_stats), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "xm_match stats");
            stats_add(h_stats);
            return XM_OK;
        };
        st = body();
    }
    if (st != XM_OK) {
        free_result(R);
        return st;
    }
    *out = R;
    return XM_OK;
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

// xm_levels.cu -- the normalised distance of every pair of an "all" result:
// the best pair of each A source by it (a reading of the "best pairs" of
// §2.2) and the levels of concentric scaled regions (§3, ClumpPopulator).
//
//   k_lvl_a64     per A source: float64 sines and cosines of its latitude
//                 and orientation, reciprocals of its semi-axes, once (the
//                 pairs of a source share them)
//   k_lvl_pair    per pair: float64 normalised distance from the exact
//                 positions (from their differences by short series when B
//                 is within half a degree of A, else from unit vectors), its
//                 level among the scales, the count of its copy, the smallest
//                 distance of its A source
//   k_lvl_best    per pair at that smallest distance: the lowest B row
//   k_lvl_finish  per A source: counts made cumulative over the copies, the
//                 best pair written out
//
// Every decision (dist <= s_k, the smallest distance) is taken in float64 on
// the same values, so the levels and best pairs are the float64 ones.
#include <math.h>

#include <new>

#include "xm_internal.cuh"

namespace xm {

constexpr int kMaxScales = 64;

struct Scales {
    double s[kMaxScales];
    int32_t k;
};

}  // namespace xm

struct xm_levels {
    int64_t n_pairs = 0, n_a = 0;
    int32_t n_scales = 0;
    double* dist = nullptr;  // one allocation: dist, best_dist, best_b, level, n_within
    double* best_dist = nullptr;
    int64_t* best_b = nullptr;
    int32_t* level = nullptr;
    int32_t* n_within = nullptr;
    cudaStream_t stream = nullptr;  // the arrays are written, and freed, in its order
};

namespace xm {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }

// What the pairs of an A source share: its position (degrees), the sine and
// cosine of its latitude and orientation, its semi-axes and their
// reciprocals. The longitude's sine and cosine are left to the pairs that
// need them (the ones farther than the series' reach).
struct LvA {
    double lon, lat;
    double sd, cd, st, ct;
    double a, b, inv_a, inv_b;
};

// (count: when the descriptions are by A row, only the rows with members
// hold one, and only those are read later)
__global__ void k_lvl_a64(const ACold* __restrict__ acold, int64_t n, const int32_t* count,
                          LvA* __restrict__ out) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (count && count[i] == 0)) return;
    const ACold C = acold[i];
    LvA L;
    L.lon = C.lon;
    L.lat = C.lat;
    sincospi(C.lat * (1.0 / 180.0), &L.sd, &L.cd);  // degrees reduced exactly
    sincos(C.theta, &L.st, &L.ct);
    L.a = C.a;
    L.b = C.b;
    L.inv_a = 1.0 / C.a;
    L.inv_b = 1.0 / C.b;
    out[i] = L;
}

// sin x and 1 - cos x for |x| <= 0.01 rad by their Taylor series (the first
// omitted terms are below 1e-21 of the result).
__device__ __forceinline__ void sin_vers_small(double x, double* s, double* v) {
    const double x2 = x * x;
    *s = x * (1.0 - x2 * (1.0 / 6.0) * (1.0 - x2 * (1.0 / 20.0) * (1.0 - x2 * (1.0 / 42.0))));
    *v = x2 * 0.5 * (1.0 - x2 * (1.0 / 12.0) * (1.0 - x2 * (1.0 / 30.0) * (1.0 - x2 * (1.0 / 56.0))));
}

// The normalised distance of B from its east/north components (x, y) in A's
// frame, B in A's hemisphere and s2 = x^2 + y^2 < 1e-4 (separation below
// ~0.57 deg): the quantity norm64 computes, with rho / sin(rho) from its
// series, one square root and the semi-axes' reciprocals.
__device__ __forceinline__ double norm_small(const LvA& L, int shape, double x, double y,
                                             double s2) {
    if (L.a == 0.0 || L.b == 0.0) return INFINITY;
    const double k = rho_over_s(s2);
    if (shape == XM_CIRCLE) return k * sqrt(s2) * L.inv_a;
    const double X = x * L.st + y * L.ct;
    const double Y = x * L.ct - y * L.st;
    if (shape == XM_ELLIPSE) {
        const double u = X * L.inv_a, v = Y * L.inv_b;
        return k * sqrt(u * u + v * v);
    }
    return k * fmax(fabs(X) * L.inv_a, fabs(Y) * L.inv_b);
}

__global__ void k_lvl_pair(IndexGeom G, const LvA* __restrict__ a64,
                           const int32_t* __restrict__ a_slot, int shape,
                           const int64_t* __restrict__ pa, const int64_t* __restrict__ pb,
                           int64_t n, Scales S, double* __restrict__ dist,
                           int32_t* __restrict__ level, int32_t* __restrict__ within,
                           unsigned long long* __restrict__ mind) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t a = pa[p];
    const LvA& L = a64[a_slot ? a_slot[a] : a];
    const int32_t row = (int32_t)pb[p];
    double d = 0.0;
    bool near = false;
    // B within half a degree of A in both coordinates: its east and north
    // components in A's frame follow exactly from the differences of the
    // positions (rotation by the latitude difference, then by the longitude
    // difference), whose sines the series give without a trigonometric call
    const double2 q = G.pos[row];
    double dlon = q.x - L.lon;
    if (dlon > 180.0) dlon -= 360.0;
    else if (dlon < -180.0) dlon += 360.0;
    const double dlat = q.y - L.lat;
    if (fabs(dlon) <= 0.5 && fabs(dlat) <= 0.5) {  // separation below 0.71 deg: z > 0
        double sa, va, sd, vd;
        sin_vers_small(dlon * kDeg, &sa, &va);
        sin_vers_small(dlat * kDeg, &sd, &vd);
        const double cb = L.cd * (1.0 - vd) - L.sd * sd;  // cos(lat_B)
        const double x = cb * sa;
        const double y = sd + cb * L.sd * va;  // sin(dlat) + cos(lat_B) sin(lat_A) (1 - cos dlon)
        const double s2 = x * x + y * y;
        if (s2 < 1e-4) {
            d = norm_small(L, shape, x, y, s2);
            near = true;
        }
    }
    if (!near) {  // from B's unit vector and A's full basis
        A64 A;
        sincospi(L.lon * (1.0 / 180.0), &A.sa, &A.ca);
        A.sd = L.sd;
        A.cd = L.cd;
        A.st = L.st;
        A.ct = L.ct;
        A.a = L.a;
        A.b = L.b;
        double px, py, pz;
        if (G.px) {
            px = G.px[row];
            py = G.py[row];
            pz = G.pz[row];
        } else {
            double sl, cl, sb, cb;
            sincospi(q.x * (1.0 / 180.0), &sl, &cl);
            sincospi(q.y * (1.0 / 180.0), &sb, &cb);
            px = cb * cl;
            py = cb * sl;
            pz = sb;
        }
        d = norm64(A, shape, px, py, pz);
    }
    dist[p] = d;
    atomicMin(&mind[a], (unsigned long long)dbits(d));  // d >= 0: bit order is value order
    if (S.k > 0) {
        int32_t k = 0;  // copies that do not hold the pair
        while (k < S.k && !(d <= S.s[k])) k++;
        level[p] = k;
        if (k < S.k) atomicAdd(&within[a * S.k + k], 1);
    }
}

__global__ void k_lvl_best(const int64_t* __restrict__ pa, const int64_t* __restrict__ pb,
                           int64_t n, const double* __restrict__ dist,
                           const unsigned long long* __restrict__ mind,
                           unsigned long long* __restrict__ best) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t a = pa[p];
    if (dbits(dist[p]) == (uint64_t)mind[a]) atomicMin(&best[a], (unsigned long long)pb[p]);
}

__global__ void k_lvl_finish(int64_t n_a, int32_t k, const unsigned long long* __restrict__ mind,
                             const unsigned long long* __restrict__ best,
                             int32_t* __restrict__ within, int64_t* __restrict__ best_b,
                             double* __restrict__ best_dist) {
    pdl_wait();
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n_a) return;
    const bool has = best[a] != ~0ull;
    best_b[a] = has ? (int64_t)best[a] : -1;
    best_dist[a] = has ? __longlong_as_double((long long)mind[a]) : (double)NAN;
    int32_t run = 0;
    for (int32_t j = 0; j < k; j++) {
        run += within[a * k + j];
        within[a * k + j] = run;
    }
}

unsigned grid_of(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace
}  // namespace xm

using namespace xm;

extern "C" xm_status xm_levels_compute(const xm_index* X, const xm_result* R, const double* scales,
                                       int32_t n_scales, void* stream, xm_levels** out) {
    if (!out) return set_error(XM_EINVAL, "xm_levels_compute: out is NULL");
    *out = nullptr;
    if (!X || !R) return set_error(XM_EINVAL, "xm_levels_compute: NULL argument");
    if (n_scales < 0 || n_scales > kMaxScales)
        return set_error(XM_EINVAL, "xm_levels_compute: %d scales (0..%d)", n_scales, kMaxScales);
    if (n_scales > 0 && !scales) return set_error(XM_EINVAL, "xm_levels_compute: scales is NULL");
    Scales S{};
    S.k = n_scales;
    for (int32_t j = 0; j < n_scales; j++) {
        const double v = scales[j];
        if (!(v > 0.0 && v <= 1.0) || (j > 0 && !(v > scales[j - 1])))
            return set_error(XM_EINVAL, "xm_levels_compute: scales must increase within (0, 1]");
        S.s[j] = v;
    }
    if (!(R->selection & XM_SEL_ALL))
        return set_error(XM_EINVAL, "xm_levels_compute: the result holds no ALL selection");
    if (!R->acold)
        return set_error(XM_EUNSUPPORTED, "xm_levels_compute: the result holds no positions "
                                          "(batch view or exact-value match)");
    if (R->n_b != X->n) return set_error(XM_EINVAL, "xm_levels_compute: the result is of another index");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = R->n_pairs, nA = R->n_a;
    xm_levels* L = new (std::nothrow) xm_levels();
    if (!L) return set_error(XM_ENOMEM, "xm_levels_compute: host allocation");
    L->n_pairs = n;
    L->n_a = nA;
    L->n_scales = n_scales;
    L->stream = s;
    const int64_t n1 = n > 0 ? n : 1, a1 = nA > 0 ? nA : 1;
    const int64_t nw = n_scales > 0 ? nA * n_scales : 0;
    // dist, best_dist (f64), best_b (i64), level (i32, padded to 8 B), n_within (i32)
    const size_t lvl_bytes = n_scales > 0 ? ((size_t)n1 * sizeof(int32_t) + 7) / 8 * 8 : 0;
    const size_t bytes = (size_t)n1 * sizeof(double) + (size_t)a1 * (sizeof(double) + sizeof(int64_t)) +
                         lvl_bytes + (size_t)(nw > 0 ? nw : 0) * sizeof(int32_t);
    unsigned char* base = (unsigned char*)dev_alloc(bytes, s);
    LvA* a64 = (LvA*)dev_alloc((size_t)a1 * sizeof(LvA), s);
    unsigned long long* w = (unsigned long long*)dev_alloc(2 * (size_t)a1 * sizeof(unsigned long long), s);
    auto body = [&]() -> xm_status {
        if (!base || !a64 || !w) return set_error(XM_ENOMEM, "xm_levels_compute: %lld pairs", (long long)n);
        L->dist = (double*)base;
        L->best_dist = L->dist + n1;
        L->best_b = (int64_t*)(L->best_dist + a1);
        unsigned char* tail = (unsigned char*)(L->best_b + a1);
        if (n_scales > 0) {
            L->level = (int32_t*)tail;
            L->n_within = (int32_t*)(tail + lvl_bytes);
        }
        unsigned long long *mind = w, *best = w + a1;
        cudaError_t e = cudaMemsetAsync(w, 0xFF, 2 * (size_t)a1 * sizeof(unsigned long long), s);
        if (e == cudaSuccess && nw > 0) e = cudaMemsetAsync(L->n_within, 0, nw * sizeof(int32_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_levels_compute: memset");
        if (nA > 0)  // A descriptions are stored by slot; the slots are a permutation of the rows
            XM_LAUNCH("k_lvl_a64", grid_of(nA), kBlock, 0, s, k_lvl_a64, R->acold, nA,
                      R->a_slot ? (const int32_t*)nullptr : R->count, a64);
        if (n > 0) {
            const IndexGeom G = X->geom();
            XM_LAUNCH("k_lvl_pair", grid_of(n), kBlock, 0, s, k_lvl_pair, G, a64, R->a_slot,
                      R->shape, R->a_row, R->b_row, n, S, L->dist, L->level, L->n_within, mind);
            XM_LAUNCH("k_lvl_best", grid_of(n), kBlock, 0, s, k_lvl_best, R->a_row, R->b_row, n,
                      L->dist, mind, best);
        }
        if (nA > 0)
            XM_LAUNCH("k_lvl_finish", grid_of(nA), kBlock, 0, s, k_lvl_finish, nA, n_scales, mind,
                      best, L->n_within, L->best_b, L->best_dist);
        return XM_OK;
    };
    const xm_status st = body();
    dev_free(a64, s);
    dev_free(w, s);
    if (st != XM_OK) {
        dev_free(base, s);
        delete L;
        return st;
    }
    *out = L;
    return XM_OK;
}

extern "C" xm_status xm_levels_free(xm_levels* L) {
    if (!L) return XM_OK;
    dev_free(L->dist, L->stream);
    delete L;
    return XM_OK;
}

extern "C" xm_status xm_levels_get(const xm_levels* L, xm_levels_view* v) {
    if (!L || !v) return set_error(XM_EINVAL, "xm_levels_get: NULL argument");
    v->n_pairs = L->n_pairs;
    v->n_a = L->n_a;
    v->n_scales = L->n_scales;
    v->dist = L->dist;
    v->best_b_row = L->best_b;
    v->best_dist = L->best_dist;
    v->level = L->level;
    v->n_within = L->n_within;
    return XM_OK;
}

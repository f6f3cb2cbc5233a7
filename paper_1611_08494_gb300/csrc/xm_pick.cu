// xm_pick.cu -- further readings of the paper's "best pairs" (§2.2) over the
// pair list of an "all" result: the best pair of every B source, and the
// pairs that are best for both their A and their B source.
//
//   k_pick_min    per pair: smallest reported separation of its B source
//   k_pick_cont   per pair within the float32 error band of that minimum:
//                 contender count and lowest contender of the B source
//   k_pick_exact  contenders of B sources with more than one: float64
//                 separation from the exact positions, its minimum per B
//   k_pick_first  the lowest pair (lowest A row) at that exact minimum
//   k_pick_flag   per pair: kept or not; prefix sum; k_pick_write the rows
//
// Reported separations of float32-path sources are within 9e-5 arcsec of
// the float64 value, so a B source whose two best candidates differ by more
// than twice that needs no float64 work; the others are decided in float64
// as the definition (and the oracle) does.
#include <math.h>

#include <new>

#include "xm_internal.cuh"

namespace xm {
namespace {

constexpr int kBlock = 256;
constexpr double kBandArcsec = 2.0 * 9e-5;  // twice the float32 separation bound

__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }

__global__ void k_pick_min(const int64_t* __restrict__ pb, const double* __restrict__ ps,
                           int64_t n, unsigned long long* __restrict__ minbits) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    atomicMin(&minbits[pb[p]], (unsigned long long)dbits(ps[p]));
}

__global__ void k_pick_cont(const int64_t* __restrict__ pb, const double* __restrict__ ps,
                            int64_t n, const unsigned long long* __restrict__ minbits,
                            int32_t* __restrict__ ncont, unsigned long long* __restrict__ first) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t b = pb[p];
    const double m = __longlong_as_double((long long)minbits[b]);
    if (ps[p] <= m + kBandArcsec + 1e-9 * m) {
        atomicAdd(&ncont[b], 1);
        atomicMin(&first[b], (unsigned long long)p);
    }
}

// Float64 separation (arcsec) of pair p from the exact positions.
__device__ __forceinline__ double sep64_of(const IndexGeom& G, const ACold* __restrict__ acold,
                                           const int32_t* __restrict__ a_slot, int64_t a,
                                           int64_t b) {
    const ACold& C = acold[a_slot ? a_slot[a] : a];
    const A64 A = make_a64(C);
    double px, py, pz, rho;
    const int32_t row = (int32_t)b;
    if (G.px) {
        px = G.px[row];
        py = G.py[row];
        pz = G.pz[row];
    } else {
        const double2 q = G.pos[row];
        unit64_deg(q.x, q.y, &px, &py, &pz);
    }
    test64(A, XM_CIRCLE, px, py, pz, &rho);
    return rho * kRadToArcsec;
}

__global__ void k_pick_exact(IndexGeom G, const ACold* __restrict__ acold,
                             const int32_t* __restrict__ a_slot, const int64_t* __restrict__ pa,
                             const int64_t* __restrict__ pb, const double* __restrict__ ps, int64_t n,
                             const unsigned long long* __restrict__ minbits,
                             const int32_t* __restrict__ ncont,
                             unsigned long long* __restrict__ min64) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t b = pb[p];
    if (ncont[b] < 2) return;
    const double m = __longlong_as_double((long long)minbits[b]);
    if (!(ps[p] <= m + kBandArcsec + 1e-9 * m)) return;
    atomicMin(&min64[b], (unsigned long long)dbits(sep64_of(G, acold, a_slot, pa[p], b)));
}

__global__ void k_pick_first(IndexGeom G, const ACold* __restrict__ acold,
                             const int32_t* __restrict__ a_slot, const int64_t* __restrict__ pa,
                             const int64_t* __restrict__ pb, const double* __restrict__ ps, int64_t n,
                             const unsigned long long* __restrict__ minbits,
                             const int32_t* __restrict__ ncont,
                             const unsigned long long* __restrict__ min64,
                             unsigned long long* __restrict__ first_exact) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t b = pb[p];
    if (ncont[b] < 2) return;
    const double m = __longlong_as_double((long long)minbits[b]);
    if (!(ps[p] <= m + kBandArcsec + 1e-9 * m)) return;
    // the same computation as k_pick_exact, so equal values compare equal
    if (dbits(sep64_of(G, acold, a_slot, pa[p], b)) == (uint64_t)min64[b])
        atomicMin(&first_exact[b], (unsigned long long)p);
}

__global__ void k_pick_flag(const int64_t* __restrict__ pa, const int64_t* __restrict__ pb,
                            int64_t n, const int32_t* __restrict__ ncont,
                            const unsigned long long* __restrict__ first,
                            const unsigned long long* __restrict__ first_exact,
                            const int64_t* __restrict__ best_b, int mutual,
                            int32_t* __restrict__ flag) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t b = pb[p];
    const unsigned long long w = ncont[b] > 1 ? first_exact[b] : first[b];
    bool keep = w == (unsigned long long)p;
    if (keep && mutual) keep = best_b[pa[p]] == b;
    flag[p] = keep ? 1 : 0;
}

__global__ void k_pick_write(const int64_t* __restrict__ pa, const int64_t* __restrict__ pb,
                             const double* __restrict__ ps, int64_t n,
                             const int32_t* __restrict__ flag, const int64_t* __restrict__ off,
                             int64_t* __restrict__ oa, int64_t* __restrict__ ob,
                             double* __restrict__ os) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !flag[p]) return;
    const int64_t o = off[p];
    oa[o] = pa[p];
    ob[o] = pb[p];
    os[o] = ps[p];
}

unsigned grid_of(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace
}  // namespace xm

using namespace xm;

extern "C" xm_status xm_pick_pairs(const xm_index* X, const xm_result* R, int32_t pick,
                                   void* stream, xm_rows** out) {
    if (!out) return set_error(XM_EINVAL, "xm_pick_pairs: out is NULL");
    *out = nullptr;
    if (!X || !R) return set_error(XM_EINVAL, "xm_pick_pairs: NULL argument");
    if (pick != XM_PICK_BEST_B && pick != XM_PICK_MUTUAL)
        return set_error(XM_EINVAL, "xm_pick_pairs: bad pick %d", pick);
    if (!(R->selection & XM_SEL_ALL))
        return set_error(XM_EINVAL, "xm_pick_pairs: the result holds no ALL selection");
    if (pick == XM_PICK_MUTUAL && !(R->selection & XM_SEL_BEST))
        return set_error(XM_EINVAL, "xm_pick_pairs: MUTUAL needs the BEST selection too");
    if (!R->acold)
        return set_error(XM_EUNSUPPORTED, "xm_pick_pairs: the result holds no positions (batch view "
                                          "or exact-value match)");
    if (R->n_b != X->n) return set_error(XM_EINVAL, "xm_pick_pairs: the result is of another index");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = R->n_pairs, nB = R->n_b;
    xm_rows* J = new (std::nothrow) xm_rows();
    if (!J) return set_error(XM_ENOMEM, "xm_pick_pairs: host allocation");
    J->stream = s;
    const int64_t nb1 = nB > 0 ? nB : 1, n1 = n > 0 ? n : 1;
    // per B: min reported sep, contenders, lowest contender, exact min, lowest exact
    unsigned long long* w = (unsigned long long*)dev_alloc(4 * nb1 * sizeof(unsigned long long), s);
    int32_t* ncont = (int32_t*)dev_alloc(nb1 * sizeof(int32_t), s);
    int32_t* flag = (int32_t*)dev_alloc(n1 * sizeof(int32_t), s);
    int64_t* off = (int64_t*)dev_alloc((n1 + 1) * sizeof(int64_t), s);  // [n]: total
    int32_t* err = (int32_t*)dev_alloc(sizeof(int32_t), s);
    auto body = [&]() -> xm_status {
        if (!w || !ncont || !flag || !off || !err) return set_error(XM_ENOMEM, "xm_pick_pairs: work");
        unsigned long long *minbits = w, *first = w + nb1, *min64 = w + 2 * nb1,
                           *first_exact = w + 3 * nb1;
        cudaError_t e = cudaMemsetAsync(w, 0xFF, 4 * nb1 * sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ncont, 0, nb1 * sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_pick_pairs: memset");
        const IndexGeom G = X->geom();
        if (n > 0) {
            XM_LAUNCH("k_pick_min", grid_of(n), kBlock, 0, s, k_pick_min, R->b_row, R->sep, n, minbits);
            XM_LAUNCH("k_pick_cont", grid_of(n), kBlock, 0, s, k_pick_cont, R->b_row, R->sep, n,
                      minbits, ncont, first);
            XM_LAUNCH("k_pick_exact", grid_of(n), kBlock, 0, s, k_pick_exact, G, R->acold, R->a_slot,
                      R->a_row, R->b_row, R->sep, n, minbits, ncont, min64);
            XM_LAUNCH("k_pick_first", grid_of(n), kBlock, 0, s, k_pick_first, G, R->acold,
                      R->a_slot, R->a_row, R->b_row, R->sep, n, minbits, ncont, min64, first_exact);
            XM_LAUNCH("k_pick_flag", grid_of(n), kBlock, 0, s, k_pick_flag, R->a_row, R->b_row, n,
                      ncont, first, first_exact, R->best_b, pick == XM_PICK_MUTUAL ? 1 : 0, flag);
        }
        xm_status st = exclusive_scan_i32(flag, off, n, off + n1, err, s);
        if (st != XM_OK) return st;
        int64_t total = 0;
        int32_t h_err = 0;
        HostReads rd(s);
        e = rd.add(&total, off + n1, sizeof(int64_t));
        if (e == cudaSuccess) e = rd.add(&h_err, err, sizeof(int32_t));
        if (e == cudaSuccess) e = rd.sync();
        if (e != cudaSuccess) return cuda_fail(e, "xm_pick_pairs sync");
        if (h_err & kErrTimeout) return set_error(XM_ETIMEOUT, "xm_pick_pairs: scan look-back timed out");
        J->n = total;
        const int64_t nr = total > 0 ? total : 1;
        J->a_row = (int64_t*)dev_alloc(nr * (2 * sizeof(int64_t) + sizeof(double)), s);
        if (!J->a_row) return set_error(XM_ENOMEM, "xm_pick_pairs: %lld rows", (long long)total);
        J->b_row = J->a_row + nr;
        J->sep = (double*)(J->b_row + nr);
        if (n > 0)
            XM_LAUNCH("k_pick_write", grid_of(n), kBlock, 0, s, k_pick_write, R->a_row, R->b_row,
                      R->sep, n, flag, off, J->a_row, J->b_row, J->sep);
        return XM_OK;
    };
    const xm_status st = body();
    dev_free(w, s);
    dev_free(ncont, s);
    dev_free(flag, s);
    dev_free(off, s);
    dev_free(err, s);
    if (st != XM_OK) {
        xm_rows_free(J);
        return st;
    }
    *out = J;
    return XM_OK;
}

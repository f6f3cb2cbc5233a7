// xm_values.cu -- the Exact Value functional case (paper §2.1): A_i and B_j
// match when their key columns hold the same value. The result has the
// layout of a positional match (pairs in ascending A row then B row, member
// counts, the best pair = the lowest B row), so the joins of §2.2 apply
// unchanged.
//
//   k_val_key     keys to order-preserving unsigned codes (int64: sign bit
//                 flipped; float64: IEEE total order with -0 folded into +0;
//                 NaN -> all ones, above every number, never looked up), row
//                 payloads, and the AND / OR of all B codes (bits that never
//                 differ need no sort pass)
//   radix sort    stable, so equal keys keep ascending B rows (xm_sort.cu):
//                 on the codes themselves when they differ in at most 32
//                 bits, else on a 32-bit hash of them (half the passes;
//                 equal keys still form one run, now shared with the few
//                 keys whose hash collides, told apart by the codes)
//   k_val_lut     a bucket table over the sorted codes (one bucket per two
//                 to four keys; long runs of entries by k_val_runs)
//   k_val_probe   per A: the run of equal B codes, searched inside one
//                 bucket; count, best B row, first sorted position
//   prefix sum    pair offsets
//   k_val_emit    the pairs of each A row
#include <math.h>

#include <new>

#include "xm_internal.cuh"

namespace xm {
namespace {

constexpr int kBlock = 256;
constexpr uint64_t kNaNCode = ~0ull;

__device__ __forceinline__ uint64_t key_code(const void* keys, int64_t i, int32_t type) {
    if (type == XM_KEY_INT64) return (uint64_t)((const int64_t*)keys)[i] ^ 0x8000000000000000ull;
    double v = ((const double*)keys)[i];
    uint64_t u = (uint64_t)__double_as_longlong(v);
    if ((u & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) return kNaNCode;  // NaN
    if ((u << 1) == 0) u = 0;  // -0 is +0
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// 32-bit hash of a code (the finaliser of the SplitMix64 generator, Steele,
// Lea & Flood 2014, high half): equal codes hash equally, distinct ones
// collide with probability about 2^-32.
__device__ __forceinline__ uint64_t code_hash(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x >> 32;
}

// Grid-stride over B (a few blocks per SM), so the AND / OR of all codes
// costs one pair of atomics per block. Writes the codes by row and, for the
// hashed order, their hashes.
__global__ void k_val_key(const void* __restrict__ keys, int64_t n, int32_t type,
                          uint64_t* __restrict__ codes, uint64_t* __restrict__ hashes,
                          uint32_t* __restrict__ rows, unsigned long long* __restrict__ and_or) {
    pdl_wait();
    __shared__ unsigned long long s_and, s_or;
    if (threadIdx.x == 0) {
        s_and = ~0ull;
        s_or = 0ull;
    }
    __syncthreads();
    uint64_t c_and = ~0ull, c_or = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t c = key_code(keys, i, type);
        codes[i] = c;
        hashes[i] = code_hash(c);
        rows[i] = (uint32_t)i;
        c_and &= c;
        c_or |= c;
    }
    for (int s = 16; s > 0; s >>= 1) {
        c_and &= __shfl_xor_sync(0xffffffffu, c_and, s);
        c_or |= __shfl_xor_sync(0xffffffffu, c_or, s);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAnd(&s_and, (unsigned long long)c_and);
        atomicOr(&s_or, (unsigned long long)c_or);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAnd(&and_or[0], s_and);
        atomicOr(&and_or[1], s_or);
    }
}

// Bucket table over the sorted codes: the codes share every bit above
// end_bit; bucket(c) = low end_bit bits of c >> shift, and lut[k] is the
// first sorted position whose bucket reaches k (lut[nb] = n). Runs of
// entries longer than kRunInline go to a list filled by k_val_runs.
struct ValLut {
    uint64_t prefix, mask;  // common high bits, mask of the low end_bit bits
    uint32_t shift, nb;     // bucket shift, buckets
    uint32_t* lut;
};

struct ValRun {
    int64_t first;
    uint32_t count, value;
};

constexpr int64_t kRunInline = 32;

__device__ __forceinline__ uint32_t val_bucket(const ValLut& V, uint64_t c) {
    return (uint32_t)((c & V.mask) >> V.shift);
}

__global__ void k_val_lut(const uint64_t* __restrict__ sorted, int64_t n, ValLut V,
                          ValRun* __restrict__ runs, unsigned long long* __restrict__ n_runs,
                          long long run_cap, int32_t* err) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = val_bucket(V, sorted[i]);
    const int64_t pb = i == 0 ? -1 : (int64_t)val_bucket(V, sorted[i - 1]);
    auto run = [&](int64_t first, int64_t count, uint32_t value) {
        if (count <= 0) return;
        if (count <= kRunInline) {
            for (int64_t k = 0; k < count; k++) V.lut[first + k] = value;
        } else {
            const unsigned long long g = atomicAdd(n_runs, 1ull);
            if ((long long)g < run_cap) runs[g] = ValRun{first, (uint32_t)count, value};
            else atomicOr(err, kErrOverflow);
        }
    };
    run(pb + 1, b - pb, (uint32_t)i);
    if (i == n - 1) run(b + 1, (int64_t)V.nb - b, (uint32_t)n);
}

__global__ void k_val_runs(const ValRun* __restrict__ runs, const unsigned long long* n_runs,
                           long long run_cap, uint32_t* __restrict__ lut) {
    pdl_wait();
    const long long nr = min((long long)*n_runs, run_cap);
    for (long long r = blockIdx.x; r < nr; r += gridDim.x) {
        const ValRun R = runs[r];
        for (uint32_t k = threadIdx.x; k < R.count; k += blockDim.x) lut[R.first + k] = R.value;
    }
}

// First position in sorted[lo, hi) whose code is >= c (or > c when upper).
__device__ __forceinline__ int64_t bound(const uint64_t* __restrict__ sorted, int64_t lo, int64_t hi,
                                         uint64_t c, bool upper) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        const uint64_t v = __ldg(&sorted[mid]);
        if (upper ? v <= c : v < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_val_probe(const void* __restrict__ a_keys, int64_t n_a, int32_t type,
                            const uint64_t* __restrict__ sorted, const uint32_t* __restrict__ rows,
                            int64_t n_b, ValLut V, int32_t* __restrict__ count,
                            int64_t* __restrict__ first, int64_t* __restrict__ best_b,
                            double* __restrict__ best_sep) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_a) return;
    const uint64_t c = key_code(a_keys, i, type);
    int64_t lo = 0, hi = 0;
    // (NaN never matches; the int64 maximum has the same code and does)
    if (n_b > 0 && !(type == XM_KEY_FLOAT64 && c == kNaNCode) && (c & ~V.mask) == V.prefix) {
        const uint32_t b = val_bucket(V, c);
        const int64_t b0 = __ldg(&V.lut[b]), b1 = __ldg(&V.lut[b + 1]);
        lo = bound(sorted, b0, b1, c, false);
        hi = lo < b1 && __ldg(&sorted[lo]) == c ? bound(sorted, lo, b1, c, true) : lo;
    }
    const int64_t m = hi - lo;
    count[i] = (int32_t)(m < 2147483647 ? m : 2147483647);
    first[i] = lo;
    if (best_b) {
        best_b[i] = m > 0 ? (int64_t)rows[lo] : -1;
        best_sep[i] = m > 0 ? 0.0 : NAN;
    }
}

// Hashed order: the run of A's hash, then the B rows whose code is A's.
__global__ void k_val_probe_hashed(const void* __restrict__ a_keys, int64_t n_a, int32_t type,
                                   const uint64_t* __restrict__ sorted,
                                   const uint32_t* __restrict__ rows,
                                   const uint64_t* __restrict__ codes, int64_t n_b, ValLut V,
                                   int32_t* __restrict__ count, int64_t* __restrict__ first,
                                   int64_t* __restrict__ best_b, double* __restrict__ best_sep) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_a) return;
    const uint64_t c = key_code(a_keys, i, type);
    int64_t lo = 0, m = 0, best = -1;
    if (n_b > 0 && !(type == XM_KEY_FLOAT64 && c == kNaNCode)) {
        const uint64_t h = code_hash(c);
        const uint32_t b = val_bucket(V, h);
        const int64_t b0 = __ldg(&V.lut[b]), b1 = __ldg(&V.lut[b + 1]);
        lo = bound(sorted, b0, b1, h, false);
        for (int64_t p = lo; p < b1 && __ldg(&sorted[p]) == h; p++) {
            const uint32_t r = __ldg(&rows[p]);
            if (__ldg(&codes[r]) == c) {
                if (m == 0) best = r;
                m++;
            }
        }
    }
    count[i] = (int32_t)(m < 2147483647 ? m : 2147483647);
    first[i] = lo;
    if (best_b) {
        best_b[i] = best;
        best_sep[i] = m > 0 ? 0.0 : NAN;
    }
}

__global__ void k_val_emit_hashed(const void* __restrict__ a_keys, int32_t type,
                                  const int32_t* __restrict__ count,
                                  const int64_t* __restrict__ first,
                                  const int64_t* __restrict__ pair_off,
                                  const uint32_t* __restrict__ rows,
                                  const uint64_t* __restrict__ codes, int64_t n_a,
                                  int64_t* __restrict__ pa, int64_t* __restrict__ pb,
                                  double* __restrict__ ps) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_a) return;
    const int32_t c = count[i];
    if (c == 0) return;
    const uint64_t code = key_code(a_keys, i, type);
    const int64_t o = pair_off[i];
    int32_t k = 0;
    for (int64_t p = first[i]; k < c; p++) {  // (the run holds all c matches)
        const uint32_t r = rows[p];
        if (codes[r] != code) continue;
        pa[o + k] = i;
        pb[o + k] = r;
        ps[o + k] = 0.0;
        k++;
    }
}

__global__ void k_val_emit(const int32_t* __restrict__ count, const int64_t* __restrict__ first,
                           const int64_t* __restrict__ pair_off, const uint32_t* __restrict__ rows,
                           int64_t n_a, int64_t* __restrict__ pa, int64_t* __restrict__ pb,
                           double* __restrict__ ps) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_a) return;
    const int32_t c = count[i];
    const int64_t o = pair_off[i], f = first[i];
    for (int32_t k = 0; k < c; k++) {
        pa[o + k] = i;
        pb[o + k] = rows[f + k];
        ps[o + k] = 0.0;
    }
}

unsigned grid_of(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

int top_bit(uint64_t x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

}  // namespace
}  // namespace xm

using namespace xm;

extern "C" xm_status xm_match_values(const void* a_keys, int64_t n_a, const void* b_keys,
                                     int64_t n_b, int32_t key_type, int32_t on_device,
                                     int32_t selection, void* stream, xm_result** out) {
    if (!out) return set_error(XM_EINVAL, "xm_match_values: out is NULL");
    *out = nullptr;
    if (n_a < 0 || n_b < 0 || n_a > 2147483647LL || n_b > 2147483647LL ||
        (n_a > 0 && !a_keys) || (n_b > 0 && !b_keys))
        return set_error(XM_EINVAL, "xm_match_values: bad key columns");
    if (key_type != XM_KEY_INT64 && key_type != XM_KEY_FLOAT64)
        return set_error(XM_EINVAL, "xm_match_values: bad key type %d", key_type);
    if (selection < 1 || selection > 3)
        return set_error(XM_EINVAL, "xm_match_values: bad selection %d", selection);
    cudaStream_t s = (cudaStream_t)stream;
    xm_result* R = new (std::nothrow) xm_result();
    if (!R) return set_error(XM_ENOMEM, "xm_match_values: host allocation");
    R->stream = (cudaStream_t)stream;
    cudaGetDevice(&R->device);
    R->selection = selection;
    R->precision = XM_PREC_FP64;
    R->shape = -1;
    R->n_a = n_a;
    R->n_b = n_b;
    const int64_t na1 = n_a > 0 ? n_a : 1, nb1 = n_b > 0 ? n_b : 1;
    const bool want_best = (selection & XM_SEL_BEST) != 0;
    R->count = (int32_t*)dev_alloc(na1 * sizeof(int32_t), s);
    R->pair_off = (int64_t*)dev_alloc(na1 * sizeof(int64_t), s);
    if (want_best) {
        R->best_b = (int64_t*)dev_alloc(na1 * (sizeof(int64_t) + sizeof(double)), s);
        R->best_sep = R->best_b ? (double*)(R->best_b + na1) : nullptr;
    }
    // temporaries: host key copies, codes and rows (and sort scratch), first
    // positions, totals and the error word
    void* d_a = nullptr;
    void* d_b = nullptr;
    uint64_t* codes = (uint64_t*)dev_alloc(2 * nb1 * sizeof(uint64_t), s);
    uint64_t* hashes = (uint64_t*)dev_alloc(2 * nb1 * sizeof(uint64_t), s);
    uint32_t* rows = (uint32_t*)dev_alloc(2 * nb1 * sizeof(uint32_t), s);
    int64_t* first = (int64_t*)dev_alloc(na1 * sizeof(int64_t), s);
    unsigned long long* small = (unsigned long long*)dev_alloc(4 * sizeof(unsigned long long), s);
    uint32_t* lut = nullptr;
    ValRun* runs = nullptr;
    auto body = [&]() -> xm_status {
        if (!R->count || !R->pair_off || (want_best && !R->best_b) || !codes || !hashes || !rows ||
            !first || !small)
            return set_error(XM_ENOMEM, "xm_match_values: work buffers");
        cudaError_t e;
        const void* ak = a_keys;
        const void* bk = b_keys;
        if (!on_device) {
            d_a = dev_alloc(na1 * 8, s);
            d_b = dev_alloc(nb1 * 8, s);
            if (!d_a || !d_b) return set_error(XM_ENOMEM, "xm_match_values: key copies");
            e = n_a ? cudaMemcpyAsync(d_a, a_keys, n_a * 8, cudaMemcpyHostToDevice, s) : cudaSuccess;
            if (e == cudaSuccess && n_b)
                e = cudaMemcpyAsync(d_b, b_keys, n_b * 8, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "xm_match_values: key copies");
            ak = d_a;
            bk = d_b;
        }
        // small: [0] AND of codes, [1] OR, [2] pair total, [3] error bits
        const unsigned long long init[4] = {~0ull, 0ull, 0ull, 0ull};
        e = cudaMemcpyAsync(small, init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_match_values: init");
        int32_t* err = (int32_t*)(small + 3);
        if (n_b > 0) {
            const unsigned gk = grid_of(n_b) < 8 * 152 ? grid_of(n_b) : 8 * 152;
            XM_LAUNCH("k_val_key", gk, kBlock, 0, s, k_val_key, bk, n_b, key_type, codes, hashes,
                      rows, small);
        }
        unsigned long long h_ao[2] = {~0ull, 0ull};
        e = cudaMemcpyAsync(h_ao, small, sizeof(h_ao), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_match_values sync");
        // bits where the codes differ: the sort covers only those, or the
        // 32 bits of the hash when there are more
        const int code_bits = top_bit(h_ao[0] ^ h_ao[1]);
        const bool hashed = code_bits > 32;
        const int end_bit = hashed ? 32 : code_bits;
        uint64_t* sorted = hashed ? hashes : codes;
        if (n_b > 1 && end_bit > 0) {
            xm_status r = radix_sort_u64(sorted, rows, sorted + nb1, rows + nb1, n_b, 0, end_bit, err, s);
            if (r != XM_OK) return r;
        }
        // bucket table: about one bucket per 2-4 keys over the differing bits
        ValLut V{};
        V.mask = end_bit >= 64 ? ~0ull : ((1ull << end_bit) - 1);
        V.prefix = hashed ? 0ull : (h_ao[0] & ~V.mask);
        int lg = top_bit((uint64_t)nb1) - 2;
        lg = lg < 1 ? 1 : (lg > 28 ? 28 : lg);
        if (lg > end_bit) lg = end_bit > 0 ? end_bit : 0;
        V.shift = (uint32_t)(end_bit - lg);
        V.nb = 1u << lg;
        lut = (uint32_t*)dev_alloc(((size_t)V.nb + 1) * sizeof(uint32_t), s);
        const long long run_cap = (long long)(V.nb + 1) / (kRunInline + 1) + 16;
        runs = (ValRun*)dev_alloc(run_cap * sizeof(ValRun) + 16, s);
        if (!lut || !runs) return set_error(XM_ENOMEM, "xm_match_values: bucket table");
        V.lut = lut;
        unsigned long long* n_runs = (unsigned long long*)(runs + run_cap);
        e = cudaMemsetAsync(n_runs, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_match_values: memset");
        if (n_b > 0) {
            XM_LAUNCH("k_val_lut", grid_of(n_b), kBlock, 0, s, k_val_lut, sorted, n_b, V, runs,
                      n_runs, run_cap, err);
            XM_LAUNCH("k_val_runs", 4 * 152, kBlock, 0, s, k_val_runs, runs, n_runs, run_cap, lut);
        }
        if (n_a > 0 && hashed)
            XM_LAUNCH("k_val_probe", grid_of(n_a), kBlock, 0, s, k_val_probe_hashed, ak, n_a,
                      key_type, sorted, rows, codes, n_b, V, R->count, first, R->best_b,
                      R->best_sep);
        else if (n_a > 0)
            XM_LAUNCH("k_val_probe", grid_of(n_a), kBlock, 0, s, k_val_probe, ak, n_a, key_type,
                      codes, rows, n_b, V, R->count, first, R->best_b, R->best_sep);
        xm_status r = exclusive_scan_i32(R->count, R->pair_off, n_a, (int64_t*)(small + 2), err, s);
        if (r != XM_OK) return r;
        unsigned long long h[2] = {0, 0};
        e = cudaMemcpyAsync(h, small + 2, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "xm_match_values sync");
        if ((int32_t)h[1] & kErrTimeout) return set_error(XM_ETIMEOUT, "xm_match_values: look-back timed out");
        if ((int32_t)h[1] & kErrOverflow) return set_error(XM_ECUDA, "xm_match_values: run list overflow");
        R->n_pairs = (selection & XM_SEL_ALL) ? (int64_t)h[0] : 0;
        if (selection & XM_SEL_ALL) {
            const int64_t np = R->n_pairs > 0 ? R->n_pairs : 1;
            R->a_row = (int64_t*)dev_alloc(np * (2 * sizeof(int64_t) + sizeof(double)), s);
            if (!R->a_row) return set_error(XM_ENOMEM, "xm_match_values: %lld pairs", (long long)R->n_pairs);
            R->b_row = R->a_row + np;
            R->sep = (double*)(R->b_row + np);
            if (n_a > 0 && hashed)
                XM_LAUNCH("k_val_emit", grid_of(n_a), kBlock, 0, s, k_val_emit_hashed, ak, key_type,
                          R->count, first, R->pair_off, rows, codes, n_a, R->a_row, R->b_row,
                          R->sep);
            else if (n_a > 0)
                XM_LAUNCH("k_val_emit", grid_of(n_a), kBlock, 0, s, k_val_emit, R->count, first,
                          R->pair_off, rows, n_a, R->a_row, R->b_row, R->sep);
        }
        return XM_OK;
    };
    const xm_status st = body();
    dev_free(d_a, s);
    dev_free(d_b, s);
    dev_free(codes, s);
    dev_free(hashes, s);
    dev_free(rows, s);
    dev_free(first, s);
    dev_free(small, s);
    dev_free(lut, s);
    dev_free(runs, s);
    if (st != XM_OK) {
        xm_result_free(R);
        return st;
    }
    *out = R;
    return XM_OK;
}

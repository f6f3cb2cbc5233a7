// xm_join.cu -- the join types of paper §2.2 over a selected pair set.
//
// i) 1 and 2: the selected pairs; ii) 1 or 2: pairs, unmatched A rows and
// unmatched B rows; iii) all from 1 (2): pairs plus unmatched A (B) rows;
// iv) 1 not 2 (2 not 1): unmatched A (B) rows; v) 1 xor 2: unmatched A and
// unmatched B rows. A source is matched when it appears in the selected
// pairs. Row order: rows carrying an A source in ascending (a_row, b_row),
// then unmatched B rows in ascending b_row.
//
// Device steps: a bitset of matched B rows (idempotent atomicOr, so the
// result is deterministic), rows per A source and their prefix sum, unmatched
// B counts per 32-row word and their prefix sum, then two writers.
#include <math.h>

#include <mutex>
#include <new>

#include "xm_internal.cuh"

namespace xm {
namespace {

constexpr int kBlock = 256;

unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Grid of a grid-stride kernel: enough blocks to fill the GPU, no more.
unsigned grid_cap(int64_t n) {
    const unsigned g = grid_for(n);
    return g < 8u * 152u ? g : 8u * 152u;
}

__global__ void k_mark_b(const int64_t* __restrict__ b_row, int64_t n, uint32_t* __restrict__ bits) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t b = b_row[i];
    if (b >= 0) atomicOr(&bits[b >> 5], 1u << (b & 31));
}

// Rows each A source contributes, and the number of unmatched A sources.
// (grid-stride; the unmatched A sources are summed per block, so the one
// counter takes an atomic per block, not per warp)
__global__ void k_rows_a(const int32_t* __restrict__ count, int64_t nA, int sel_all,
                         int with_pairs, int with_un_a, int32_t* __restrict__ rows,
                         unsigned long long* __restrict__ n_un_a) {
    pdl_wait();
    __shared__ unsigned long long block_un;
    if (threadIdx.x == 0) block_un = 0;
    __syncthreads();
    uint32_t un = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nA;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = count[i];
        const int32_t sel = sel_all ? c : (c > 0 ? 1 : 0);
        int32_t r = with_pairs ? sel : 0;
        if (sel == 0 && with_un_a) r = 1;
        rows[i] = r;
        un += c == 0;
    }
    un = __reduce_add_sync(0xffffffffu, un);
    if ((threadIdx.x & 31) == 0 && un) atomicAdd(&block_un, (unsigned long long)un);
    __syncthreads();
    if (threadIdx.x == 0 && block_un) atomicAdd(n_un_a, block_un);
}

__device__ __forceinline__ uint32_t word_valid(int64_t w, int64_t nB) {
    int64_t rem = nB - (w << 5);
    return rem >= 32 ? 0xFFFFFFFFu : ((1u << rem) - 1u);
}

__global__ void k_word_unmatched(const uint32_t* __restrict__ bits, int64_t nwords, int64_t nB,
                                 int32_t* __restrict__ wcount) {
    pdl_wait();
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    wcount[w] = __popc(~bits[w] & word_valid(w, nB));
}

// A-side join rows, one thread per A row. With pairs_apart the pair rows of
// the "all" selection are written by k_write_pairs instead.
__global__ void k_write_a(const int32_t* __restrict__ count, const int64_t* __restrict__ pair_off,
                          const int64_t* __restrict__ pb, const double* __restrict__ ps,
                          const int64_t* __restrict__ best_b, const double* __restrict__ best_s,
                          const int64_t* __restrict__ row_off, int64_t nA, int sel_all,
                          int with_pairs, int with_un_a, int pairs_apart, int64_t a_off,
                          int64_t* __restrict__ oa, int64_t* __restrict__ ob,
                          double* __restrict__ os) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nA) return;
    int32_t c = count[i];
    int64_t o = row_off[i];
    if (c > 0) {
        if (!with_pairs) return;
        if (sel_all) {
            if (pairs_apart) return;
            int64_t p = pair_off[i];
            for (int32_t k = 0; k < c; k++) {
                oa[o + k] = i + a_off;
                ob[o + k] = pb[p + k];
                os[o + k] = ps[p + k];
            }
        } else {
            oa[o] = i + a_off;
            ob[o] = best_b[i];
            os[o] = best_s[i];
        }
    } else if (with_un_a) {
        oa[o] = i + a_off;
        ob[o] = -1;
        os[o] = NAN;
    }
}

// The pair rows of the "all" selection, one thread per pair: pair p of A
// row a goes to row_off[a] + (p - pair_off[a]); reads and writes run in pair
// order (coalesced).
__global__ void k_write_pairs(const int64_t* __restrict__ pa, const int64_t* __restrict__ pb,
                              const double* __restrict__ ps, const int64_t* __restrict__ pair_off,
                              const int64_t* __restrict__ row_off, int64_t n_pairs, int64_t a_off,
                              int64_t* __restrict__ oa, int64_t* __restrict__ ob,
                              double* __restrict__ os) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int64_t a = pa[p];
    const int64_t o = row_off[a] + (p - pair_off[a]);
    oa[o] = a + a_off;
    ob[o] = pb[p];
    os[o] = ps[p];
}

// B-only rows after the A-side rows: base_ptr (device) holds their count.
__global__ void k_write_b(const uint32_t* __restrict__ bits, const int64_t* __restrict__ word_off,
                          int64_t nB, const int64_t* __restrict__ base_ptr, int64_t* __restrict__ oa,
                          int64_t* __restrict__ ob, double* __restrict__ os) {
    pdl_wait();
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nB) return;
    const int64_t base = *base_ptr;
    int64_t w = j >> 5;
    uint32_t un = ~bits[w] & word_valid(w, nB);
    uint32_t bit = 1u << (j & 31);
    if (!(un & bit)) return;
    int64_t o = base + word_off[w] + __popc(un & (bit - 1u));
    oa[o] = -1;
    ob[o] = j;
    os[o] = NAN;
}

}  // namespace
}  // namespace xm

namespace xm {

// ------------------------------------------------ join without allocation
//
// Some callers cannot allocate device memory at the moment they need a join:
// a serving process or a framework whose caching allocator has reserved the
// whole GPU (a cudaMalloc would fail or fragment its pool), or a
// latency-critical loop that must not enter the driver's allocator.
// xm_join_noalloc gives them the join with no allocation at all: the caller
// passes the output arrays, and the scratch lives in one file-scope device
// array sized for results of at most kNoAllocMaxA A rows and kNoAllocMaxB B
// rows. Every GPU that loads the library holds that array (about 16 MB)
// until the process exits.

namespace {

constexpr int64_t kNoAllocMaxA = 1 << 20;  // A rows
constexpr int64_t kNoAllocMaxB = 1 << 23;  // B rows
constexpr int64_t kNoAllocWords = kNoAllocMaxB / 32;

struct JoinScratch {
    uint32_t bits[kNoAllocWords];      // matched B rows
    int32_t rows[kNoAllocMaxA];        // rows per A source
    int64_t row_off[kNoAllocMaxA];
    int32_t wcount[kNoAllocWords];     // unmatched B rows per word
    int64_t word_off[kNoAllocWords];
    int64_t ws_a[2 * (kNoAllocMaxA / 4096)];     // scan workspace (rows)
    int64_t ws_b[2 * (kNoAllocWords / 4096)];    // scan workspace (words)
    int64_t small[4];                  // totals, unmatched A count
};

static __device__ __align__(256) JoinScratch g_join_scratch;

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is not a device address); *dev_out
// is the current device. Thread-safe.
xm_status join_scratch(JoinScratch** out, int* dev_out) {
    static std::mutex mu;
    static JoinScratch* addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(XM_EUNSUPPORTED, "device %d", dev);
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_join_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(join scratch)");
        addr[dev] = (JoinScratch*)p;
    }
    *out = addr[dev];
    *dev_out = dev;
    return XM_OK;
}

}  // namespace
}  // namespace xm

extern "C" xm_status xm_join_noalloc(const xm_result* R, int32_t selection, int32_t join_type,
                                     int64_t* a_row, int64_t* b_row, double* sep,
                                     int64_t capacity, int64_t* n_rows, void* stream) {
    using namespace xm;
    if (!n_rows) return set_error(XM_EINVAL, "xm_join_noalloc: n_rows is NULL");
    *n_rows = 0;
    if (!R) return set_error(XM_EINVAL, "xm_join_noalloc: NULL result");
    if (selection != XM_SEL_ALL && selection != XM_SEL_BEST)
        return set_error(XM_EINVAL, "xm_join_noalloc: selection must be ALL or BEST");
    if (!(R->selection & selection))
        return set_error(XM_EINVAL, "xm_join_noalloc: selection not computed by xm_match");
    if (join_type < XM_JOIN_AND || join_type > XM_JOIN_XOR)
        return set_error(XM_EINVAL, "xm_join_noalloc: bad join type %d", join_type);
    if (capacity < 0 || (capacity > 0 && (!a_row || !b_row || !sep)))
        return set_error(XM_EINVAL, "xm_join_noalloc: bad output arrays");
    const int64_t nA = R->n_a, nB = R->n_b;
    if (nA > kNoAllocMaxA || nB > kNoAllocMaxB)
        return set_error(XM_EOVERFLOW,
                         "xm_join_noalloc: the result has %lld A rows and %lld B rows; this entry "
                         "point takes at most %lld and %lld (use xm_join)",
                         (long long)nA, (long long)nB, (long long)kNoAllocMaxA,
                         (long long)kNoAllocMaxB);
    const bool with_pairs = join_type == XM_JOIN_AND || join_type == XM_JOIN_OR ||
                            join_type == XM_JOIN_ALL1 || join_type == XM_JOIN_ALL2;
    const bool with_un_a = join_type == XM_JOIN_OR || join_type == XM_JOIN_ALL1 ||
                           join_type == XM_JOIN_NOT1_2 || join_type == XM_JOIN_XOR;
    const bool with_un_b = join_type == XM_JOIN_OR || join_type == XM_JOIN_ALL2 ||
                           join_type == XM_JOIN_NOT2_1 || join_type == XM_JOIN_XOR;
    const int sel_all = selection == XM_SEL_ALL;
    const int64_t nwords = (nB + 31) / 32;
    cudaStream_t s = (cudaStream_t)stream;
    JoinScratch* S = nullptr;
    int dev = -1;
    xm_status st = join_scratch(&S, &dev);
    if (st != XM_OK) return st;
    // the scratch array is the current device's; the result's arrays live on
    // the device it was computed on
    if (dev != R->device)
        return set_error(XM_EINVAL, "xm_join_noalloc: the result belongs to device %d, current is %d",
                         R->device, dev);
    // the array keeps the previous call's contents: clear what starts at zero
    cudaError_t e = cudaMemsetAsync(S->bits, 0, (nwords > 0 ? nwords : 1) * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->small, 0, sizeof(S->small), s);
    if (e != cudaSuccess) return cuda_fail(e, "xm_join_noalloc memset");
    if (sel_all) {
        if (R->n_pairs > 0) k_mark_b<<<grid_for(R->n_pairs), kBlock, 0, s>>>(R->b_row, R->n_pairs, S->bits);
    } else if (nA > 0) {
        k_mark_b<<<grid_for(nA), kBlock, 0, s>>>(R->best_b, nA, S->bits);
    }
    if (nA > 0)
        k_rows_a<<<grid_cap(nA), kBlock, 0, s>>>(R->count, nA, sel_all, (int)with_pairs,
                                                 (int)with_un_a, S->rows,
                                                 (unsigned long long*)&S->small[2]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "xm_join_noalloc launch");
    st = exclusive_scan_i32_ws(S->rows, S->row_off, nA, &S->small[0], S->ws_a, s);
    if (st != XM_OK) return st;
    if (nwords > 0)
        k_word_unmatched<<<grid_for(nwords), kBlock, 0, s>>>(S->bits, nwords, nB, S->wcount);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "xm_join_noalloc launch");
    st = exclusive_scan_i32_ws(S->wcount, S->word_off, nwords, &S->small[1], S->ws_b, s);
    if (st != XM_OK) return st;
    int64_t h[4];
    e = cudaMemcpyAsync(h, S->small, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "xm_join_noalloc sync");
    const int64_t total_a = h[0], un_b = h[1];
    const int64_t n = total_a + (with_un_b ? un_b : 0);
    *n_rows = n;
    if (n > capacity)
        return set_error(XM_EOVERFLOW, "xm_join_noalloc: %lld rows do not fit the capacity %lld",
                         (long long)n, (long long)capacity);
    if (nA > 0)
        k_write_a<<<grid_for(nA), kBlock, 0, s>>>(R->count, R->pair_off, R->b_row, R->sep, R->best_b,
                                                 R->best_sep, S->row_off, nA, sel_all,
                                                 (int)with_pairs, (int)with_un_a, 0, (int64_t)0,
                                                 a_row, b_row, sep);
    if (with_un_b && nB > 0)
        k_write_b<<<grid_for(nB), kBlock, 0, s>>>(S->bits, S->word_off, nB, &S->small[0], a_row,
                                                 b_row, sep);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "xm_join_noalloc launch");
    return XM_OK;
}

using namespace xm;

// The rows' memory returns to the pool in the order of the stream they were
// written on, after whatever the caller queued there to read them.
static void free_rows(xm_rows* J) {
    if (!J) return;
    dev_free(J->a_row, J->stream);
    dev_free(J->pending, J->stream);
    delete J;
}

// Reads the counts of a join launched without synchronising (once).
static std::mutex g_rows_mu;

static xm_status resolve_rows(xm_rows* J) {
    std::lock_guard<std::mutex> g(g_rows_mu);
    if (!J->pending) return XM_OK;
    int64_t h[5];
    HostReads rd(J->stream);
    cudaError_t e = rd.add(h, J->pending, sizeof(h));
    if (e == cudaSuccess) e = rd.sync();
    if (e != cudaSuccess) return cuda_fail(e, "xm_rows_get sync");
    if ((int32_t)h[4] & kErrTimeout) return set_error(XM_ETIMEOUT, "xm_join: scan look-back timed out");
    J->n_unmatched_a = h[2];
    J->n_unmatched_b = h[1];
    J->n = h[0] + (J->with_un_b ? h[1] : 0);
    dev_free(J->pending, J->stream);
    J->pending = nullptr;
    return XM_OK;
}

// The rows of one join type over one selection of a result. ext_bits
// (nullable): the matched B rows of a catalogue 1 split over several results
// (the union of their selections), which then decides the unmatched B rows
// instead of this result's own pairs; a_off is added to every A row written;
// with_b: write the B-only rows (else only count them).
static xm_status join_impl(const xm_result* R, int32_t selection, int32_t join_type,
                           const uint32_t* ext_bits, int64_t a_off, bool with_b, void* stream,
                           xm_rows** out, const char* who) {
    if (!out) return set_error(XM_EINVAL, "%s: out is NULL", who);
    *out = nullptr;
    if (!R) return set_error(XM_EINVAL, "%s: NULL result", who);
    if (selection != XM_SEL_ALL && selection != XM_SEL_BEST)
        return set_error(XM_EINVAL, "%s: selection must be ALL or BEST", who);
    if (!(R->selection & selection))
        return set_error(XM_EINVAL, "%s: selection not computed by xm_match", who);
    if (join_type < XM_JOIN_AND || join_type > XM_JOIN_XOR)
        return set_error(XM_EINVAL, "%s: bad join type %d", who, join_type);
    if (a_off < 0) return set_error(XM_EINVAL, "%s: negative A row offset", who);
    const bool with_pairs = join_type == XM_JOIN_AND || join_type == XM_JOIN_OR ||
                            join_type == XM_JOIN_ALL1 || join_type == XM_JOIN_ALL2;
    const bool with_un_a = join_type == XM_JOIN_OR || join_type == XM_JOIN_ALL1 ||
                           join_type == XM_JOIN_NOT1_2 || join_type == XM_JOIN_XOR;
    const bool with_un_b = join_type == XM_JOIN_OR || join_type == XM_JOIN_ALL2 ||
                           join_type == XM_JOIN_NOT2_1 || join_type == XM_JOIN_XOR;
    const bool write_b = with_un_b && with_b;
    const int sel_all = selection == XM_SEL_ALL;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nA = R->n_a, nB = R->n_b;
    const int64_t nwords = (nB + 31) / 32;
    xm_rows* J = new (std::nothrow) xm_rows();
    if (!J) return set_error(XM_ENOMEM, "%s: host allocation", who);

    uint32_t* own_bits = ext_bits ? nullptr : (uint32_t*)dev_alloc((nwords > 0 ? nwords : 1) * sizeof(uint32_t), s);
    const uint32_t* bits = ext_bits ? ext_bits : own_bits;
    int32_t* rows = (int32_t*)dev_alloc((nA > 0 ? nA : 1) * sizeof(int32_t), s);
    int64_t* row_off = (int64_t*)dev_alloc((nA > 0 ? nA : 1) * sizeof(int64_t), s);
    int32_t* wcount = (int32_t*)dev_alloc((nwords > 0 ? nwords : 1) * sizeof(int32_t), s);
    int64_t* word_off = (int64_t*)dev_alloc((nwords > 0 ? nwords : 1) * sizeof(int64_t), s);
    // counts read later by xm_rows_get: [0] A-side rows, [1] unmatched B,
    // [2] unmatched A, [4] error bits
    int64_t* small = (int64_t*)dev_alloc(5 * sizeof(int64_t), s);
    J->pending = small;
    J->stream = s;
    J->with_un_b = write_b;
    auto body = [&]() -> xm_status {
        if (!bits || !rows || !row_off || !wcount || !word_off || !small)
            return set_error(XM_ENOMEM, "%s: work buffers", who);
        cudaError_t e = cudaMemsetAsync(small, 0, 5 * sizeof(int64_t), s);
        if (e == cudaSuccess && own_bits)
            e = cudaMemsetAsync(own_bits, 0, (nwords > 0 ? nwords : 1) * sizeof(uint32_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "memset");
        if (own_bits) {
            if (sel_all) {
                if (R->n_pairs > 0)
                    XM_LAUNCH("k_mark_b", grid_for(R->n_pairs), kBlock, 0, s, k_mark_b, R->b_row,
                              R->n_pairs, own_bits);
            } else if (nA > 0) {
                XM_LAUNCH("k_mark_b", grid_for(nA), kBlock, 0, s, k_mark_b, R->best_b, nA, own_bits);
            }
        }
        if (nA > 0)
            XM_LAUNCH("k_rows_a", grid_cap(nA), kBlock, 0, s, k_rows_a, R->count, nA, sel_all,
                      (int)with_pairs, (int)with_un_a, rows, (unsigned long long*)small + 2);
        int32_t* err = (int32_t*)(small + 4);
        xm_status r = exclusive_scan_i32(rows, row_off, nA, small + 0, err, s);
        if (r != XM_OK) return r;
        if (nwords > 0)
            XM_LAUNCH("k_word_unmatched", grid_for(nwords), kBlock, 0, s, k_word_unmatched, bits,
                      nwords, nB, wcount);
        r = exclusive_scan_i32(wcount, word_off, nwords, small + 1, err, s);
        if (r != XM_OK) return r;
        // rows are written at device-side offsets into room for the most
        // rows the join can have; the count is read by xm_rows_get
        const int64_t a_side = (with_pairs ? (sel_all ? R->n_pairs : nA) : 0) + (with_un_a ? nA : 0);
        const int64_t bound = a_side + (write_b ? nB : 0);
        int64_t nr = bound > 0 ? bound : 1;
        J->a_row = (int64_t*)dev_alloc(nr * (2 * sizeof(int64_t) + sizeof(double)), s);
        if (!J->a_row) return set_error(XM_ENOMEM, "%s: %lld rows", who, (long long)bound);
        J->b_row = J->a_row + nr;
        J->sep = (double*)(J->b_row + nr);
        const int pairs_apart = sel_all && with_pairs && R->n_pairs > 0 && R->a_row;
        if (pairs_apart)
            XM_LAUNCH("k_write_pairs", grid_for(R->n_pairs), kBlock, 0, s, k_write_pairs, R->a_row,
                      R->b_row, R->sep, R->pair_off, row_off, R->n_pairs, a_off, J->a_row,
                      J->b_row, J->sep);
        if (nA > 0 && (with_un_a || !pairs_apart))
            XM_LAUNCH("k_write_a", grid_for(nA), kBlock, 0, s, k_write_a, R->count, R->pair_off,
                      R->b_row, R->sep, R->best_b, R->best_sep, row_off, nA, sel_all,
                      (int)with_pairs, (int)with_un_a, pairs_apart, a_off, J->a_row, J->b_row,
                      J->sep);
        if (write_b && nB > 0)
            XM_LAUNCH("k_write_b", grid_for(nB), kBlock, 0, s, k_write_b, bits, word_off, nB,
                      small + 0, J->a_row, J->b_row, J->sep);
        return XM_OK;
    };
    xm_status st = body();
    dev_free(own_bits, s);
    dev_free(rows, s);
    dev_free(row_off, s);
    dev_free(wcount, s);
    dev_free(word_off, s);
    if (st != XM_OK) {
        free_rows(J);  // (frees the counts too)
        return st;
    }
    *out = J;
    return XM_OK;
}

extern "C" xm_status xm_join(const xm_result* R, int32_t selection, int32_t join_type,
                             void* stream, xm_rows** out) {
    return join_impl(R, selection, join_type, nullptr, 0, true, stream, out, "xm_join");
}

extern "C" xm_status xm_result_mark_b(const xm_result* R, int32_t selection, uint32_t* bits,
                                      void* stream) {
    if (!R || !bits) return set_error(XM_EINVAL, "xm_result_mark_b: NULL argument");
    if (selection != XM_SEL_ALL && selection != XM_SEL_BEST)
        return set_error(XM_EINVAL, "xm_result_mark_b: selection must be ALL or BEST");
    if (!(R->selection & selection))
        return set_error(XM_EINVAL, "xm_result_mark_b: selection not computed by xm_match");
    cudaStream_t s = (cudaStream_t)stream;
    if (selection == XM_SEL_ALL) {
        if (R->n_pairs > 0)
            XM_LAUNCH("k_mark_b", grid_for(R->n_pairs), kBlock, 0, s, k_mark_b, R->b_row,
                      R->n_pairs, bits);
    } else if (R->n_a > 0) {
        XM_LAUNCH("k_mark_b", grid_for(R->n_a), kBlock, 0, s, k_mark_b, R->best_b, R->n_a, bits);
    }
    return XM_OK;
}

extern "C" xm_status xm_join_shard(const xm_result* R, int32_t selection, int32_t join_type,
                                   const uint32_t* b_matched, int64_t a_row_offset,
                                   int32_t with_b_rows, void* stream, xm_rows** out) {
    if (!b_matched) {
        if (out) *out = nullptr;
        return set_error(XM_EINVAL, "xm_join_shard: b_matched is NULL");
    }
    return join_impl(R, selection, join_type, b_matched, a_row_offset, with_b_rows != 0, stream,
                     out, "xm_join_shard");
}

extern "C" xm_status xm_rows_free(xm_rows* J) {
    free_rows(J);
    return XM_OK;
}

extern "C" xm_status xm_rows_get(const xm_rows* J, xm_rows_view* v) {
    if (!J || !v) return set_error(XM_EINVAL, "xm_rows_get: NULL argument");
    const xm_status st = resolve_rows(const_cast<xm_rows*>(J));
    if (st != XM_OK) return st;
    v->n = J->n;
    v->a_row = J->a_row;
    v->b_row = J->b_row;
    v->sep_arcsec = J->sep;
    v->n_unmatched_a = J->n_unmatched_a;
    v->n_unmatched_b = J->n_unmatched_b;
    return XM_OK;
}

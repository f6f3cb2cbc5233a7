// xm_sort.cu -- device radix sort and prefix sums.
//
// The sky partition of paper §2.3 assigns every source of the second
// catalogue to a cell; here the assignment is realised by sorting sources on
// a (zone, RA) key. The sort is a stable least-significant-digit radix sort
// with 8-bit digits, one pass per digit, each pass three phases with no
// inter-block waiting:
//   1. per tile of 4096 keys, a histogram of the pass's digit;
//   2. an exclusive scan of the digit-major (digit, tile) counts, giving each
//      tile the first output slot of each of its digits;
//   3. per tile, stable local ranks by warp-level match (lanes with equal
//      digits), a tile-local reorder in shared memory, then coalesced stores.
// Prefix sums are reduce-then-scan over tiles of 4096 elements, applied
// recursively to the tile sums.
#include "xm_internal.cuh"

namespace xm {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kWarps = kSortThreads / 32;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint64_t* __restrict__ keys,
                                                             int64_t n, int shift, int64_t ntiles,
                                                             int32_t* __restrict__ hist) {
    __shared__ int32_t h[kWarps][kRadix];
    int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int k = 0; k < kSortItems; k++) {
        int64_t i = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[warp][(keys[i] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        int32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) s += h[w][d];
        hist[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

struct ScatterSmem {
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
    int32_t wcount[kWarps][kRadix];  // per-warp digit counts, then warp offsets
    int32_t dstart[kRadix];          // tile-local start of each digit
    int64_t gstart[kRadix];          // global start of each digit for this tile
};

__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(
    const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, int64_t n,
    int shift, int64_t ntiles, const int64_t* __restrict__ offs, uint64_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&S.wcount[0][0])[i] = 0;
    __syncthreads();

    const int64_t tile_base = (int64_t)blockIdx.x * kSortTile;
    const int64_t warp_base = tile_base + (int64_t)warp * (kSortItems * 32);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    int32_t rank[kSortItems];
    // warp-striped: item k of lane l is element warp_base + 32 k + l, so the
    // (k, lane) order is the input order and ranks are stable
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        int64_t i = warp_base + 32 * k + lane;
        bool valid = i < n;
        key[k] = valid ? keys_in[i] : 0;
        val[k] = valid ? vals_in[i] : 0;
        uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        rank[k] = -1;
        if (valid) {
            uint32_t d = (uint32_t)(key[k] >> shift) & 0xFF;
            uint32_t peers = __match_any_sync(vmask, d);
            int32_t before = S.wcount[warp][d];
            rank[k] = before + __popc(peers & lt_mask);
            __syncwarp(vmask);
            if ((peers & lt_mask) == 0) S.wcount[warp][d] = before + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive scan over warps; tile total per digit
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        int32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            int32_t c = S.wcount[w][d];
            S.wcount[w][d] = run;
            run += c;
        }
        S.dstart[d] = run;  // total, scanned below
        S.gstart[d] = offs[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of 256 digit totals by one warp
        int32_t v[8], s = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) { v[j] = S.dstart[lane * 8 + j]; s += v[j]; }
        int32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int32_t run = incl - s;
#pragma unroll
        for (int j = 0; j < 8; j++) { S.dstart[lane * 8 + j] = run; run += v[j]; }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        if (rank[k] >= 0) {
            uint32_t d = (uint32_t)(key[k] >> shift) & 0xFF;
            int32_t p = S.dstart[d] + S.wcount[warp][d] + rank[k];
            S.keys[p] = key[k];
            S.vals[p] = val[k];
        }
    }
    __syncthreads();
    int64_t valid_n = n - tile_base;
    if (valid_n > kSortTile) valid_n = kSortTile;
    for (int p = threadIdx.x; p < valid_n; p += kSortThreads) {
        uint64_t kk = S.keys[p];
        uint32_t d = (uint32_t)(kk >> shift) & 0xFF;
        int64_t g = S.gstart[d] + (p - S.dstart[d]);
        keys_out[g] = kk;
        vals_out[g] = S.vals[p];
    }
}

// ------------------------------------------------------------- prefix sums

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ int64_t block_sum(int64_t v) {
    __shared__ int64_t red[kScanThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const T* __restrict__ in, int64_t n,
                                                            int64_t* __restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
#pragma unroll 4
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) v += (int64_t)in[i];
    }
    int64_t t = block_sum<T>(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

// Exclusive scan of one tile in blocked order (thread t owns elements
// [t*items, (t+1)*items)), offset by tile_offs[blockIdx] (or 0).
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T* __restrict__ in, int64_t n,
                                                            const int64_t* __restrict__ tile_offs,
                                                            int64_t* __restrict__ out,
                                                            int64_t* __restrict__ total) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        v[k] = i < n ? (int64_t)in[i] : 0;
        s += v[k];
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int64_t woff = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; w++) {
        if (w < warp) woff += warp_tot[w];
        all += warp_tot[w];
    }
    int64_t run = (tile_offs ? tile_offs[blockIdx.x] : 0) + woff + incl - s;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1)
        *total = (tile_offs ? tile_offs[blockIdx.x] : 0) + all;
}

template <typename T>
xm_status scan_impl(const T* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t s) {
    if (n <= 0) {
        if (total) {
            cudaError_t e = cudaMemsetAsync(total, 0, sizeof(int64_t), s);
            if (e != cudaSuccess) return cuda_fail(e, "memset");
        }
        return XM_OK;
    }
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        XM_LAUNCH("k_tile_scan", 1, kScanThreads, 0, s, k_tile_scan<T>, in, n, nullptr, out, total);
        return XM_OK;
    }
    int64_t* sums = (int64_t*)dev_alloc(2 * ntiles * sizeof(int64_t), s);
    if (!sums) return set_error(XM_ENOMEM, "scan: %lld tile sums", (long long)ntiles);
    int64_t* offs = sums + ntiles;
    xm_status st = XM_OK;
    do {
        launch_begin("k_tile_sums", s);
        k_tile_sums<T><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, sums);
        cudaError_t e = launch_end("k_tile_sums", s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_tile_sums"); break; }
        st = scan_impl<int64_t>(sums, offs, ntiles, nullptr, s);
        if (st != XM_OK) break;
        launch_begin("k_tile_scan", s);
        k_tile_scan<T><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, offs, out, total);
        e = launch_end("k_tile_scan", s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_tile_scan"); break; }
    } while (0);
    dev_free(sums, s);
    return st;
}

}  // namespace

xm_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                             cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, total, s);
}

xm_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                             cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, total, s);
}

xm_status radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n,
                         int end_bit, cudaStream_t s) {
    if (n <= 1 || end_bit <= 0) return XM_OK;
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    int32_t* hist = (int32_t*)dev_alloc(kRadix * ntiles * sizeof(int32_t), s);
    int64_t* offs = (int64_t*)dev_alloc(kRadix * ntiles * sizeof(int64_t), s);
    if (!hist || !offs) {
        dev_free(hist, s);
        dev_free(offs, s);
        return set_error(XM_ENOMEM, "radix sort of %lld keys", (long long)n);
    }
    static bool attr_done = false;
    size_t smem = sizeof(ScatterSmem);
    if (!attr_done) {
        cudaFuncSetAttribute(k_digit_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_done = true;
    }
    xm_status st = XM_OK;
    uint64_t *ki = keys, *ko = tk;
    uint32_t *vi = vals, *vo = tv;
    int passes = (end_bit + 7) / 8;
    for (int p = 0; p < passes && st == XM_OK; p++) {
        int shift = 8 * p;
        launch_begin("k_digit_hist", s);
        k_digit_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ki, n, shift, ntiles, hist);
        cudaError_t e = launch_end("k_digit_hist", s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_digit_hist"); break; }
        st = exclusive_scan_i32(hist, offs, kRadix * ntiles, nullptr, s);
        if (st != XM_OK) break;
        launch_begin("k_digit_scatter", s);
        k_digit_scatter<<<(unsigned)ntiles, kSortThreads, smem, s>>>(ki, vi, n, shift, ntiles, offs,
                                                                      ko, vo);
        e = launch_end("k_digit_scatter", s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_digit_scatter"); break; }
        uint64_t* t = ki; ki = ko; ko = t;
        uint32_t* u = vi; vi = vo; vo = u;
    }
    if (st == XM_OK && ki != keys) {
        cudaError_t e1 = cudaMemcpyAsync(keys, ki, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(vals, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = cuda_fail(e1 != cudaSuccess ? e1 : e2, "sort copy");
    }
    dev_free(hist, s);
    dev_free(offs, s);
    return st;
}

}  // namespace xm

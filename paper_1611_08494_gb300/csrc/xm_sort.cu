// xm_sort.cu -- device radix sort and prefix sums.
//
// The sky partition of paper §2.3 assigns every source of the second
// catalogue to a cell; here the assignment is realised by sorting sources on
// a (zone, RA) key. The sort is a stable least-significant-digit radix sort
// with 8-bit digits: one kernel counts the digits of every pass at once
// (they do not depend on the order of the keys) and turns the counts into
// output offsets, then one kernel per pass in the single-kernel Onesweep
// form: tiles of 4096 keys take ids in launch order, rank their keys stably
// per warp (lanes with equal digits found by one vote per digit bit), publish
// their per-digit counts, add the counts of earlier tiles by a decoupled
// look-back (bounded, see kSpinLimit), and scatter through shared memory so
// stores of one digit are contiguous.
// Prefix sums are reduce-then-scan over tiles of 4096 elements, applied
// recursively to the tile sums, or a single chained pass.
#include <atomic>
#include <mutex>

#include "xm_internal.cuh"

namespace xm {

namespace {

constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kWarps = kSortThreads / 32;
constexpr int kRadix = 256;

// The virtual key of an index key under a plan.
__device__ __forceinline__ uint64_t plan_key(const SortPlan& P, uint64_t key) {
    const uint32_t z = (uint32_t)(key >> 32);
    const uint32_t ra = (uint32_t)key >> kIndexSortBeginBit;
    const uint32_t rmask = P.rb >= 32 ? 0xFFFFFFFFu : ((1u << P.rb) - 1u);
    return ((uint64_t)(z - P.zmin) << P.rb) | (ra & rmask);
}

// Digit histograms of every pass at once (they do not depend on the order of
// the keys): hist[p * 256 + d] counts keys whose digit p is d; the digits are
// those of key >> begin_bit, or of the plan's virtual key. The last block to
// finish turns every pass's counts into exclusive offsets (the first output
// slot of each digit), so the passes need not scan them.
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint64_t* __restrict__ keys,
                                                             int64_t n, int begin_bit,
                                                             const SortPlan* plan, int passes,
                                                             unsigned long long* hist,
                                                             unsigned int* done) {
    pdl_wait();
    __shared__ uint32_t h[8][kRadix];
    __shared__ bool last;
    for (int i = threadIdx.x; i < 8 * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    SortPlan P{};
    if (plan) P = *plan;
    // (passes a plan leaves out are not counted: all their digits are 0)
    const int counted = plan ? min(passes, (int)P.active) : passes;
    for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kSortThreads) {
        const uint64_t k = plan ? plan_key(P, keys[i]) : keys[i] >> begin_bit;
        for (int p = 0; p < counted; p++) atomicAdd(&h[p][(k >> (8 * p)) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(&hist[i], (unsigned long long)v);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < passes) {  // one warp per pass: exclusive scan of its 256 counts
        unsigned long long* row = hist + warp * kRadix;
        unsigned long long v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) { v[j] = __ldcg(row + lane * 8 + j); sum += v[j]; }
        unsigned long long incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        unsigned long long run = incl - sum;
#pragma unroll
        for (int j = 0; j < 8; j++) { row[lane * 8 + j] = run; run += v[j]; }
    }
}

__global__ void k_plan_init(SortPlan* plan) {
    pdl_wait();
    *plan = SortPlan{0xFFFFFFFFu, 0u, 0xFFFFFFFFu, 0u, 0u, 0u};
}

// The plan from the accumulated ranges: bits of the zone offset and of the
// varying RA bits, passes needed (none for no keys).
__global__ void k_plan_finish(SortPlan* plan) {
    pdl_wait();
    SortPlan P = *plan;
    if (P.zmin > P.zmax) {
        P.rb = 0;
        P.active = 0;
        *plan = P;
        return;
    }
    const uint32_t ra_diff = P.ra_and ^ P.ra_or;
    P.rb = ra_diff ? 32 - __clz(ra_diff) : 0;
    const uint32_t zd = P.zmax - P.zmin;
    const uint32_t zb = zd ? 32 - __clz(zd) : 0;
    P.active = (P.rb + zb + 7) / 8;
    *plan = P;
}

// Look-back status word of one (tile, digit): flag in the top two bits,
// count (or inclusive prefix) below.
constexpr uint64_t kStAgg = 1ull << 62;   // tile's own count is available
constexpr uint64_t kStInc = 2ull << 62;   // inclusive prefix is available
constexpr uint64_t kStMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 22;      // polls before a look-back gives up (~1-2 s)
constexpr int kLookWindow = 8;           // status words loaded per look-back step

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A pass's shared memory; a pass that carries a 64-bit payload per key has
// kSortTile more words of it after the struct.
struct OnesweepSmem {
    uint64_t keys[kSortTile];
    uint32_t vals[kSortTile];
    uint8_t dig[kSortTile];          // digit of each placed key
    int32_t wcount[kWarps][kRadix];  // per-warp digit counts, then warp offsets
    int32_t hist[kRadix];            // the tile's digit counts (published early)
    int32_t dstart[kRadix];          // tile-local start of each digit
    int64_t gstart[kRadix];          // global start of each digit for this tile, less its
                                     // tile-local start (output slot = gstart[d] + p)
    int tile;
};

// One counting pass, in the single-kernel form of the Onesweep sort: tiles
// take ids in launch order from a counter, rank their keys stably in shared
// memory, publish their per-digit counts, add up the counts of the tiles
// before them by walking back through the published words until a tile with
// an inclusive prefix, then scatter through shared memory. A walk that finds
// no progress for kSpinLimit polls flags a timeout and carries on, so no
// block can wait forever; the caller turns the flag into XM_ETIMEOUT.
//
// spin_limit is the poll budget of one look-back (kSpinLimit unless a test
// lowers it); silent_tile (-1 = none) is a tile that publishes nothing, so
// the look-backs after it wait on words nobody writes -- the test form of a
// stalled predecessor, which must end in XM_ETIMEOUT and never in a hang.
//
// PAY: every key also carries a 64-bit payload (pay_in -> pay_out), moved
// with its row.
template <bool PAY>
__global__ void __launch_bounds__(kSortThreads, 2) k_onesweep(
    const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    const uint64_t* __restrict__ pay_in, int64_t n, int shift,
    const unsigned long long* __restrict__ offs, uint64_t* status, unsigned int* tile_counter,
    uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
    uint64_t* __restrict__ pay_out, int32_t* err, const SortPlan* plan, int pass,
    unsigned long long* stats, int spin_limit, int silent_tile) {
    pdl_wait();
    // with a plan: the digit of pass `pass` of the virtual key, and nothing
    // to do past the passes the plan needs (uniform over the grid)
    SortPlan P{};
    const bool planned = plan != nullptr;
    if (planned) {
        P = *plan;
        if (pass >= (int)P.active) return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnesweepSmem& S = *reinterpret_cast<OnesweepSmem*>(smem_raw);
    uint64_t* S_pay = reinterpret_cast<uint64_t*>(smem_raw + sizeof(OnesweepSmem));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int given_up;
    if (threadIdx.x == 0) {
        S.tile = (int)atomicAdd(tile_counter, 1u);
        if (S.tile == 0 && stats) {  // keys this pass (and with a payload)
            atomicAdd(&stats[5], (unsigned long long)n);
            if (PAY) atomicAdd(&stats[6], (unsigned long long)n);
        }
        given_up = (*(volatile int32_t*)err & kErrTimeout) != 0;
    }
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&S.wcount[0][0])[i] = 0;
    if (threadIdx.x < kRadix) S.hist[threadIdx.x] = 0;
    __syncthreads();
    const int tile = S.tile;
    // A look-back of this sort gave up (in this pass or an earlier one): the
    // keys of this pass may hold holes and repeats, so their digit counts no
    // longer match the offsets. Scatter nothing (every write stays in
    // bounds), and publish inclusive words so no later tile waits here; the
    // sort's guard then leaves a valid permutation for whoever reads it.
    if (given_up) {
        if (threadIdx.x < kRadix) st_relaxed(status + (int64_t)tile * kRadix + threadIdx.x, kStInc);
        return;
    }
    const int64_t tile_base = (int64_t)tile * kSortTile;
    const int64_t warp_base = tile_base + (int64_t)warp * (kSortItems * 32);
    const uint32_t lt_mask = (1u << lane) - 1u;
    // the digit's first output slot (thread d), read now so the load
    // overlaps the tile's own loads
    const unsigned long long off_d = threadIdx.x < kRadix ? offs[threadIdx.x] : 0ull;
    uint64_t key[kSortItems];
    int32_t rank[kSortItems];
    // warp-striped: item k of lane l is element warp_base + 32 k + l, so the
    // (k, lane) order is the input order and ranks are stable. All key loads
    // are issued before the ranking so they overlap; the rows (and payloads)
    // are read only when placed (fewer live registers: reading them with the
    // keys measured slower).
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        const int64_t i = warp_base + 32 * k + lane;
        key[k] = i < n ? keys_in[i] : 0;
    }
    // The tile's digit counts first (shared-memory atomics), published at
    // once: the tiles after this one find them while this one still ranks,
    // so their look-backs rarely wait.
    uint32_t dpack[kSortItems / 4] = {};
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        const uint32_t d = (uint32_t)((planned ? plan_key(P, key[k]) : key[k]) >> shift) & 0xFF;
        dpack[k >> 2] |= d << (8 * (k & 3));
        if (warp_base + 32 * k + lane < n) atomicAdd(&S.hist[d], 1);
    }
    __syncthreads();
    const bool silent = tile == silent_tile;
    if (threadIdx.x < kRadix && !silent) {
        const int d = threadIdx.x;
        st_relaxed(status + (int64_t)tile * kRadix + d,
                   (tile == 0 ? kStInc : kStAgg) | (uint64_t)S.hist[d]);
    }
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        const bool valid = warp_base + 32 * k + lane < n;
        const uint32_t d = (dpack[k >> 2] >> (8 * (k & 3))) & 0xFF;
        // lanes holding the same digit: one vote per digit bit (the
        // multisplit form), cheaper than a match instruction
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const uint32_t vote = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? vote : ~vote;
        }
        // every lane reads its digit's count, then the first lane of each
        // digit adds the digit's lanes (no per-digit synchronisation, which
        // would run the digits' lanes one group after another)
        const int32_t before = valid ? S.wcount[warp][d] : 0;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) S.wcount[warp][d] = before + __popc(peers);
        // rank within the warp's keys of digit d (< 256), the digit above it
        rank[k] = valid ? (int32_t)(d << 16) + before + __popc(peers & lt_mask) : -1;
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread d): warp offsets, tile count, look-back
    static_assert(kSortThreads >= kRadix, "one thread per digit");
    if (threadIdx.x < kRadix) {
        const int d = threadIdx.x;
        int32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            const int32_t c = S.wcount[w][d];
            S.wcount[w][d] = run;
            run += c;
        }
        S.dstart[d] = run;  // tile count (= hist[d]), scanned below
        uint64_t* my = status + (int64_t)tile * kRadix + d;
        int64_t prefix = 0;
        if (tile != 0) {  // (tile 0 published its inclusive counts already)
            // walk back kLookWindow tiles per step: their words are loaded
            // together, then taken in order until an inclusive prefix (done)
            // or a tile that has not published yet (wait there)
            int t = tile - 1;
            int spins = 0;
            bool done = false;
            while (t >= 0 && !done) {
                uint64_t w[kLookWindow];
#pragma unroll
                for (int j = 0; j < kLookWindow; j++)
                    w[j] = t - j >= 0 ? ld_relaxed(status + (int64_t)(t - j) * kRadix + d) : kStInc;
#pragma unroll
                for (int j = 0; j < kLookWindow; j++) {
                    if (done) break;
                    const uint64_t flag = w[j] & ~kStMask;
                    if (flag == 0) break;  // not published: reload from here
                    prefix += (int64_t)(w[j] & kStMask);  // (before tile 0: 0)
                    if (flag == kStInc) done = true;
                    else t--;
                }
                if (!done && t >= 0 && (w[0] & ~kStMask) == 0) {
                    if (++spins > spin_limit) {
                        atomicOr(err, kErrTimeout);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (!silent) st_relaxed(my, kStInc | (uint64_t)(prefix + run));
        }
        S.gstart[d] = (int64_t)off_d + prefix;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 tile counts by one warp
        int32_t v[8], sm = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) { v[j] = S.dstart[lane * 8 + j]; sm += v[j]; }
        int32_t incl = sm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int32_t run = incl - sm;
#pragma unroll
        for (int j = 0; j < 8; j++) { S.dstart[lane * 8 + j] = run; run += v[j]; }
    }
    __syncthreads();
    if (threadIdx.x < kRadix) S.gstart[threadIdx.x] -= S.dstart[threadIdx.x];
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
        if (rank[k] >= 0) {
            const uint32_t d = (uint32_t)rank[k] >> 16;
            const int32_t p = S.dstart[d] + S.wcount[warp][d] + (rank[k] & 0xFFFF);
            S.keys[p] = key[k];
            S.vals[p] = vals_in[warp_base + 32 * k + lane];
            if (PAY) S_pay[p] = pay_in[warp_base + 32 * k + lane];
            S.dig[p] = (uint8_t)d;
        }
    }
    __syncthreads();
    int64_t valid_n = n - tile_base;
    if (valid_n > kSortTile) valid_n = kSortTile;
#pragma unroll
    for (int j = 0; j < kSortItems; j++) {
        const int p = threadIdx.x + j * kSortThreads;
        if (p < valid_n) {
            const int64_t g = S.gstart[S.dig[p]] + p;
            if ((uint64_t)g < (uint64_t)n) {  // (always, unless a look-back gave up)
                keys_out[g] = S.keys[p];
                vals_out[g] = S.vals[p];
                if (PAY) pay_out[g] = S_pay[p];
            }
        }
    }
}

// After the counting passes of a sort: if a look-back gave up, the keys and
// rows are not a sorted permutation (a tile that timed out scattered with a
// partial prefix, later tiles and passes scattered nothing). Both buffers of
// the pair are then set to one valid, sorted content -- every key 0, rows in
// order -- so the kernels that read the sort before the host sees
// XM_ETIMEOUT index only rows that exist. Returns at once otherwise.
__global__ void k_sort_guard(const int32_t* err, uint64_t* k0, uint32_t* v0, uint64_t* k1,
                             uint32_t* v1, int64_t n) {
    pdl_wait();
    if (!(*(volatile const int32_t*)err & kErrTimeout)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        k0[i] = 0;
        k1[i] = 0;
        v0[i] = (uint32_t)i;
        v1[i] = (uint32_t)i;
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
    pdl_wait();
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
    pdl_wait();
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

// Single-pass exclusive scan: tiles take ids in launch order, scan their
// 4096 elements in blocked order, publish their sum, and add the sums of
// earlier tiles by a decoupled look-back in which one warp reads 32
// predecessors' words per step (bounded like the sort's; a timeout sets
// kErrTimeout in *err). The last tile writes the total.
// Elements move between global memory and the threads through shared memory
// (padded by one word per thread's run), so every global load and store is
// warp-contiguous while each thread scans kScanItems consecutive elements.
__device__ __forceinline__ int scan_pad(int e) { return e + (e >> 4); }

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_chained(
    const T* __restrict__ in, int64_t n, int64_t* __restrict__ out, int64_t* __restrict__ total,
    uint64_t* status, unsigned int* tile_counter, int32_t* err) {
    pdl_wait();
    static_assert(kScanItems == 16, "one pad word per 16 elements");
    __shared__ int64_t xs[kScanTile + kScanTile / 16];
    __shared__ int64_t warp_tot[kScanThreads / 32];
    __shared__ int64_t tile_prefix;
    __shared__ unsigned int tile_s;
    if (threadIdx.x == 0) tile_s = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const int64_t tile = tile_s;
    const int64_t tbase = tile * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int e = k * kScanThreads + threadIdx.x;
        xs[scan_pad(e)] = tbase + e < n ? (int64_t)in[tbase + e] : 0;
    }
    __syncthreads();
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = xs[scan_pad(threadIdx.x * kScanItems + k)];
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
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
    if (warp == 0) {  // publish, then look back 32 tiles per step
        uint64_t* my = status + tile;
        int64_t prefix = 0;
        if (tile == 0) {
            if (lane == 0) st_relaxed(my, kStInc | (uint64_t)all);
        } else {
            if (lane == 0) st_relaxed(my, kStAgg | (uint64_t)all);
            int64_t top = tile - 1;  // lane j reads tile top - j (before tile 0: an inclusive 0)
            int spins = 0;
            while (true) {
                const int64_t j = top - lane;
                const uint64_t w = j >= 0 ? ld_relaxed(status + j) : kStInc;
                const uint64_t flag = w & ~kStMask;
                const uint32_t inc = __ballot_sync(0xffffffffu, flag == kStInc);
                const uint32_t unready = __ballot_sync(0xffffffffu, flag == 0);
                const int first = inc ? __ffs(inc) - 1 : 31;  // words needed: lanes 0..first
                const uint32_t need = first == 31 ? 0xffffffffu : ((1u << (first + 1)) - 1u);
                if (unready & need) {
                    if (++spins > kSpinLimit) {
                        if (lane == 0) atomicOr(err, kErrTimeout);
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                int64_t v = lane <= first ? (int64_t)(w & kStMask) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                prefix += v;
                if (inc) break;
                top -= 32;
            }
            if (lane == 0) st_relaxed(my, kStInc | (uint64_t)(prefix + all));
        }
        if (lane == 0) {
            tile_prefix = prefix;
            if (total && (tile + 1) * kScanTile >= n) *total = prefix + all;
        }
    }
    __syncthreads();
    int64_t run = tile_prefix + woff + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        xs[scan_pad(threadIdx.x * kScanItems + k)] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int e = k * kScanThreads + threadIdx.x;
        if (tbase + e < n) out[tbase + e] = xs[scan_pad(e)];
    }
}

template <typename T>
xm_status scan_impl(const T* in, int64_t* out, int64_t n, int64_t* total, int32_t* err,
                    cudaStream_t s) {
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
    // status words of the tiles and the tile counter
    const size_t bytes = (size_t)(ntiles + 1) * sizeof(uint64_t);
    uint64_t* status = (uint64_t*)dev_alloc(bytes, s);
    if (!status) return set_error(XM_ENOMEM, "scan: %lld tiles", (long long)ntiles);
    unsigned int* counter = (unsigned int*)(status + ntiles);
    xm_status st = XM_OK;
    cudaError_t e = cudaMemsetAsync(status, 0, bytes, s);
    if (e != cudaSuccess) st = cuda_fail(e, "scan memset");
    if (st == XM_OK) {
        launch_begin("k_scan_chained", s);
        launch_pdl(k_scan_chained<T>, dim3((unsigned)ntiles), dim3(kScanThreads), 0, s, in, n, out,
                   total, status, counter, err);
        e = launch_end("k_scan_chained", s);
        if (e != cudaSuccess) st = cuda_fail(e, "k_scan_chained");
    }
    dev_free(status, s);
    return st;
}

}  // namespace

// Exclusive scan of up to 4096 tiles of int32 input with caller-provided
// workspace (2 * ceil(n / 4096) int64 values) instead of allocations; used
// by the entry point that must not allocate. Plain launches, no profiling.
xm_status exclusive_scan_i32_ws(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                                int64_t* ws, cudaStream_t s) {
    if (n <= 0) {
        if (total && cudaMemsetAsync(total, 0, sizeof(int64_t), s) != cudaSuccess)
            return set_error(XM_ECUDA, "scan memset");
        return XM_OK;
    }
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > kScanTile) return set_error(XM_EOVERFLOW, "scan workspace: %lld elements", (long long)n);
    if (ntiles == 1) {
        k_tile_scan<int32_t><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out, total);
    } else {
        k_tile_sums<int32_t><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, ws);
        k_tile_scan<int64_t><<<1, kScanThreads, 0, s>>>(ws, ntiles, nullptr, ws + ntiles, nullptr);
        k_tile_scan<int32_t><<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, ws + ntiles, out, total);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? XM_OK : cuda_fail(e, "scan");
}

xm_status exclusive_scan_i32(const int32_t* in, int64_t* out, int64_t n, int64_t* total,
                             int32_t* err, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, total, err, s);
}

xm_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                             int32_t* err, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, total, err, s);
}

size_t onesweep_smem(bool pay) {
    return sizeof(OnesweepSmem) + (pay ? kSortTile * sizeof(uint64_t) : 0);
}

void radix_sort_prepare() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(k_onesweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)onesweep_smem(false));
    cudaFuncSetAttribute(k_onesweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)onesweep_smem(true));
    done[dev] = true;
}

// Test settings of the look-back (xm_debug_lookback): poll budget and the
// tile that withholds its status words.
std::atomic<int> g_spin_limit{kSpinLimit};
std::atomic<int> g_silent_tile{-1};

// One pass: two tiles of 512 threads x 8 keys per SM (64 registers, no
// spills). Tiles of 256 x 16, 256 x 8, 384 x 12 and 512 x 12 keys, two to
// four per SM with the rows read with the keys, measured from 3 % faster to
// 29 % slower on the all-sky index.
void onesweep_pass(int64_t ntiles, cudaStream_t s, const uint64_t* ki, const uint32_t* vi,
                   const uint64_t* pi, int64_t n, int shift, const unsigned long long* offs,
                   uint64_t* status, unsigned int* counter, uint64_t* ko, uint32_t* vo,
                   uint64_t* po, int32_t* err, const SortPlan* plan, int pass) {
    if (pi)
        launch_pdl(k_onesweep<true>, dim3((unsigned)ntiles), dim3(kSortThreads), onesweep_smem(true),
                   s, ki, vi, pi, n, shift, offs, status, counter, ko, vo, po, err, plan, pass,
                   device_stats(), g_spin_limit.load(), g_silent_tile.load());
    else
        launch_pdl(k_onesweep<false>, dim3((unsigned)ntiles), dim3(kSortThreads), onesweep_smem(false),
                   s, ki, vi, pi, n, shift, offs, status, counter, ko, vo, po, err, plan, pass,
                   device_stats(), g_spin_limit.load(), g_silent_tile.load());
}

xm_status sort_guard(const int32_t* err, uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1,
                     int64_t n, cudaStream_t s) {
    XM_LAUNCH("k_sort_guard", 2 * 152, 256, 0, s, k_sort_guard, err, k0, v0, k1, v1, n);
    return XM_OK;
}

xm_status sort_plan_init(SortPlan* plan, cudaStream_t s) {
    XM_LAUNCH("k_plan_init", 1, 1, 0, s, k_plan_init, plan);
    return XM_OK;
}

xm_status index_sort(uint64_t* keys, uint32_t* vals, uint64_t* pay, uint64_t* tk, uint32_t* tv,
                     uint64_t* tp, int64_t n, SortPlan* plan, int max_passes, int32_t* err,
                     cudaStream_t s) {
    if (max_passes < 1 || max_passes > 8) return set_error(XM_EINVAL, "index sort: passes");
    XM_LAUNCH("k_plan_finish", 1, 1, 0, s, k_plan_finish, plan);
    if (n <= 1) return XM_OK;  // (one key: the plan needs no pass)
    const int passes = max_passes;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const size_t st_words = (size_t)ntiles * kRadix;
    const size_t bytes = passes * (kRadix * sizeof(unsigned long long) + st_words * sizeof(uint64_t) +
                                   sizeof(uint64_t)) + 16;
    unsigned char* work = (unsigned char*)dev_alloc(bytes, s);
    if (!work) return set_error(XM_ENOMEM, "index sort of %lld keys", (long long)n);
    unsigned long long* hist = (unsigned long long*)work;
    uint64_t* status = (uint64_t*)(hist + passes * kRadix);
    unsigned int* counters = (unsigned int*)(status + passes * st_words);
    radix_sort_prepare();
    xm_status st = XM_OK;
    cudaError_t e = cudaMemsetAsync(work, 0, bytes, s);
    if (e != cudaSuccess) st = cuda_fail(e, "index sort memset");
    if (st == XM_OK) {
        const unsigned hg = (unsigned)(ntiles < 4 * 152 ? ntiles : 4 * 152);
        launch_begin("k_digit_hist", s);
        // (counters + passes: a spare word of the zeroed work area)
        launch_pdl(k_digit_hist, dim3(hg), dim3(kSortThreads), 0, s, keys, n, 0, plan, passes, hist,
                   counters + passes);
        e = launch_end("k_digit_hist", s);
        if (e != cudaSuccess) st = cuda_fail(e, "k_digit_hist");
    }
    uint64_t *ki = keys, *ko = tk, *pi = pay, *po = tp;
    uint32_t *vi = vals, *vo = tv;
    for (int p = 0; p < passes && st == XM_OK; p++) {
        launch_begin("k_onesweep", s);
        onesweep_pass(ntiles, s, ki, vi, pi, n, 8 * p, hist + p * kRadix, status + p * st_words,
                      counters + p, ko, vo, po, err, plan, p);
        e = launch_end("k_onesweep", s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_onesweep"); break; }
        uint64_t* t = ki; ki = ko; ko = t;
        uint32_t* u = vi; vi = vo; vo = u;
        t = pi; pi = po; po = t;
    }
    if (st == XM_OK) st = sort_guard(err, keys, vals, tk, tv, n, s);
    dev_free(work, s);
    return st;
}

xm_status radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* tk, uint32_t* tv, int64_t n,
                         int begin_bit, int end_bit, int32_t* err, cudaStream_t s) {
    if (n <= 1 || end_bit <= begin_bit) return XM_OK;
    const int passes = (end_bit - begin_bit + 7) / 8;
    if (passes > 8) return set_error(XM_EINVAL, "radix sort: more than 64 key bits");
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    // per pass: 256 histogram counters (then offsets), ntiles x 256 status
    // words, a tile counter; plus the histogram kernel's completion counter
    const size_t st_words = (size_t)ntiles * kRadix;
    const size_t bytes = passes * (kRadix * sizeof(unsigned long long) + st_words * sizeof(uint64_t) +
                                   sizeof(uint64_t)) + 16;
    unsigned char* work = (unsigned char*)dev_alloc(bytes, s);
    if (!work) return set_error(XM_ENOMEM, "radix sort of %lld keys", (long long)n);
    unsigned long long* hist = (unsigned long long*)work;
    uint64_t* status = (uint64_t*)(hist + passes * kRadix);
    unsigned int* counters = (unsigned int*)(status + passes * st_words);
    radix_sort_prepare();
    xm_status st = XM_OK;
    cudaError_t e = cudaMemsetAsync(work, 0, bytes, s);
    if (e != cudaSuccess) st = cuda_fail(e, "radix sort memset");
    uint64_t *ki = keys, *ko = tk;
    uint32_t *vi = vals, *vo = tv;
    if (st == XM_OK) {
        const unsigned hg = (unsigned)(ntiles < 4 * 152 ? ntiles : 4 * 152);
        launch_begin("k_digit_hist", s);
        launch_pdl(k_digit_hist, dim3(hg), dim3(kSortThreads), 0, s, keys, n, begin_bit,
                   (const SortPlan*)nullptr, passes, hist, counters + passes);
        e = launch_end("k_digit_hist", s);
        if (e != cudaSuccess) st = cuda_fail(e, "k_digit_hist");
    }
    for (int p = 0; p < passes && st == XM_OK; p++) {
        launch_begin("k_onesweep", s);
        onesweep_pass(ntiles, s, ki, vi, nullptr, n, begin_bit + 8 * p, hist + p * kRadix,
                      status + p * st_words, counters + p, ko, vo, nullptr, err, nullptr, p);
        e = launch_end("k_onesweep", s);
        if (e != cudaSuccess) { st = cuda_fail(e, "k_onesweep"); break; }
        uint64_t* t = ki; ki = ko; ko = t;
        uint32_t* u = vi; vi = vo; vo = u;
    }
    if (st == XM_OK) st = sort_guard(err, keys, vals, tk, tv, n, s);
    if (st == XM_OK && ki != keys) {
        cudaError_t e1 = cudaMemcpyAsync(keys, ki, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(vals, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = cuda_fail(e1 != cudaSuccess ? e1 : e2, "sort copy");
    }
    dev_free(work, s);
    return st;
}

}  // namespace xm

extern "C" xm_status xm_debug_lookback(int32_t spin_limit, int32_t silent_tile) {
    using namespace xm;
    if (spin_limit < 0 || silent_tile < -1)
        return set_error(XM_EINVAL, "xm_debug_lookback: spin_limit %d, silent_tile %d", spin_limit,
                         silent_tile);
    g_spin_limit.store(spin_limit ? spin_limit : kSpinLimit);
    g_silent_tile.store(silent_tile);
    return XM_OK;
}

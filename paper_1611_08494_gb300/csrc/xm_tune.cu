// xm_tune.cu -- the autotuner. The paper leaves the resolution of its sky
// partition and the number of concurrent processes to the user (§2.3, §4);
// here both are chosen by timed trials: the zone height of the index (one
// build per candidate) and the blocks per SM of the persistent batch kernel,
// on a sample batch of the real workload. Answers are cached per
// (size of B, frame, sample size, precision, candidate lists).
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "xm_internal.cuh"

namespace {

using Key = std::tuple<int64_t, int32_t, int64_t, int64_t, int32_t, std::vector<double>,
                       std::vector<int32_t>>;
std::map<Key, xm_tuned> g_cache;
std::mutex g_cache_mu;

}  // namespace

extern "C" xm_status xm_autotune(const xm_columns* B, const xm_request* sample, int64_t n_sample,
                                 const xm_tune_space* space, int32_t precision, void* stream,
                                 xm_tuned* out) {
    using namespace xm;
    if (!B || !out || n_sample < 1 || !sample)
        return set_error(XM_EINVAL, "xm_autotune: bad arguments");
    std::vector<double> zh;
    std::vector<int32_t> bl;
    if (space && space->n_zone_heights > 0)
        zh.assign(space->zone_heights_arcsec,
                  space->zone_heights_arcsec + std::min(space->n_zone_heights, 8));
    else
        zh = {6.0, 12.0, 24.0, 48.0};
    if (space && space->n_blocks > 0)
        bl.assign(space->blocks_per_sm, space->blocks_per_sm + std::min(space->n_blocks, 4));
    else
        bl = {2, 4, 8};
    const int reps = (space && space->repeats > 0) ? space->repeats : 2;
    int64_t total_a = 0;
    for (int64_t r = 0; r < n_sample; r++) total_a += sample[r].A.n;
    const Key key{B->n, B->frame, n_sample, total_a, precision, zh, bl};
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *out = it->second;
            out->trials = 0;
            return XM_OK;
        }
    }
    xm_tuned best{0.0, 0, 0, 1e300};
    for (double h : zh) {
        xm_index_opts io{h, 0, 0};
        xm_index* idx = nullptr;
        xm_status st = xm_build_index(B, &io, stream, &idx);
        if (st != XM_OK) return st;
        for (int32_t b : bl) {
            double ms_min = 1e300;
            for (int k = 0; k < reps; k++) {
                xm_batch_opts bo{precision, 0, b, 0, 0, 0};
                xm_batch* batch = nullptr;
                st = xm_match_batch(idx, sample, n_sample, &bo, stream, &batch);
                if (st != XM_OK) {
                    xm_index_free(idx);
                    return st;
                }
                double ms = 0.0;
                xm_batch_info(batch, nullptr, nullptr, &ms);
                xm_batch_free(batch);
                ms_min = std::min(ms_min, ms);
            }
            best.trials++;
            if (ms_min < best.best_ms) {
                best.best_ms = ms_min;
                best.zone_height_arcsec = h;
                best.persistent_blocks = b;
            }
        }
        xm_index_free(idx);
    }
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        g_cache[key] = best;
    }
    *out = best;
    return XM_OK;
}

// Tile-schedule autotuner of a batched call (interp_tune_batched).
//
// The persistent tile launches split every column of every field into work
// items of `run` consecutive 8-plane slabs and run a grid of CTAs per SM.
// Longer runs recompute fewer closing planes; shorter ones spread the work of
// uneven fields more evenly over the CTAs; fewer resident CTAs leave each one
// more of the SM.  Which balance wins depends on the batch, so the tuner times
// the candidates on the device, picks the fastest for compression and for
// decompression, and remembers the pick for batches of the same shapes.
#include <cinttypes>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace {

// The batch as the tuner sees it: shapes, configuration, bounds and the
// alignment of the buffers that decide which load and store paths run.
std::string batch_key(const interp_compress_item *c, int n)
{
    std::string k;
    char buf[256];
    for (int i = 0; i < n; ++i) {
        const interp_config &g = c[i].cfg;
        std::snprintf(buf, sizeof(buf),
                      "%" PRId64 "x%" PRId64 "x%" PRId64 ";%d%d%d;%d%d%d;%d%d%d;%d;%d;%d;%d;%d;%.17g;%.17g;%d%d|",
                      c[i].dims[0], c[i].dims[1], c[i].dims[2], g.dim_order[0], g.dim_order[1], g.dim_order[2],
                      g.level_kind[0], g.level_kind[1], g.level_kind[2], g.cubic_kind[0], g.cubic_kind[1],
                      g.cubic_kind[2], g.eb_mode, g.autotune, g.radius, g.domain_x, g.ndim, g.alpha, c[i].eb,
                      (int)(reinterpret_cast<uintptr_t>(c[i].d_x) % 16 == 0),
                      (int)(reinterpret_cast<uintptr_t>(c[i].d_codes) % 16 == 0));
        k += buf;
    }
    return k;
}

struct Picked {
    interp_tile_schedule c, d;
};

std::mutex g_mu;
std::map<std::string, Picked> g_cache;

// Candidate schedules: the cost model's run and fixed runs up to whole columns,
// each with the occupancy limit and one or two CTAs per SM fewer.
std::vector<interp_tile_schedule> candidates(const interp_compress_item *c, int n)
{
    int max_slabs = 1;
    for (int i = 0; i < n; ++i) max_slabs = std::max(max_slabs, (int)((c[i].dims[0] - 1 + 7) / 8));
    std::vector<int> runs{0};
    for (int r = 1; r < max_slabs; r *= 2) runs.push_back(r);
    runs.push_back(max_slabs);
    std::vector<interp_tile_schedule> out;
    for (int r : runs)
        for (int ctas : {0, 4, 3}) out.push_back(interp_tile_schedule{r, ctas});
    return out;
}

}  // namespace

extern "C" int interp_tune_batched(const interp_compress_item *citems, const interp_decompress_item *ditems, int n,
                                   int32_t force, interp_tile_schedule *csched, interp_tile_schedule *dsched,
                                   interp_stream_t stream)
{
    if (!citems || !ditems || !csched || !dsched || n < 1 || n > gi::kMaxBatch) return INTERP_EINVAL;
    const std::string key = batch_key(citems, n);
    if (!force) {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *csched = it->second.c;
            *dsched = it->second.d;
            return INTERP_OK;
        }
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        return INTERP_ECUDA;
    }
    const std::vector<interp_tile_schedule> cand = candidates(citems, n);
    int rc = INTERP_OK;
    // time(kind, schedule): one warm-up call, then the mean of two, in milliseconds
    auto timed = [&](bool compress, const interp_tile_schedule &sc, float &ms) -> int {
        auto call = [&]() {
            return compress ? interp_compress_batched_scheduled(citems, n, &sc, stream)
                            : interp_decompress_batched_scheduled(ditems, n, &sc, stream);
        };
        int r = call();
        if (r != INTERP_OK) return r;
        if (cudaEventRecord(ev[0], s) != cudaSuccess) return INTERP_ECUDA;
        for (int k = 0; k < 2 && r == INTERP_OK; ++k) r = call();
        if (r != INTERP_OK) return r;
        if (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess) return INTERP_ECUDA;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) return INTERP_ECUDA;
        ms *= 0.5f;
        return INTERP_OK;
    };
    Picked best{};
    float best_c = 1e30f, best_d = 1e30f;
    for (const auto &sc : cand) {
        float ms = 0.0f;
        rc = timed(true, sc, ms);
        if (rc != INTERP_OK) break;
        if (ms < best_c) {
            best_c = ms;
            best.c = sc;
        }
    }
    // decompression reads the codes of the last compression, identical for every schedule
    for (const auto &sc : cand) {
        if (rc != INTERP_OK) break;
        float ms = 0.0f;
        rc = timed(false, sc, ms);
        if (rc != INTERP_OK) break;
        if (ms < best_d) {
            best_d = ms;
            best.d = sc;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != INTERP_OK) return rc;
    *csched = best.c;
    *dsched = best.d;
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = best;
    return INTERP_OK;
}

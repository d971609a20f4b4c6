// pg_tune.cu -- autotuner for the traversal launch shape.
//
// The paper leaves tau tunable (Sec. 2.1); on the GPU the local-queue size,
// the task chunk, the threads per CTA and the CTAs per SM matter as much, and
// so do the load-balance thresholds of high-degree splitting.
// Knobs, single-source BFS and reachability: local-search organisation (CTA
// / warp), tau, task chunk, warp queue, CTA queue, threads per CTA, CTAs per
// SM, hub degree (the out-degree from which a vertex's edges are split).
// Knobs, batched BFS: chunk length of the high-degree split (hub_degree),
// the push-to-pull threshold alpha, CTAs per SM.
// Coordinate descent: for each knob in turn, time every candidate value
// with the others fixed at the best so far (median of `trials` CUDA-event
// timed runs) and keep the fastest.  Outputs go to scratch buffers that the
// tuner allocates and frees itself.
#include <algorithm>
#include <vector>

#include "pg_internal.cuh"

namespace {

pg_status time_once(pg_graph *g, uint32_t kind, const uint32_t *sources, uint32_t k, uint32_t dir,
                    void *out0, void *out1, const pg_config &c, cudaStream_t s, cudaEvent_t e0,
                    cudaEvent_t e1, float *ms) {
    PG_CK(cudaEventRecord(e0, s));
    pg_status st = (kind == 0)   ? pg_bfs(g, sources[0], (uint32_t *)out0, &c, nullptr, s)
                   : (kind == 1) ? pg_reach_multi(g, sources, k, dir, (uint64_t *)out0,
                                                  (uint64_t *)out1, &c, nullptr, s)
                                 : pg_bfs_multi(g, sources, k, (uint32_t *)out0, &c, nullptr, s);
    if (st) return st;
    PG_CK(cudaEventRecord(e1, s));
    PG_CK(cudaEventSynchronize(e1));
    PG_CK(cudaEventElapsedTime(ms, e0, e1));
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_autotune(pg_graph *g, uint32_t kind, const uint32_t *sources, uint32_t k,
                                 uint32_t dir, uint32_t trials, pg_config *cfg, void *stream) {
    if (!g || !sources || !cfg) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (kind > 2) return pg_set_error(PG_ERR_INVALID_ARG, "kind %u", kind);
    if (kind >= 1 && (k == 0 || k > 64)) return pg_set_error(PG_ERR_INVALID_ARG, "k=%u", k);
    if (cfg->struct_size != sizeof(pg_config))
        return pg_set_error(PG_ERR_INVALID_ARG, "pg_config.struct_size mismatch");
    if (trials == 0) trials = 1;
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    void *out0 = nullptr, *out1 = nullptr;
    const size_t bytes = (size_t)g->n * (kind == 0   ? sizeof(uint32_t)
                                         : kind == 1 ? sizeof(uint64_t)
                                                     : (size_t)k * sizeof(uint32_t));
    PG_CK(cudaMalloc(&out0, bytes));
    if (kind == 1 && cudaMalloc(&out1, bytes) != cudaSuccess) {
        cudaFree(out0);
        return pg_cuda_error(cudaErrorMemoryAllocation, "cudaMalloc(autotune)");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pg_config best = *cfg;
    best.schedule = PG_SCHED_FIXED;
    best.trace_out = nullptr;
    best.trace_cap = 0;
    pg_status st = PG_OK;
    float best_ms = 1e30f;
    auto measure = [&](const pg_config &c, float *med) -> pg_status {
        std::vector<float> t;
        for (uint32_t i = 0; i < trials; i++) {
            float ms = 0;
            pg_status r = time_once(g, kind, sources, k, dir, out0, out1, c, s, e0, e1, &ms);
            if (r) return r;
            t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        *med = t[t.size() / 2];
        return PG_OK;
    };
    // warm-up and baseline
    st = measure(best, &best_ms);
    const uint32_t modes[] = {PG_VGC_CTA, PG_VGC_WARP};
    const uint32_t taus[] = {1, 2, 4, 8, 16, 32, 64};
    const uint32_t chunks[] = {1, 2, 4, 8, 32};
    const uint32_t queues[] = {128, 512, 2048};
    const uint32_t ctaq[] = {1024, 2048, 4096};
    const uint32_t threads[] = {256, 512};
    const uint32_t bps[] = {1, 2, 3, 4};
    const uint32_t hubs[] = {512, 2048, 8192};
    const uint32_t clens[] = {256, 512, 1024, 2048, 4096};
    const uint32_t alphas[] = {4, 8, 15, 30};
    // knob ids: 0 mode, 1 tau, 2 chunk, 3 warp queue, 4 CTA queue, 5 threads,
    // 6 CTAs per SM, 7 hub degree, 8 batched chunk length, 9 alpha
    const int knobs_single[] = {0, 1, 2, 3, 4, 5, 6, 7};
    const int knobs_batch[] = {8, 9, 6};
    const int *knobs = kind == 2 ? knobs_batch : knobs_single;
    const int nknobs = kind == 2 ? 3 : 8;
    for (int ki = 0; ki < nknobs && !st; ki++) {
        const int knob = knobs[ki];
        const uint32_t *vals;
        int nv;
        switch (knob) {
            case 0: vals = modes; nv = 2; break;
            case 1: vals = taus; nv = 7; break;
            case 2: vals = chunks; nv = 5; break;
            case 3: vals = queues; nv = 3; break;
            case 4: vals = ctaq; nv = 3; break;
            case 5: vals = threads; nv = 2; break;
            case 6: vals = bps; nv = 4; break;
            case 7: vals = hubs; nv = 3; break;
            case 8: vals = clens; nv = 5; break;
            default: vals = alphas; nv = 4; break;
        }
        pg_config cur = best;
        for (int i = 0; i < nv && !st; i++) {
            pg_config c = best;
            switch (knob) {
                case 0: c.vgc_mode = vals[i]; break;
                case 1: c.tau = vals[i]; break;
                case 2: c.chunk = vals[i]; break;
                case 3: c.local_queue = vals[i]; break;
                case 4: c.cta_queue = vals[i]; break;
                case 5: c.threads_per_block = vals[i]; break;
                case 6: c.blocks_per_sm = vals[i]; break;
                case 7: case 8: c.hub_degree = vals[i]; break;
                default: c.alpha = vals[i]; break;
            }
            float ms = 0;
            pg_status r = measure(c, &ms);
            if (r == PG_ERR_INVALID_ARG) continue;  // shape does not fit: skip
            if (r) { st = r; break; }
            if (ms < best_ms) { best_ms = ms; cur = c; }
        }
        best = cur;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out0);
    cudaFree(out1);
    if (st) return st;
    cfg->blocks_per_sm = best.blocks_per_sm;
    cfg->hub_degree = best.hub_degree;
    if (kind == 2) {
        cfg->alpha = best.alpha;
        return PG_OK;
    }
    cfg->vgc_mode = best.vgc_mode;
    cfg->cta_queue = best.cta_queue;
    cfg->tau = best.tau;
    cfg->chunk = best.chunk;
    cfg->local_queue = best.local_queue;
    cfg->threads_per_block = best.threads_per_block;
    return PG_OK;
}

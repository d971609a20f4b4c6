// pg_sssp.cu -- single-source shortest paths with uint32 arc weights (pg_sssp).
//
// Sec. 2.2 (parallel SSSP): the stepping-algorithm framework, with vertical
// granularity control and a frontier bag.  Round i of Algorithm 1 takes the
// frontier bag F_i; the smallest tentative distance L among its entries and
// the step width delta give the round's threshold theta = L + delta.  Entries
// below theta are expanded (every out-arc relaxed with a 64-bit atomicMin on
// the target's distance); entries at or above theta are kept for a later
// round.  With VGC a warp keeps expanding, in a shared-memory FIFO, the
// vertices its own relaxations improve below theta (up to tau x 8 local
// expansions per task of 32 frontier entries), so one round covers many
// hops of a step; every other improvement goes to the next bag (one entry
// per vertex and round, de-duplicated by a round tag).  Every improvement is
// expanded or queued, so when the bag is empty every arc satisfies
// dist[x] <= dist[u] + w(u, x) and every distance is a real path length:
// the exact shortest-path distances, whatever delta and tau.
#include "pg_internal.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr unsigned long long kInf64 = ~0ull;
constexpr uint32_t kSp = 128;  // per-warp spill staging entries

// Per-round counters; round r reads slot r % 4 and fills slot (r + 1) % 4.
struct alignas(128) SsCount {
    unsigned size;            // entries appended to the bag
    unsigned head;            // grab cursor
    unsigned pad0, pad1;
    unsigned long long min;   // smallest distance of an attempted append
    unsigned long long pad[13];
};

}  // namespace

struct PgSsspWork {
    uint32_t *w;                // arc weights, forward CSR order
    unsigned long long wsum;    // their sum (automatic step width)
    SsCount *cnt;               // [4]
};

void pg_sssp_release(pg_graph *g) {
    if (g && g->sssp) {
        cudaFree(g->sssp->w);
        cudaFree(g->sssp->cnt);
        delete g->sssp;
        g->sssp = nullptr;
    }
}

namespace {

struct SsArgs {
    const uint32_t *off, *idx, *w;
    uint32_t n;
    unsigned long long *dist;
    uint32_t *bag;     // [2][cap]
    uint32_t cap;
    uint32_t *stamp;   // [n] round tags
    uint32_t tag0;
    PgCtrl *ctrl;
    SsCount *cnt;
    uint32_t src;
    unsigned long long delta;
    uint32_t budget;   // local expansions per task
    uint32_t qcap;     // local FIFO entries (power of two)
    unsigned long long timeout_ns;
    uint32_t max_rounds, stall_block;
};

struct SsWarp {
    uint32_t *incl, *base;      // [32] edge deal of a wave
    unsigned long long *val;    // [32]
    uint32_t *lq;               // local FIFO [qcap]: vertex
    unsigned long long *lqd;    //                    its distance
    uint32_t *sp;               // spill staging [kSp]
    unsigned long long *spd;
};

struct SsTask {
    uint32_t qhead, qtail, budget, nsp;
    unsigned long long mn;      // this lane's smallest attempted append
};

__device__ __forceinline__ unsigned long long wmin64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Append the lanes' staged spills (batches of 32) to the next bag.
__device__ void ss_flush(const SsArgs &A, SsCount *sn, uint32_t nxt, uint32_t tag, const SsWarp &S,
                         SsTask &T, int lane, unsigned long long &pushes) {
    __syncwarp();
    for (uint32_t b0 = 0; b0 < T.nsp; b0 += 32u) {
        const uint32_t i = b0 + (uint32_t)lane;
        const bool go = i < T.nsp;
        uint32_t v = 0;
        if (go) {
            v = S.sp[i];
            T.mn = min(T.mn, S.spd[i]);
        }
        const bool keep = go && atomicExch(A.stamp + v, tag) != tag;
        const unsigned bal = __ballot_sync(kFull, keep);
        if (!bal) continue;
        uint32_t pos = 0;
        if (lane == 0) pos = atomicAdd(&sn->size, (unsigned)__popc(bal));
        pos = __shfl_sync(kFull, pos, 0);
        if (keep) {
            const uint32_t p = pos + __popc(bal & lanemask_lt());
            if (p < A.cap) A.bag[(size_t)nxt * A.cap + p] = v;
            else atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
        }
        if (lane == 0) pushes += __popc(bal);
    }
    T.nsp = 0;
    __syncwarp();
}

// Route each lane's improved vertex: into the local FIFO when it lies below
// theta and there is room and budget, else into the spill staging.
__device__ __forceinline__ void ss_route(const SsArgs &A, SsCount *sn, uint32_t nxt, uint32_t tag,
                                         const SsWarp &S, SsTask &T, bool imp, uint32_t x,
                                         unsigned long long nd, unsigned long long theta, int lane,
                                         unsigned long long &pushes) {
    const unsigned lt = lanemask_lt();
    const bool want = imp && nd < theta;
    const unsigned bl = __ballot_sync(kFull, want);
    bool loc = false;
    if (bl) {
        const uint32_t room = min(A.qcap - (T.qtail - T.qhead), T.budget);
        const uint32_t nl = min((uint32_t)__popc(bl), room);
        const uint32_t rank = __popc(bl & lt);
        loc = want && rank < nl;
        if (loc) {
            const uint32_t p = (T.qtail + rank) & (A.qcap - 1u);
            S.lq[p] = x;
            S.lqd[p] = nd;
        }
        T.qtail += nl;
        T.budget -= nl;
    }
    const bool spill = imp && !loc;
    const unsigned bs = __ballot_sync(kFull, spill);
    if (bs) {
        if (T.nsp + (uint32_t)__popc(bs) > kSp) ss_flush(A, sn, nxt, tag, S, T, lane, pushes);
        if (spill) {
            const uint32_t p = T.nsp + __popc(bs & lt);
            S.sp[p] = x;
            S.spd[p] = nd;
        }
        T.nsp += __popc(bs);
    }
}

// Expand one wave (<= 32 vertices, one per lane, with their distances): the
// wave's out-arcs laid end to end and dealt 32 per step.
__device__ void ss_wave(const SsArgs &A, SsCount *sn, uint32_t nxt, uint32_t tag, const SsWarp &S,
                        SsTask &T, uint32_t v, unsigned long long d, unsigned long long theta,
                        int lane, unsigned long long &pushes, unsigned long long &exps) {
    uint32_t beg = 0, deg = 0;
    if (v != PG_NONE) {
        beg = __ldg(A.off + v);
        deg = __ldg(A.off + v + 1) - beg;
        exps++;
    }
    uint32_t incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    __syncwarp();
    S.incl[lane] = incl;
    S.base[lane] = beg - (incl - deg);
    S.val[lane] = d;
    __syncwarp();
    for (uint32_t j0 = 0; j0 < total; j0 += 32u) {
        const uint32_t j = j0 + (uint32_t)lane;
        bool imp = false;
        uint32_t x = 0;
        unsigned long long nd = 0;
        if (j < total) {
            uint32_t o = 0;
#pragma unroll
            for (uint32_t step = 16; step >= 1; step >>= 1)
                if (S.incl[o + step - 1] <= j) o += step;
            const uint32_t e = S.base[o] + j;  // u32 sum (the base may wrap)
            x = __ldg(A.idx + e);
            nd = S.val[o] + __ldg(A.w + e);
            imp = nd < atomicMin(A.dist + x, nd);
        }
        ss_route(A, sn, nxt, tag, S, T, imp, x, nd, theta, lane, pushes);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(512, 1) pg_sssp_kernel(const SsArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t n = A.n;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;
    // shared memory per warp: val[32], lqd[qcap], spd[kSp] (u64); incl, base,
    // lq[qcap], sp[kSp] (u32)
    const size_t per_warp = 8u * (32u + A.qcap + kSp) + 4u * (64u + A.qcap + kSp);
    unsigned char *mine = smem + (size_t)wib * per_warp;
    SsWarp S;
    S.val = reinterpret_cast<unsigned long long *>(mine);
    S.lqd = S.val + 32;
    S.spd = S.lqd + A.qcap;
    S.incl = reinterpret_cast<uint32_t *>(S.spd + kSp);
    S.base = S.incl + 32;
    S.lq = S.base + 32;
    S.sp = S.lq + A.qcap;
    PgCtrl *ctrl = A.ctrl;
    unsigned gen = 0;

    for (uint32_t v = gtid; v < n; v += gthreads) A.dist[v] = (v == A.src) ? 0ull : kInf64;
    if (gtid == 0) {
        A.bag[0] = A.src;
        A.cnt[0].size = 1;
        A.cnt[0].min = 0;
        A.cnt[1].min = kInf64;
        A.cnt[2].min = kInf64;
        A.cnt[3].min = kInf64;
    }
    if (A.stall_block == blockIdx.x) return;  // fault injection: never arrive
    if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) return;

    const unsigned long long t_deadline = pg_gtimer() + 16ull * A.timeout_ns;
    unsigned long long pushes = 0, exps = 0;
    uint32_t r = 0;
    for (;; r++) {
        SsCount *sc = &A.cnt[r & 3u];
        SsCount *sn = &A.cnt[(r + 1u) & 3u];
        const uint32_t cur = r & 1u, nxt = cur ^ 1u;
        const uint32_t tag = A.tag0 + r + 1u;
        const uint32_t F = __ldcg(&sc->size);
        const unsigned long long L = pg_ldcg64(&sc->min);
        if (F == 0) break;
        if ((A.max_rounds && r >= A.max_rounds) || F > A.cap || tag == 0u) {
            if (gtid == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        if (gtid == 0) {
            SsCount *cr = &A.cnt[(r + 2u) & 3u];  // neither read nor filled in this round
            cr->size = 0;
            cr->head = 0;
            cr->min = kInf64;
            if (pg_gtimer() > t_deadline) atomicOr(&ctrl->status, PG_DEV_TIMEOUT);
        }
        const unsigned long long theta = (L > kInf64 - A.delta) ? kInf64 : L + A.delta;
        SsTask T;
        T.nsp = 0;
        T.mn = kInf64;
        for (;;) {
            uint32_t b = 0;
            if (lane == 0) b = atomicAdd(&sc->head, 32u);
            b = __shfl_sync(kFull, b, 0);
            if (b >= F) break;
            uint32_t v = PG_NONE;
            unsigned long long d = kInf64;
            if (b + lane < F) {
                v = __ldcg(A.bag + (size_t)cur * A.cap + b + lane);
                d = pg_ldcg64(A.dist + v);
            }
            // entries at or above the threshold wait for a later round
            const bool defer = v != PG_NONE && d >= theta;
            const unsigned bs = __ballot_sync(kFull, defer);
            if (bs) {
                if (T.nsp + (uint32_t)__popc(bs) > kSp) ss_flush(A, sn, nxt, tag, S, T, lane, pushes);
                if (defer) {
                    const uint32_t p = T.nsp + __popc(bs & lanemask_lt());
                    S.sp[p] = v;
                    S.spd[p] = d;
                }
                T.nsp += __popc(bs);
            }
            if (defer) v = PG_NONE;
            T.qhead = T.qtail = 0;
            T.budget = A.budget;
            for (;;) {
                ss_wave(A, sn, nxt, tag, S, T, v, d, theta, lane, pushes, exps);
                const uint32_t avail = T.qtail - T.qhead;
                if (avail == 0) break;
                const uint32_t take = min(32u, avail);
                __syncwarp();
                const uint32_t p = (T.qhead + lane) & (A.qcap - 1u);
                v = ((uint32_t)lane < take) ? S.lq[p] : PG_NONE;
                d = ((uint32_t)lane < take) ? S.lqd[p] : kInf64;
                T.qhead += take;
                __syncwarp();
            }
        }
        ss_flush(A, sn, nxt, tag, S, T, lane, pushes);
        const unsigned long long mn = wmin64(T.mn);
        if (lane == 0 && mn != kInf64) atomicMin(&sn->min, mn);
        if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
    }
    for (int o = 16; o > 0; o >>= 1) {
        exps += __shfl_xor_sync(kFull, exps, o);
        pushes += __shfl_xor_sync(kFull, pushes, o);
    }
    if (lane == 0) {
        if (exps) atomicAdd(&ctrl->expansions, exps);
        if (pushes) atomicAdd(&ctrl->pushes, pushes);
    }
    if (gtid == 0) ctrl->rounds = r;
}

__global__ void k_weight_sum(const uint32_t *w, uint32_t m, unsigned long long *out) {
    unsigned long long s = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) s += w[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

size_t sssp_smem(uint32_t threads, uint32_t qcap) {
    return (size_t)(threads / 32u) * (8u * (32u + qcap + kSp) + 4u * (64u + qcap + kSp));
}

}  // namespace

extern "C" pg_status pg_graph_set_weights(pg_graph *g, const uint32_t *weights, void *stream) {
    if (!g || (!weights && g->m)) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->sssp) {
        PgSsspWork *W = new PgSsspWork();
        memset(W, 0, sizeof(*W));
        cudaError_t e = cudaMalloc(&W->w, (size_t)(g->m ? g->m : 1) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&W->cnt, 4 * sizeof(SsCount) + sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(W->w);
            delete W;
            return pg_cuda_error(e, "cudaMalloc(arc weights)");
        }
        g->sssp = W;
    }
    PgSsspWork &W = *g->sssp;
    if (g->m) {
        const cudaMemcpyKind kind = pg_is_device_ptr(weights) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        PG_CK(cudaMemcpyAsync(W.w, weights, (size_t)g->m * sizeof(uint32_t), kind, s));
    }
    unsigned long long *sum = reinterpret_cast<unsigned long long *>(W.cnt + 4);
    PG_CK(cudaMemsetAsync(sum, 0, sizeof(unsigned long long), s));
    if (g->m) k_weight_sum<<<g->num_sms * 4, 256, 0, s>>>(W.w, g->m, sum);
    PG_CK(cudaGetLastError());
    PG_CK(cudaMemcpyAsync(&W.wsum, sum, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    return PG_OK;
}

extern "C" pg_status pg_sssp(pg_graph *g, uint32_t src, uint64_t *dist_out, const pg_config *cfg,
                             pg_stats *stats, void *stream) {
    if (!g || !dist_out) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (src >= g->n) return pg_set_error(PG_ERR_INVALID_ARG, "src %u >= n %u", src, g->n);
    if (!g->sssp) return pg_set_error(PG_ERR_INVALID_ARG, "pg_sssp: no arc weights (pg_graph_set_weights)");
    pg_config d;
    pg_config_default(&d);
    const pg_config *c = cfg ? cfg : &d;
    if (c->struct_size != sizeof(pg_config)) return pg_set_error(PG_ERR_INVALID_ARG, "pg_config.struct_size mismatch");
    const uint32_t tau = c->tau ? c->tau : 16u;
    if (tau > (1u << 20)) return pg_set_error(PG_ERR_INVALID_ARG, "tau %u too large", tau);
    const uint32_t threads = c->threads_per_block ? c->threads_per_block : 512u;
    if (threads < 64 || threads > 512 || (threads & 31))
        return pg_set_error(PG_ERR_INVALID_ARG, "threads_per_block %u not in 64..512 / multiple of 32", threads);
    const uint32_t qcap = c->local_queue ? c->local_queue : 512u;
    if (qcap < 32 || qcap > 4096 || (qcap & (qcap - 1)))
        return pg_set_error(PG_ERR_INVALID_ARG, "local_queue %u must be a power of two in 32..4096", qcap);
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    PgSsspWork &W = *g->sssp;
    // step width: cfg->delta, else 8 x the mean arc weight
    unsigned long long delta = c->delta;
    if (delta == 0) delta = g->m ? (8ull * W.wsum + g->m - 1) / g->m : 1ull;
    if (delta == 0) delta = 1;
    unsigned long long *out = reinterpret_cast<unsigned long long *>(dist_out);
    const bool host_out = !pg_is_device_ptr(dist_out);
    const size_t bytes = (size_t)g->n * sizeof(unsigned long long);
    if (host_out) {
        void *p = nullptr;
        pg_status st = pg_stage(g, bytes, &p, s);
        if (st) return st;
        out = (unsigned long long *)p;
    }
    if (g->epoch > 0xE0000000u) {
        PG_CK(cudaMemsetAsync(g->d_stamp, 0, (size_t)2 * g->n * sizeof(uint32_t), s));
        g->epoch = 1;
    }
    const size_t smem = sssp_smem(threads, qcap);
    int maxopt = 0;
    PG_CK(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
    if (smem > (size_t)maxopt)
        return pg_set_error(PG_ERR_INVALID_ARG, "pg_sssp: %zu B shared memory > %d (threads %u, local_queue %u)",
                            smem, maxopt, threads, qcap);
    PG_CK(cudaFuncSetAttribute(pg_sssp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pg_sssp_kernel, (int)threads, smem));
    if (per_sm < 1) return pg_set_error(PG_ERR_INVALID_ARG, "pg_sssp launch shape does not fit an SM");
    const uint32_t bps = c->blocks_per_sm ? min((uint32_t)per_sm, c->blocks_per_sm) : (uint32_t)per_sm;
    SsArgs A;
    memset(&A, 0, sizeof(A));
    A.off = g->d_off;
    A.idx = g->d_idx;
    A.w = W.w;
    A.n = g->n;
    A.dist = out;
    A.bag = g->d_bag;
    A.cap = g->bag_cap;
    A.stamp = g->d_stamp;
    A.tag0 = g->epoch;
    A.ctrl = g->d_ctrl;
    A.cnt = W.cnt;
    A.src = src;
    A.delta = delta;
    A.budget = tau * 8u;
    A.qcap = qcap;
    A.timeout_ns = (unsigned long long)(c->timeout_ms ? c->timeout_ms : 5000) * 1000000ull;
    A.max_rounds = c->max_rounds;
    A.stall_block = c->test_stall_block;
    PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
    PG_CK(cudaMemsetAsync(W.cnt, 0, 4 * sizeof(SsCount), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaEventRecord(g->ev0, s));
    PG_CK(cudaLaunchCooperativeKernel((const void *)pg_sssp_kernel, dim3(bps * (uint32_t)g->num_sms),
                                      dim3(threads), args, smem, s));
    PG_CK(cudaEventRecord(g->ev1, s));
    if (host_out) PG_CK(cudaMemcpyAsync(dist_out, out, bytes, cudaMemcpyDeviceToHost, s));
    const size_t off = offsetof(PgCtrl, status);
    PG_CK(cudaMemcpyAsync((char *)g->h_ctrl + off, (const char *)g->d_ctrl + off, sizeof(PgCtrl) - off,
                          cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    const PgCtrl &h = *g->h_ctrl;
    const uint64_t next = (uint64_t)g->epoch + h.rounds + 2;
    g->epoch = next >= 0xE0000000ull ? 0xE0000001u : (uint32_t)next;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->rounds = h.rounds;
        stats->blocks = bps * (uint32_t)g->num_sms;
        stats->threads = threads;
        stats->expansions = h.expansions;
        stats->pushes = h.pushes;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev0, g->ev1) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        stats->kernel_ms = ms;
    }
    if (h.status & PG_DEV_TIMEOUT)
        return pg_set_error(PG_ERR_TIMEOUT, "device wait exceeded %llu ms (SSSP round %u)",
                            A.timeout_ns / 1000000ull, h.rounds);
    if (h.status & PG_DEV_OVERFLOW)
        return pg_set_error(PG_ERR_OVERFLOW, "frontier capacity or round limit exceeded (SSSP round %u)", h.rounds);
    return PG_OK;
}

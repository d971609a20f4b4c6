// pg_scc.cu -- strongly connected components (pg_scc) from reachability
// searches with vertical granularity control.
//
// Sec. 2.1 builds parallel SCC on reachability searches, which need no BFS
// order, and runs each search with VGC: a task keeps expanding locally for a
// bounded number of hops before it hands vertices to the next round.  Here
// the searches follow the forward-backward scheme, for every open subproblem
// at once:
//   * every unfinished vertex carries a part label (a vertex id);
//   * trimming: a vertex with no in-arc or no out-arc from another
//     unfinished vertex of its part is an SCC on its own;
//   * every part picks a pivot (largest hashed priority), and one
//     cooperative launch runs the forward and the backward search of every
//     pivot, each confined to the pivot's part, with a tau-hop local queue
//     per warp;
//   * vertices reached both ways form the pivot's SCC; the others split into
//     three new parts (forward only, backward only, neither).  Two vertices
//     of one SCC are always reached alike, so no part boundary ever cuts an
//     SCC, and every iteration finishes at least every pivot.
// The label of a vertex is the smallest vertex id of its SCC.
#include "pg_internal.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kDir = 0x80000000u;  // bag entry bit: backward search
constexpr int kMaxWarps = 16;

// murmur3's 32-bit finaliser (Appleby, public domain): pivot priorities
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__global__ void k_scc_init(uint32_t n, uint32_t *part, uint32_t *rep) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        part[v] = 0;
        rep[v] = PG_NONE;
    }
}

// true iff some arc of v in this CSR leads to another unfinished vertex of part P
__device__ __forceinline__ bool has_arc_in_part(const uint32_t *off, const uint32_t *idx,
                                                const uint32_t *part, uint32_t v, uint32_t P) {
    const uint32_t b = __ldg(off + v), e = __ldg(off + v + 1);
    for (uint32_t q = b; q < e; q++) {
        const uint32_t w = __ldg(idx + q);
        if (w != v && __ldcg(part + w) == P) return true;
    }
    return false;
}

// One trimming pass.  A vertex finished concurrently by another thread is
// either still seen with its part (v is kept: conservative) or seen finished
// (it is a genuine singleton or in an SCC not containing v), so every trim
// is correct.
__global__ void k_scc_trim(const uint32_t *off, const uint32_t *idx, const uint32_t *toff,
                           const uint32_t *tidx, uint32_t n, uint32_t *part, uint32_t *rep) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t P = __ldcg(part + v);
        if (P == PG_NONE) continue;
        if (has_arc_in_part(off, idx, part, v, P) && has_arc_in_part(toff, tidx, part, v, P)) continue;
        rep[v] = v;
        __stcg(part + v, PG_NONE);
    }
}

// piv[P] = max over unfinished v of part P of (priority(v) << 32 | v)
__global__ void k_scc_pivot(uint32_t n, const uint32_t *part, unsigned long long *piv, uint32_t seed) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t P = part[v];
        if (P == PG_NONE) continue;
        const unsigned long long key = ((unsigned long long)fmix32(v ^ seed) << 32) | v;
        atomicMax(piv + P, key);
    }
}

struct SccArgs {
    const uint32_t *off, *idx, *toff, *tidx;
    uint32_t n;
    const uint32_t *part;
    uint32_t *flag;                   // bit 0: reached forward, bit 1: reached backward
    const unsigned long long *piv;
    uint32_t *bag;                    // [2][cap]
    uint32_t cap;
    PgCtrl *ctrl;
    uint32_t tau, qcap;
    unsigned long long timeout_ns;
};

struct SccWarp {
    uint32_t *s_incl, *s_base, *s_part, *s_ent, *s_hop;  // [32] each
    uint32_t *lq, *lh;                                    // local queue [qcap] entries, hops
};

// Append the lanes' `go` entries to the next bag (one atomic per warp).
__device__ __forceinline__ void scc_push(const SccArgs &A, PgSlot *sn, uint32_t nxt, bool go,
                                         uint32_t ent, int lane) {
    const unsigned bal = __ballot_sync(kFull, go);
    if (!bal) return;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(&sn->size, (unsigned)__popc(bal));
    pos = __shfl_sync(kFull, pos, 0);
    if (go) {
        const uint32_t p = pos + __popc(bal & pg_lanemask_lt());
        if (p < A.cap) A.bag[(size_t)nxt * A.cap + p] = ent;
        else atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
    }
}

// Expand one wave (one entry per lane, hop count h): every arc to an
// unfinished vertex of the same part sets the direction's bit; a vertex
// whose bit was new is searched on, locally while its hop count stays below
// tau and the local queue has room, else in the next round.
__device__ void scc_wave(const SccArgs &A, const SccWarp &S, PgSlot *sn, uint32_t nxt,
                         uint32_t ent, uint32_t hop, int lane, uint32_t &qhead, uint32_t &qtail,
                         unsigned long long &exp) {
    const bool valid = ent != PG_NONE;
    const uint32_t v = ent & ~kDir;
    const uint32_t dir = ent >> 31;
    uint32_t beg = 0, deg = 0, P = PG_NONE;
    if (valid) {
        const uint32_t *o = dir ? A.toff : A.off;
        beg = __ldg(o + v);
        deg = __ldg(o + v + 1) - beg;
        P = __ldg(A.part + v);
        exp++;
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
    S.s_incl[lane] = incl;
    S.s_base[lane] = beg - (incl - deg);  // u32: wraps, and the sum below unwraps
    S.s_part[lane] = P;
    S.s_ent[lane] = dir ? kDir : 0u;
    S.s_hop[lane] = hop;
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32u) {
        const uint32_t j = base + (uint32_t)lane;
        bool imp = false, local = false;
        uint32_t went = 0, wh = 0;
        if (j < total) {
            uint32_t o = 0;
#pragma unroll
            for (uint32_t step = 16; step >= 1; step >>= 1)
                if (S.s_incl[o + step - 1] <= j) o += step;
            const uint32_t d = S.s_ent[o];
            const uint32_t e = S.s_base[o] + j;
            const uint32_t w = __ldg((d ? A.tidx : A.idx) + e);
            const uint32_t pw = __ldg(A.part + w);
            if (pw == S.s_part[o] && pw != PG_NONE) {
                const uint32_t bit = d ? 2u : 1u;
                imp = (atomicOr(A.flag + w, bit) & bit) == 0u;
            }
            went = w | d;
            wh = S.s_hop[o] + 1u;
            local = imp && wh < A.tau;
        }
        // local queue first (ring of qcap), the rest to the next bag
        const unsigned bl = __ballot_sync(kFull, local);
        const uint32_t room = A.qcap - (qtail - qhead);
        const uint32_t rank = __popc(bl & pg_lanemask_lt());
        const bool to_q = local && rank < room;
        if (to_q) {
            const uint32_t p = (qtail + rank) & (A.qcap - 1u);
            S.lq[p] = went;
            S.lh[p] = wh;
        }
        qtail += min((uint32_t)__popc(bl), room);
        scc_push(A, sn, nxt, imp && !to_q, went, lane);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(512, 1) k_scc_reach(const SccArgs A) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t per_warp = 5u * 32u + 2u * A.qcap;
    uint32_t *mine = sm + (size_t)wib * per_warp;
    SccWarp S;
    S.s_incl = mine;
    S.s_base = mine + 32;
    S.s_part = mine + 64;
    S.s_ent = mine + 96;
    S.s_hop = mine + 128;
    S.lq = mine + 160;
    S.lh = S.lq + A.qcap;
    PgCtrl *ctrl = A.ctrl;
    unsigned gen = 0;
    const uint32_t n = A.n;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;

    // seeds: every part's pivot, forward and backward
    for (uint32_t b0 = gtid - (uint32_t)lane; b0 < n; b0 += gthreads) {
        const uint32_t v = b0 + (uint32_t)lane;
        bool piv = false;
        if (v < n) {
            const uint32_t P = __ldg(A.part + v);
            if (P != PG_NONE) {
                piv = (uint32_t)A.piv[P] == v;
                A.flag[v] = piv ? 3u : 0u;
            }
        }
        scc_push(A, &ctrl->slot[0], 0u, piv, v, lane);
        scc_push(A, &ctrl->slot[0], 0u, piv, v | kDir, lane);
    }
    if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) return;

    const unsigned long long t_deadline = pg_gtimer() + 16ull * A.timeout_ns;
    unsigned long long exp = 0;
    uint32_t r = 0;
    for (;; r++) {
        PgSlot *sc = &ctrl->slot[r % PG_NUM_SLOTS];
        PgSlot *sn = &ctrl->slot[(r + 1) % PG_NUM_SLOTS];
        const uint32_t cur = r & 1u, nxt = cur ^ 1u;
        const uint32_t F = __ldcg(&sc->size);
        if (F == 0) break;
        if (F > A.cap) {
            if (gtid == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        if (gtid == 0) {
            PgSlot *sr = &ctrl->slot[(r + 2) % PG_NUM_SLOTS];
            sr->size = 0;
            sr->head = 0;
            if (pg_gtimer() > t_deadline) atomicOr(&ctrl->status, PG_DEV_TIMEOUT);
        }
        for (;;) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&sc->head, 32u);
            base = __shfl_sync(kFull, base, 0);
            if (base >= F) break;
            uint32_t ent = (base + lane < F) ? __ldcg(A.bag + (size_t)cur * A.cap + base + lane) : PG_NONE;
            uint32_t hop = 0;
            uint32_t qhead = 0, qtail = 0;
            for (;;) {
                scc_wave(A, S, sn, nxt, ent, hop, lane, qhead, qtail, exp);
                const uint32_t avail = qtail - qhead;
                if (avail == 0) break;
                const uint32_t take = min(32u, avail);
                __syncwarp();
                const uint32_t p = (qhead + lane) & (A.qcap - 1u);
                ent = ((uint32_t)lane < take) ? S.lq[p] : PG_NONE;
                hop = ((uint32_t)lane < take) ? S.lh[p] : 0u;
                qhead += take;
                __syncwarp();
            }
        }
        if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
    }
    for (int o = 16; o > 0; o >>= 1) exp += __shfl_xor_sync(kFull, exp, o);
    if (lane == 0 && exp) atomicAdd(&ctrl->expansions, exp);
    if (gtid == 0) ctrl->rounds = r;
}

// Finished both ways -> the pivot's SCC; else the vertex joins the new part
// (old part, class), named by its smallest vertex (tbl[3 P + class]).
__global__ void k_scc_split_a(uint32_t n, uint32_t *part, uint32_t *flag,
                              const unsigned long long *piv, uint32_t *rep, uint32_t *tbl) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t P = part[v];
        if (P == PG_NONE) continue;
        const uint32_t f = flag[v] & 3u;
        if (f == 3u) {
            rep[v] = (uint32_t)piv[P];
            part[v] = PG_NONE;
        } else {
            const uint32_t cls = (f & 1u) ? 1u : ((f & 2u) ? 2u : 0u);
            atomicMin(tbl + 3ull * P + cls, v);
            flag[v] = cls;
        }
    }
}

__global__ void k_scc_split_b(uint32_t n, uint32_t *part, const uint32_t *flag, const uint32_t *tbl,
                              unsigned *active) {
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned cnt = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t P = part[v];
        if (P == PG_NONE) continue;
        part[v] = tbl[3ull * P + flag[v]];
        cnt++;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(active, cnt);
}

__global__ void k_scc_min(uint32_t n, const uint32_t *rep, uint32_t *mn) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) atomicMin(mn + rep[v], v);
}

__global__ void k_scc_label(uint32_t n, const uint32_t *rep, const uint32_t *mn, uint32_t *out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = mn[rep[v]];
}

}  // namespace

struct PgSccWork {
    uint32_t *part, *rep, *flag, *tbl;
    unsigned long long *piv;
    unsigned *counter;
};

void pg_scc_release(pg_graph *g) {
    if (g && g->scc) {
        cudaFree(g->scc->part);
        cudaFree(g->scc->piv);
        delete g->scc;
        g->scc = nullptr;
    }
}

static size_t scc_smem(uint32_t threads, uint32_t qcap) {
    return (size_t)(threads / 32u) * (5u * 32u + 2u * qcap) * sizeof(uint32_t);
}

extern "C" pg_status pg_scc(pg_graph *g, uint32_t *label_out, const pg_config *cfg, pg_stats *stats,
                            uint32_t *iterations, void *stream) {
    if (!g || !label_out) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (!g->has_transpose)
        return pg_set_error(PG_ERR_UNSUPPORTED, "pg_scc needs the transpose (PG_BUILD_TRANSPOSE)");
    pg_config d;
    pg_config_default(&d);
    const pg_config *c = cfg ? cfg : &d;
    if (c->struct_size != sizeof(pg_config)) return pg_set_error(PG_ERR_INVALID_ARG, "pg_config.struct_size mismatch");
    const uint32_t tau = c->tau ? c->tau : 16u;
    const uint32_t threads = c->threads_per_block ? c->threads_per_block : 512u;
    const uint32_t qcap = c->local_queue ? c->local_queue : 512u;
    if (threads < 64 || threads > 32u * kMaxWarps || (threads & 31))
        return pg_set_error(PG_ERR_INVALID_ARG, "threads_per_block %u not in 64..512 / multiple of 32", threads);
    if (qcap < 32 || qcap > 4096 || (qcap & (qcap - 1)))
        return pg_set_error(PG_ERR_INVALID_ARG, "local_queue %u must be a power of two in 32..4096", qcap);
    if (tau > (1u << 20)) return pg_set_error(PG_ERR_INVALID_ARG, "tau %u too large", tau);
    const unsigned long long timeout_ns = (unsigned long long)(c->timeout_ms ? c->timeout_ms : 5000) * 1000000ull;
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = g->n;
    if (!g->scc) {
        PgSccWork *W = new PgSccWork();
        memset(W, 0, sizeof(*W));
        uint32_t *p = nullptr;
        cudaError_t e = cudaMalloc(&p, ((size_t)6 * n + 8) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&W->piv, (size_t)n * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(p);
            delete W;
            return pg_cuda_error(e, "cudaMalloc(SCC workspace)");
        }
        W->part = p;
        W->rep = p + n;
        W->flag = p + 2 * (size_t)n;
        W->tbl = p + 3 * (size_t)n;               // 3n group minima
        W->counter = p + 6 * (size_t)n;
        g->scc = W;
    }
    PgSccWork &W = *g->scc;
    uint32_t *out = label_out;
    const bool host_out = !pg_is_device_ptr(label_out);
    if (host_out) {
        void *p = nullptr;
        pg_status st = pg_stage(g, (size_t)n * sizeof(uint32_t), &p);
        if (st) return st;
        out = (uint32_t *)p;
    }
    const size_t smem = scc_smem(threads, qcap);
    PG_CK(cudaFuncSetAttribute(k_scc_reach, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scc_reach, threads, smem));
    if (per_sm < 1) return pg_set_error(PG_ERR_INVALID_ARG, "SCC search does not fit an SM (threads %u, queue %u)", threads, qcap);
    const uint32_t blocks = (uint32_t)g->num_sms;  // one CTA per SM
    const int grid = g->num_sms * 4;

    SccArgs A;
    memset(&A, 0, sizeof(A));
    A.off = g->d_off;
    A.idx = g->d_idx;
    A.toff = g->d_toff;
    A.tidx = g->d_tidx;
    A.n = n;
    A.part = W.part;
    A.flag = W.flag;
    A.piv = W.piv;
    A.bag = g->d_bag;
    A.cap = g->bag_cap;
    A.ctrl = g->d_ctrl;
    A.tau = tau;
    A.qcap = qcap;
    A.timeout_ns = timeout_ns;

    PG_CK(cudaEventRecord(g->ev0, s));
    k_scc_init<<<grid, 256, 0, s>>>(n, W.part, W.rep);
    PG_CK(cudaGetLastError());
    uint32_t iter = 0, rounds = 0;
    unsigned long long expansions = 0;
    const uint32_t max_iter = n + 1;
    for (;; iter++) {
        if (iter >= max_iter) return pg_set_error(PG_ERR_OVERFLOW, "SCC did not finish in %u iterations", max_iter);
        for (int t = 0; t < 2; t++)
            k_scc_trim<<<grid, 256, 0, s>>>(g->d_off, g->d_idx, g->d_toff, g->d_tidx, n, W.part, W.rep);
        PG_CK(cudaMemsetAsync(W.piv, 0, (size_t)n * sizeof(unsigned long long), s));
        k_scc_pivot<<<grid, 256, 0, s>>>(n, W.part, W.piv, c->seed * 0x9E3779B9u + iter);
        PG_CK(cudaGetLastError());
        PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
        void *args[] = {(void *)&A};
        PG_CK(cudaLaunchCooperativeKernel((const void *)k_scc_reach, dim3(blocks), dim3(threads), args, smem, s));
        PG_CK(cudaMemsetAsync(W.tbl, 0xFF, (size_t)3 * n * sizeof(uint32_t), s));
        PG_CK(cudaMemsetAsync(W.counter, 0, sizeof(unsigned), s));
        k_scc_split_a<<<grid, 256, 0, s>>>(n, W.part, W.flag, W.piv, W.rep, W.tbl);
        k_scc_split_b<<<grid, 256, 0, s>>>(n, W.part, W.flag, W.tbl, W.counter);
        PG_CK(cudaGetLastError());
        // status of the search and the number of unfinished vertices
        const size_t off = offsetof(PgCtrl, status);
        PG_CK(cudaMemcpyAsync((char *)g->h_ctrl + off, (const char *)g->d_ctrl + off, sizeof(PgCtrl) - off,
                              cudaMemcpyDeviceToHost, s));
        unsigned active = 0;
        PG_CK(cudaMemcpyAsync(&active, W.counter, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        PG_CK(cudaStreamSynchronize(s));
        const PgCtrl &h = *g->h_ctrl;
        rounds += h.rounds;
        expansions += h.expansions;
        if (h.status & PG_DEV_TIMEOUT)
            return pg_set_error(PG_ERR_TIMEOUT, "device wait exceeded %llu ms (SCC iteration %u)",
                                timeout_ns / 1000000ull, iter);
        if (h.status & PG_DEV_OVERFLOW)
            return pg_set_error(PG_ERR_OVERFLOW, "frontier capacity exceeded (SCC iteration %u)", iter);
        if (active == 0) break;
    }
    PG_CK(cudaMemsetAsync(W.tbl, 0xFF, (size_t)n * sizeof(uint32_t), s));
    k_scc_min<<<grid, 256, 0, s>>>(n, W.rep, W.tbl);
    k_scc_label<<<grid, 256, 0, s>>>(n, W.rep, W.tbl, out);
    PG_CK(cudaGetLastError());
    PG_CK(cudaEventRecord(g->ev1, s));
    if (host_out) PG_CK(cudaMemcpyAsync(label_out, out, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    if (iterations) *iterations = iter + 1;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->rounds = rounds;
        stats->blocks = blocks;
        stats->threads = threads;
        stats->expansions = expansions;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev0, g->ev1) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        stats->kernel_ms = ms;
    }
    return PG_OK;
}

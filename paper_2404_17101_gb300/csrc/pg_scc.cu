// pg_scc.cu -- strongly connected components (pg_scc) from reachability
// searches with vertical granularity control.
//
// Sec. 2.1 builds parallel SCC on reachability searches, which need no BFS
// order, and runs each search with VGC: a task keeps expanding locally for a
// bounded number of hops before it hands vertices to the next round.  Here
// the searches decompose every open part of the graph at once (colouring):
//   * every unfinished vertex carries a part label (a vertex id);
//   * trimming: a vertex with no in-arc or no out-arc from another
//     unfinished vertex of its part is an SCC on its own;
//   * colouring: every vertex of a part gets a random key (priority << 32 |
//     id), and a forward search propagates the largest key along the arcs
//     inside the part (atomicMax, label-correcting to a fixpoint); a vertex
//     ends with the largest key among the vertices that reach it;
//   * a vertex whose final key is its own is a root; a backward search from
//     every root, confined to the vertices of its colour, finds exactly the
//     root's SCC (they reach the root, and the root reaches them because its
//     key flowed to them);
//   * the rest take their colour's root as their new part: the vertices of
//     one SCC have the same ancestors, hence the same colour, so no part
//     boundary ever cuts an SCC.  Every part holds at least one root (its
//     largest key), so every iteration finishes vertices.
// Both searches run in one persistent cooperative kernel each, with a
// tau-hop local queue per warp and round tags that keep each vertex at most
// once per bag.  The label of a vertex is the smallest vertex id of its SCC.
#include "pg_internal.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kMaxWarps = 16;

// murmur3's 32-bit finaliser (Appleby, public domain): vertex priorities
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ unsigned long long scc_key(uint32_t v, uint32_t seed) {
    return ((unsigned long long)fmix32(v ^ seed) << 32) | v;
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

__global__ void k_scc_color_init(uint32_t n, const uint32_t *part, unsigned long long *col, uint32_t seed) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (part[v] != PG_NONE) col[v] = scc_key(v, seed);
}

// roots: the vertices whose final colour is their own key
__global__ void k_scc_roots(uint32_t n, const uint32_t *part, const unsigned long long *col,
                            uint32_t *flag, uint32_t seed) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (part[v] != PG_NONE) flag[v] = (col[v] == scc_key(v, seed)) ? 1u : 0u;
}

struct SccArgs {
    const uint32_t *off, *idx, *toff, *tidx;
    uint32_t n;
    const uint32_t *part;
    unsigned long long *col;          // colour (largest key reaching the vertex)
    uint32_t *flag;                   // 1: in its root's SCC (backward search)
    uint32_t *stamp;                  // round tags: one bag entry per vertex and round
    uint32_t tag0;
    uint32_t *bag;                    // [2][cap]
    uint32_t cap;
    PgCtrl *ctrl;
    uint32_t tau, qcap;
    unsigned long long timeout_ns;
    uint32_t stall_block;             // fault injection: this CTA never arrives at the grid barrier
};

struct SccWarp {
    uint32_t *s_incl, *s_base, *s_part, *s_hop;  // [32] each
    unsigned long long *s_col;                   // [32]
    uint32_t *lq, *lh;                           // local queue [qcap]: vertex, hops
};

// Append the lanes' `go` vertices to the next bag (one atomic per warp);
// `dedupe`: a vertex already appended in this round is skipped.
__device__ __forceinline__ void scc_push(const SccArgs &A, PgSlot *sn, uint32_t nxt, uint32_t tag,
                                         bool go, bool dedupe, uint32_t v, int lane) {
    if (go && dedupe) go = atomicExch(A.stamp + v, tag) != tag;
    const unsigned bal = __ballot_sync(kFull, go);
    if (!bal) return;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(&sn->size, (unsigned)__popc(bal));
    pos = __shfl_sync(kFull, pos, 0);
    if (go) {
        const uint32_t p = pos + __popc(bal & pg_lanemask_lt());
        if (p < A.cap) A.bag[(size_t)nxt * A.cap + p] = v;
        else atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
    }
}

// Expand one wave (one vertex per lane, hop count h).
//  kColor: forward arcs inside the part carry the vertex's current colour
//          (atomicMax); a raised colour is searched on.
//  else:   backward arcs to unfinished vertices of the same colour set the
//          SCC flag; a newly flagged vertex is searched on.
// Searched-on vertices stay in the warp's local queue while their hop count
// is below tau and it has room, else they go to the next round's bag.
template <bool kColor>
__device__ void scc_wave(const SccArgs &A, const SccWarp &S, PgSlot *sn, uint32_t nxt, uint32_t tag,
                         uint32_t v, uint32_t hop, int lane, uint32_t &qhead, uint32_t &qtail,
                         unsigned long long &exp) {
    const bool valid = v != PG_NONE;
    const uint32_t *off = kColor ? A.off : A.toff;
    const uint32_t *idx = kColor ? A.idx : A.tidx;
    uint32_t beg = 0, deg = 0, P = PG_NONE;
    unsigned long long c = 0;
    if (valid) {
        beg = __ldg(off + v);
        deg = __ldg(off + v + 1) - beg;
        P = __ldg(A.part + v);
        c = __ldcg(A.col + v);
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
    S.s_hop[lane] = hop;
    S.s_col[lane] = c;
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32u) {
        const uint32_t j = base + (uint32_t)lane;
        bool imp = false, local = false;
        uint32_t w = 0, wh = 0;
        if (j < total) {
            uint32_t o = 0;
#pragma unroll
            for (uint32_t step = 16; step >= 1; step >>= 1)
                if (S.s_incl[o + step - 1] <= j) o += step;
            const uint32_t e = S.s_base[o] + j;
            w = __ldg(idx + e);
            const uint32_t pw = __ldg(A.part + w);
            const unsigned long long co = S.s_col[o];
            if (pw == S.s_part[o] && pw != PG_NONE) {
                if (kColor) {
                    imp = atomicMax(A.col + w, co) < co;
                } else if (__ldcg(A.col + w) == co) {
                    imp = (atomicOr(A.flag + w, 1u) & 1u) == 0u;
                }
            }
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
            S.lq[p] = w;
            S.lh[p] = wh;
        }
        qtail += min((uint32_t)__popc(bl), room);
        scc_push(A, sn, nxt, tag, imp && !to_q, kColor, w, lane);
    }
    __syncwarp();
}

// One search to its fixpoint.  Seeds: kColor, every unfinished vertex;
// else every root (flag == 1).
template <bool kColor>
__global__ void __launch_bounds__(512, 1) k_scc_search(const SccArgs A) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t per_warp = 6u * 32u + 2u * A.qcap;
    uint32_t *mine = sm + (size_t)wib * per_warp;
    SccWarp S;
    S.s_col = reinterpret_cast<unsigned long long *>(mine);  // 64 words, 8-byte aligned
    S.s_incl = mine + 64;
    S.s_base = mine + 96;
    S.s_part = mine + 128;
    S.s_hop = mine + 160;
    S.lq = mine + 192;
    S.lh = S.lq + A.qcap;
    PgCtrl *ctrl = A.ctrl;
    unsigned gen = 0;
    const uint32_t n = A.n;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;

    for (uint32_t b0 = gtid - (uint32_t)lane; b0 < n; b0 += gthreads) {
        const uint32_t v = b0 + (uint32_t)lane;
        bool seed = false;
        if (v < n && __ldg(A.part + v) != PG_NONE) seed = kColor ? true : (A.flag[v] == 1u);
        scc_push(A, &ctrl->slot[0], 0u, 0u, seed, false, v, lane);
    }
    if (A.stall_block == blockIdx.x) return;  // fault injection: never arrive
    if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) return;

    const unsigned long long t_deadline = pg_gtimer() + 16ull * A.timeout_ns;
    unsigned long long exp = 0;
    uint32_t r = 0;
    for (;; r++) {
        PgSlot *sc = &ctrl->slot[r % PG_NUM_SLOTS];
        PgSlot *sn = &ctrl->slot[(r + 1) % PG_NUM_SLOTS];
        const uint32_t cur = r & 1u, nxt = cur ^ 1u;
        const uint32_t tag = A.tag0 + r + 1u;
        const uint32_t F = __ldcg(&sc->size);
        if (F == 0) break;
        if (F > A.cap || tag == 0u) {
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
            uint32_t v = (base + lane < F) ? __ldcg(A.bag + (size_t)cur * A.cap + base + lane) : PG_NONE;
            uint32_t hop = 0;
            uint32_t qhead = 0, qtail = 0;
            for (;;) {
                scc_wave<kColor>(A, S, sn, nxt, tag, v, hop, lane, qhead, qtail, exp);
                const uint32_t avail = qtail - qhead;
                if (avail == 0) break;
                const uint32_t take = min(32u, avail);
                __syncwarp();
                const uint32_t p = (qhead + lane) & (A.qcap - 1u);
                v = ((uint32_t)lane < take) ? S.lq[p] : PG_NONE;
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

// Flagged -> finished in its root's SCC; else the colour's root names the
// vertex's new part.  Counts the unfinished vertices.
__global__ void k_scc_assign(uint32_t n, uint32_t *part, const unsigned long long *col,
                             const uint32_t *flag, uint32_t *rep, unsigned *active) {
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned cnt = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (part[v] == PG_NONE) continue;
        const uint32_t root = (uint32_t)col[v];
        if (flag[v] == 1u) {
            rep[v] = root;
            part[v] = PG_NONE;
        } else {
            part[v] = root;
            cnt++;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(active, cnt);
}

// mn[rep] = smallest vertex of each SCC.  Threads visit vertices in rising
// id order, so a component's minimum is found early and almost every later
// member sees a smaller value and skips the atomic: one giant component
// would otherwise serialise millions of same-address atomics.
__global__ void k_scc_min(uint32_t n, const uint32_t *rep, uint32_t *mn) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t r = rep[v];
        if (__ldcg(mn + r) > v) atomicMin(mn + r, v);
    }
}

__global__ void k_scc_label(uint32_t n, const uint32_t *rep, const uint32_t *mn, uint32_t *out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) out[v] = mn[rep[v]];
}

}  // namespace

struct PgSccWork {
    uint32_t *part, *rep, *flag, *mn;
    unsigned long long *col;
    unsigned *counter;
};

void pg_scc_release(pg_graph *g) {
    if (g && g->scc) {
        cudaFree(g->scc->part);
        cudaFree(g->scc->col);
        delete g->scc;
        g->scc = nullptr;
    }
}

static size_t scc_smem(uint32_t threads, uint32_t qcap) {
    return (size_t)(threads / 32u) * (6u * 32u + 2u * qcap) * sizeof(uint32_t);
}

template <bool kColor>
static pg_status scc_search(pg_graph *g, SccArgs &A, uint32_t threads, size_t smem, cudaStream_t s,
                            uint32_t *rounds, unsigned long long *expansions) {
    // round tags of this launch: epoch + r + 1; restart the tags before they wrap
    if (g->epoch > 0xE0000000u) {
        PG_CK(cudaMemsetAsync(g->d_stamp, 0, (size_t)2 * g->n * sizeof(uint32_t), s));
        g->epoch = 1;
    }
    A.tag0 = g->epoch;
    PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaLaunchCooperativeKernel((const void *)k_scc_search<kColor>, dim3((uint32_t)g->num_sms),
                                      dim3(threads), args, smem, s));
    const size_t off = offsetof(PgCtrl, status);
    PG_CK(cudaMemcpyAsync((char *)g->h_ctrl + off, (const char *)g->d_ctrl + off, sizeof(PgCtrl) - off,
                          cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    const PgCtrl &h = *g->h_ctrl;
    g->epoch += h.rounds + 2u;
    *rounds += h.rounds;
    *expansions += h.expansions;
    if (h.status & PG_DEV_TIMEOUT)
        return pg_set_error(PG_ERR_TIMEOUT, "device wait exceeded %llu ms (SCC search)", A.timeout_ns / 1000000ull);
    if (h.status & PG_DEV_OVERFLOW) return pg_set_error(PG_ERR_OVERFLOW, "frontier capacity exceeded (SCC search)");
    return PG_OK;
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
        cudaError_t e = cudaMalloc(&p, ((size_t)4 * n + 8) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&W->col, (size_t)n * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            cudaFree(p);
            delete W;
            return pg_cuda_error(e, "cudaMalloc(SCC workspace)");
        }
        W->part = p;
        W->rep = p + n;
        W->flag = p + 2 * (size_t)n;
        W->mn = p + 3 * (size_t)n;
        W->counter = p + 4 * (size_t)n;
        g->scc = W;
    }
    PgSccWork &W = *g->scc;
    uint32_t *out = label_out;
    const bool host_out = !pg_is_device_ptr(label_out);
    if (host_out) {
        void *p = nullptr;
        pg_status st = pg_stage(g, (size_t)n * sizeof(uint32_t), &p, s);
        if (st) return st;
        out = (uint32_t *)p;
    }
    const size_t smem = scc_smem(threads, qcap);
    for (int k = 0; k < 2; k++) {
        const void *kern = k ? (const void *)k_scc_search<true> : (const void *)k_scc_search<false>;
        PG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        if (per_sm < 1)
            return pg_set_error(PG_ERR_INVALID_ARG, "SCC search does not fit an SM (threads %u, queue %u)", threads, qcap);
    }
    const int grid = g->num_sms * 4;

    SccArgs A;
    memset(&A, 0, sizeof(A));
    A.off = g->d_off;
    A.idx = g->d_idx;
    A.toff = g->d_toff;
    A.tidx = g->d_tidx;
    A.n = n;
    A.part = W.part;
    A.col = W.col;
    A.flag = W.flag;
    A.stamp = g->d_stamp;
    A.bag = g->d_bag;
    A.cap = g->bag_cap;
    A.ctrl = g->d_ctrl;
    A.tau = tau;
    A.qcap = qcap;
    A.timeout_ns = timeout_ns;
    A.stall_block = c->test_stall_block;

    PG_CK(cudaEventRecord(g->ev0, s));
    k_scc_init<<<grid, 256, 0, s>>>(n, W.part, W.rep);
    PG_CK(cudaGetLastError());
    uint32_t iter = 0, rounds = 0;
    unsigned long long expansions = 0;
    for (;; iter++) {
        if (iter > n) return pg_set_error(PG_ERR_OVERFLOW, "SCC did not finish in %u iterations", n + 1);
        const uint32_t seed = (c->seed + 1u) * 0x9E3779B9u + iter * 0x85EBCA6Bu;
        k_scc_trim<<<grid, 256, 0, s>>>(g->d_off, g->d_idx, g->d_toff, g->d_tidx, n, W.part, W.rep);
        k_scc_color_init<<<grid, 256, 0, s>>>(n, W.part, W.col, seed);
        PG_CK(cudaGetLastError());
        pg_status st = scc_search<true>(g, A, threads, smem, s, &rounds, &expansions);
        if (st) return st;
        k_scc_roots<<<grid, 256, 0, s>>>(n, W.part, W.col, W.flag, seed);
        PG_CK(cudaGetLastError());
        st = scc_search<false>(g, A, threads, smem, s, &rounds, &expansions);
        if (st) return st;
        PG_CK(cudaMemsetAsync(W.counter, 0, sizeof(unsigned), s));
        k_scc_assign<<<grid, 256, 0, s>>>(n, W.part, W.col, W.flag, W.rep, W.counter);
        PG_CK(cudaGetLastError());
        unsigned active = 0;
        PG_CK(cudaMemcpyAsync(&active, W.counter, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        PG_CK(cudaStreamSynchronize(s));
        if (active == 0) break;
    }
    PG_CK(cudaMemsetAsync(W.mn, 0xFF, (size_t)n * sizeof(uint32_t), s));
    k_scc_min<<<grid, 256, 0, s>>>(n, W.rep, W.mn);
    k_scc_label<<<grid, 256, 0, s>>>(n, W.rep, W.mn, out);
    PG_CK(cudaGetLastError());
    PG_CK(cudaEventRecord(g->ev1, s));
    if (host_out) PG_CK(cudaMemcpyAsync(label_out, out, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    if (iterations) *iterations = iter + 1;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->rounds = rounds;
        stats->blocks = (uint32_t)g->num_sms;
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

// pg_msbfs.cu -- batched BFS from up to 64 sources (pg_bfs_multi).
//
// All k searches share every round of Algorithm 1: a vertex carries one bit
// per source in three uint64 words (seen, visit = reached in the last
// round, next).  A round is either top-down (each vertex with visit != 0
// ORs its bits into its out-neighbours' next) or bottom-up (each vertex
// still missing bits ORs the visit words of its in-neighbours, stopping as
// soon as every missing bit is found), chosen with the direction-
// optimisation test of [Beamer12] (Sec. 2.2).  A bit that first appears at a
// vertex in round L gives that source's hop distance L + 1 (Sec. 2.2).
//
// High-degree splitting (the load balance of Sec. 2.1's small-task
// discussion): a vertex with at least kHeavy edges in a direction is never
// expanded by one thread or one warp alone.  Its list is cut into chunks of
// at most kChunk edges, listed once per graph, and any warp takes a chunk:
// top-down ORs the vertex's bits into the chunk's targets, bottom-up ORs the
// chunk's visit words (32 at a time, stopping once every missing bit is
// found) and merges them into next[w] with one atomicOr.
#include "pg_internal.cuh"

namespace {
constexpr uint32_t kHeavy = 32;    // edges: below, one thread (bottom-up) / one lane (top-down)
constexpr uint32_t kChunk = 1024;  // edges per chunk of a heavy vertex
constexpr uint32_t kGather = 8;    // bottom-up: in-neighbour gathers in flight per light vertex
}  // namespace

struct PgMsbfsWork {
    unsigned long long *seen, *visit, *next;
    uint32_t n;
    uint2 *chunks[2];     // (vertex, first edge) per chunk: out-lists, in-lists
    uint32_t nchunks[2];
};

void pg_msbfs_release(pg_graph *g) {
    if (g && g->msbfs) {
        cudaFree(g->msbfs->seen);
        cudaFree(g->msbfs->chunks[0]);
        if (g->msbfs->chunks[1] != g->msbfs->chunks[0]) cudaFree(g->msbfs->chunks[1]);
        delete g->msbfs;
        g->msbfs = nullptr;
    }
}

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// chunks of each heavy vertex: cnt[v] = ceil(deg / kChunk) when deg >= kHeavy
__global__ void k_chunk_count(const uint32_t *off, uint32_t n, uint32_t *cnt) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        uint32_t c = 0;
        if (v < n) {
            const uint32_t d = off[v + 1] - off[v];
            c = d >= kHeavy ? (d + kChunk - 1) / kChunk : 0u;
        }
        cnt[v] = c;
    }
}

__global__ void k_chunk_fill(const uint32_t *off, uint32_t n, const uint32_t *pos, uint2 *chunks) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t b = off[v], d = off[v + 1] - b;
        if (d < kHeavy) continue;
        const uint32_t c = (d + kChunk - 1) / kChunk;
        for (uint32_t i = 0; i < c; i++) chunks[pos[v] + i] = make_uint2(v, b + i * kChunk);
    }
}

struct MsArgs {
    PgGraphDev G;
    const uint2 *chunks_out, *chunks_in;
    uint32_t nchunks_out, nchunks_in;
    PgCtrl *ctrl;
    unsigned long long *seen, *visit, *next;
    uint32_t *dist;       // k * n, source-major
    uint32_t k;
    uint32_t sources[64];
    uint32_t alpha, beta, allow_pull, direction;
    unsigned long long timeout_ns;
    uint32_t max_rounds, stall_block;
};

__device__ __forceinline__ unsigned long long wsum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__global__ void __launch_bounds__(512) pg_msbfs_kernel(const MsArgs A) {
    __shared__ int s_flag;
    __shared__ uint32_t s_incl[16][32];
    __shared__ uint32_t s_base[16][32];
    __shared__ unsigned long long s_bits[16][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t n = A.G.n, k = A.k;
    const unsigned long long full = (k == 64) ? ~0ull : ((1ull << k) - 1ull);
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;
    const uint32_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
    PgCtrl *ctrl = A.ctrl;
    unsigned gen = 0;

    // init: sources at distance 0
    unsigned long long fv = 0, fe = 0;
    for (uint32_t v = gtid; v < n; v += gthreads) {
        unsigned long long b = 0;
        for (uint32_t j = 0; j < k; j++)
            if (A.sources[j] == v) b |= 1ull << j;
        A.seen[v] = b;
        A.visit[v] = b;
        A.next[v] = 0;
        for (uint32_t j = 0; j < k; j++)
            if ((b >> j) & 1ull) A.dist[(size_t)j * n + v] = 0;
        if (b) { fv++; fe += A.G.off[v + 1] - A.G.off[v]; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int s = 0; s < PG_NUM_SLOTS; s++) {
            ctrl->slot[s].size = 0;
            ctrl->slot[s].out_edges = 0;
        }
    if (A.stall_block == blockIdx.x) return;
    if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) return;
    fv = wsum(fv);
    fe = wsum(fe);
    if (lane == 0 && fv) {
        atomicAdd(&ctrl->slot[0].size, (unsigned)fv);
        atomicAdd(&ctrl->slot[0].out_edges, fe);
    }
    if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) return;

    unsigned long long edges_seen = 0;
    const unsigned long long t_deadline = pg_gtimer() + 16ull * A.timeout_ns;
    bool bottom_up = false;
    uint32_t L = 0, pulls = 0;
    for (;; L++) {
        PgSlot *sc = &ctrl->slot[L % PG_NUM_SLOTS];
        PgSlot *sn = &ctrl->slot[(L + 1) % PG_NUM_SLOTS];
        const uint32_t F = __ldcg(&sc->size);
        const unsigned long long E = pg_ldcg64(&sc->out_edges);
        if (F == 0) break;
        if (A.max_rounds && L >= A.max_rounds) {
            if (gtid == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        if (gtid == 0) {
            PgSlot *sr = &ctrl->slot[(L + 2) % PG_NUM_SLOTS];
            sr->size = 0;
            sr->out_edges = 0;
            if (pg_gtimer() > t_deadline) atomicOr(&ctrl->status, PG_DEV_TIMEOUT);
        }
        if (A.allow_pull && A.direction == PG_DIR_AUTO) {
            const unsigned long long unexplored =
                (unsigned long long)A.G.m > edges_seen ? A.G.m - edges_seen : 0ull;
            if (!bottom_up) {
                if (E > unexplored / A.alpha) bottom_up = true;
            } else if ((unsigned long long)F < (unsigned long long)n / A.beta) {
                bottom_up = false;
            }
        } else {
            bottom_up = false;
        }
        edges_seen += E;
        if (bottom_up) {
            pulls++;
            // light vertices: one thread each, kGather gathers in flight
            for (uint32_t w = gtid; w < n; w += gthreads) {
                const unsigned long long need = full & ~A.seen[w];
                if (!need) continue;
                const uint32_t b = __ldg(A.G.toff + w), e = __ldg(A.G.toff + w + 1);
                if (e - b >= kHeavy) continue;  // in the chunk list
                unsigned long long acc = 0;
                for (uint32_t q = b; q < e; q += kGather) {
                    uint32_t u[kGather];
#pragma unroll
                    for (int i = 0; i < (int)kGather; i++) u[i] = (q + i < e) ? __ldg(A.G.tidx + q + i) : PG_NONE;
#pragma unroll
                    for (int i = 0; i < (int)kGather; i++)
                        if (u[i] != PG_NONE) acc |= __ldcg(A.visit + u[i]);
                    if ((acc & need) == need) break;
                }
                if (acc & need) A.next[w] = acc & need;
            }
            // heavy vertices: one warp per chunk of in-edges
            for (uint32_t c = gwarp; c < A.nchunks_in; c += nwarps) {
                const uint2 ch = A.chunks_in[c];
                const uint32_t w = ch.x;
                const unsigned long long need = full & ~__ldcg(A.seen + w);
                if (!need) continue;
                const uint32_t e = min(ch.y + kChunk, __ldg(A.G.toff + w + 1));
                unsigned long long acc = 0;
                for (uint32_t q = ch.y; q < e; q += 32u) {
                    if (q + lane < e) acc |= __ldcg(A.visit + __ldg(A.G.tidx + q + lane));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(kFull, acc, o);
                    if ((acc & need) == need) break;
                }
                if (lane == 0 && (acc & need)) atomicOr(A.next + w, acc & need);
            }
        } else {
            // top-down: warps take 32 consecutive vertices, expand the
            // active ones' edges cooperatively (32 edges per step)
            for (uint32_t base = gwarp * 32u; base < n; base += nwarps * 32u) {
                const uint32_t v = base + lane;
                unsigned long long bits = 0;
                uint32_t beg = 0, deg = 0;
                if (v < n) {
                    bits = __ldcg(A.visit + v);
                    if (bits) {
                        beg = __ldg(A.G.off + v);
                        deg = __ldg(A.G.off + v + 1) - beg;
                        if (deg >= kHeavy) deg = 0;  // in the chunk list
                    }
                }
                uint32_t incl = deg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t total = __shfl_sync(kFull, incl, 31);
                if (total == 0) continue;
                s_incl[wib][lane] = incl;
                s_base[wib][lane] = beg - (incl - deg);
                s_bits[wib][lane] = bits;
                __syncwarp();
                for (uint32_t j = lane; j < total; j += 32) {
                    uint32_t o = 0;
#pragma unroll
                    for (uint32_t step = 16; step >= 1; step >>= 1)
                        if (s_incl[wib][o + step - 1] <= j) o += step;
                    const uint32_t e = s_base[wib][o] + j;  // u32 sum (the base may wrap)
                    const uint32_t w = __ldg(A.G.idx + e);
                    atomicOr(A.next + w, s_bits[wib][o]);
                }
                __syncwarp();
            }
            // heavy frontier vertices: one warp per chunk of out-edges
            for (uint32_t c = gwarp; c < A.nchunks_out; c += nwarps) {
                const uint2 ch = A.chunks_out[c];
                const unsigned long long bits = __ldcg(A.visit + ch.x);
                if (!bits) continue;
                const uint32_t e = min(ch.y + kChunk, __ldg(A.G.off + ch.x + 1));
                for (uint32_t q = ch.y + lane; q < e; q += 32u) atomicOr(A.next + __ldg(A.G.idx + q), bits);
            }
        }
        if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
        // update: new bits -> distances, next frontier statistics
        unsigned long long nv = 0, ne = 0;
        for (uint32_t b0 = gwarp * 32u; b0 < n; b0 += nwarps * 32u) {
            const uint32_t v = b0 + lane;
            unsigned long long nb = 0;
            if (v < n) {
                const unsigned long long nx = __ldcg(A.next + v);
                const unsigned long long sn_ = A.seen[v];
                nb = nx & ~sn_ & full;
                if (nx) A.next[v] = 0;
                if (A.visit[v] != nb) A.visit[v] = nb;
                if (nb) {
                    A.seen[v] = sn_ | nb;
                    nv++;
                    ne += __ldg(A.G.off + v + 1) - __ldg(A.G.off + v);
                }
            }
            if (__any_sync(kFull, nb != 0)) {
                for (uint32_t j = 0; j < k; j++)
                    if ((nb >> j) & 1ull) A.dist[(size_t)j * n + v] = L + 1;
            }
        }
        nv = wsum(nv);
        ne = wsum(ne);
        if (lane == 0 && nv) {
            atomicAdd(&sn->size, (unsigned)nv);
            atomicAdd(&sn->out_edges, ne);
        }
        if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
    }
    // sources never reached: 0xFFFFFFFF
    if (pg_ld_volatile(&ctrl->status) == 0u) {
        for (uint32_t b0 = gwarp * 32u; b0 < n; b0 += nwarps * 32u) {
            const uint32_t v = b0 + lane;
            const unsigned long long miss = (v < n) ? (full & ~A.seen[v]) : 0ull;
            if (__any_sync(kFull, miss != 0)) {
                for (uint32_t j = 0; j < k; j++)
                    if ((miss >> j) & 1ull) A.dist[(size_t)j * n + v] = PG_INF;
            }
        }
    }
    if (gtid == 0) {
        ctrl->rounds = L;
        ctrl->pull_rounds = pulls;
    }
}

}  // namespace

// The chunk list of one direction (built once per graph, on first use).
static pg_status build_chunks(pg_graph *g, const uint32_t *off, uint2 **out, uint32_t *count,
                              cudaStream_t s) {
    const uint32_t n = g->n;
    *out = nullptr;
    *count = 0;
    uint32_t *cnt = nullptr;
    PG_CK(cudaMallocAsync(&cnt, ((size_t)n + 1) * 2 * sizeof(uint32_t), s));
    uint32_t *pos = cnt + n + 1;
    k_chunk_count<<<g->num_sms * 4, 256, 0, s>>>(off, n, cnt);
    PG_CK(cudaGetLastError());
    pg_status st = pg_exclusive_scan(cnt, pos, n + 1, s);
    if (st) return st;
    uint32_t total = 0;
    PG_CK(cudaMemcpyAsync(&total, pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    uint2 *ch = nullptr;
    PG_CK(cudaMalloc(&ch, (size_t)(total ? total : 1) * sizeof(uint2)));
    if (total) k_chunk_fill<<<g->num_sms * 4, 256, 0, s>>>(off, n, pos, ch);
    PG_CK(cudaGetLastError());
    PG_CK(cudaFreeAsync(cnt, s));
    *out = ch;
    *count = total;
    return PG_OK;
}

pg_status pg_launch_msbfs(pg_graph *g, PgLaunch &L, const uint32_t *sources, uint32_t k,
                          uint32_t *dist, cudaStream_t s) {
    if (!g->msbfs) {
        g->msbfs = new PgMsbfsWork();
        memset(g->msbfs, 0, sizeof(PgMsbfsWork));
        unsigned long long *p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)3 * g->n * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            delete g->msbfs;
            g->msbfs = nullptr;
            return pg_cuda_error(e, "cudaMalloc(batched BFS words)");
        }
        g->msbfs->seen = p;
        g->msbfs->visit = p + g->n;
        g->msbfs->next = p + 2 * (size_t)g->n;
        g->msbfs->n = g->n;
        const bool self = g->transpose_is_self || !g->d_toff;
        for (int d = 0; d < (self ? 1 : 2); d++) {
            pg_status st = build_chunks(g, d ? g->d_toff : g->d_off, &g->msbfs->chunks[d],
                                        &g->msbfs->nchunks[d], s);
            if (st) {
                pg_msbfs_release(g);
                return st;
            }
        }
        if (self) {
            g->msbfs->chunks[1] = g->msbfs->chunks[0];
            g->msbfs->nchunks[1] = g->msbfs->nchunks[0];
        }
    }
    MsArgs A;
    memset(&A, 0, sizeof(A));
    A.G.off = g->d_off;
    A.G.idx = g->d_idx;
    A.G.toff = g->d_toff ? g->d_toff : g->d_off;
    A.G.tidx = g->d_tidx ? g->d_tidx : g->d_idx;
    A.G.n = g->n;
    A.G.m = g->m;
    A.chunks_out = g->msbfs->chunks[0];
    A.nchunks_out = g->msbfs->nchunks[0];
    A.chunks_in = g->msbfs->chunks[1];
    A.nchunks_in = g->has_transpose ? g->msbfs->nchunks[1] : 0u;
    A.ctrl = g->d_ctrl;
    A.seen = g->msbfs->seen;
    A.visit = g->msbfs->visit;
    A.next = g->msbfs->next;
    A.dist = dist;
    A.k = k;
    for (uint32_t j = 0; j < k; j++) A.sources[j] = sources[j];
    A.alpha = L.alpha;
    A.beta = L.beta;
    A.allow_pull = g->has_transpose ? 1u : 0u;
    A.direction = L.direction;
    A.timeout_ns = L.timeout_ns;
    A.max_rounds = L.max_rounds;
    A.stall_block = L.stall_block;
    const uint32_t threads = 512;
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pg_msbfs_kernel, threads, 0));
    if (per_sm < 1) return pg_set_error(PG_ERR_CUDA, "batched BFS kernel does not fit an SM");
    uint32_t bps = L.blocks ? min((uint32_t)per_sm, L.blocks) : (uint32_t)per_sm;
    L.blocks = bps;
    L.threads = threads;
    PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaEventRecord(g->ev0, s));
    PG_CK(cudaLaunchCooperativeKernel((const void *)pg_msbfs_kernel, dim3(bps * g->num_sms),
                                      dim3(threads), args, 0, s));
    PG_CK(cudaEventRecord(g->ev1, s));
    return PG_OK;
}

// pg_msbfs.cu -- batched BFS from up to 64 sources (pg_bfs_multi).
//
// All k searches share every round of Algorithm 1: a vertex carries one bit
// per source in uint64 words (seen; visit = reached in the last round, two
// buffers by round parity; next = bits arriving this round).  A round is
// either top-down (the frontier's vertices OR their visit bits into their
// out-neighbours' next) or bottom-up (every vertex still missing bits ORs the
// visit words of its in-neighbours, stopping as soon as every missing bit is
// found), chosen with the direction-optimisation test of [Beamer12]
// (Sec. 2.2).  A bit that first appears at a vertex in round L gives that
// source's hop distance L + 1 (Sec. 2.2).
//
// No round sweeps the whole vertex set:
//  - a top-down round expands the frontier list (the vertices that gained
//    bits in the previous round); every vertex whose next word it turns
//    non-zero is listed once ("touched"), and only those are updated;
//  - a bottom-up round walks the list of unfinished vertices (seen != all
//    bits; every vertex before the first bottom-up round) and updates each
//    vertex in place: its new bits go to the other visit buffer, so the
//    round's gathers still read the previous round's bits; the still
//    unfinished vertices form the next such list.
//  A visit word that was not rewritten in the last round holds bits of an
//  older round; their sources already reached every out-neighbour, so the
//  "missing bits" masks filter them and no clearing is needed.
// Distances are kept as 5 bit-planes per vertex (plane b, bit j = bit b of
// the distance of source j), updated only for the bits that arrive; one
// decode pass after the last round writes the k x n source-major output with
// coalesced stores (and 0xFFFFFFFF where the bit never arrived).  A bit that
// arrives in round 31 or later is written to the output at once and marked
// with the plane code 31, which the decode pass skips.
//
// High-degree splitting (the load balance of Sec. 2.1's small-task
// discussion): a vertex with at least kHeavy edges in a direction is never
// expanded by one thread or one warp alone.  Its list is cut into chunks of
// at most `chunk_len` edges (cfg->hub_degree, default 1024; the chunk lists
// are rebuilt when it changes), listed once per graph, and any warp takes a
// chunk:
// top-down ORs the vertex's bits into the chunk's targets, bottom-up ORs the
// chunk's visit words (32 at a time, stopping once every missing bit is
// found) into next[w] with one atomicOr, and a short pass over the heavy
// vertices then updates them.
#include "pg_internal.cuh"

namespace {
constexpr uint32_t kHeavy = 32;    // edges: below, one thread (bottom-up) / one lane (top-down)
constexpr uint32_t kChunkDefault = 1024;  // edges per chunk of a heavy vertex
constexpr uint32_t kGather = 8;    // bottom-up: in-neighbour gathers in flight per light vertex
constexpr uint32_t kGatherSparse = 4;  // the same in a sparse round (bitmap word, then visit word)
constexpr uint32_t kChunkSteps = 4;  // bottom-up chunk pass: 32-edge steps per lane in flight
constexpr uint32_t kPlanes = 5;    // distance bit-planes: distances 0..30, code 31 = written directly
constexpr uint32_t kDirect = (1u << kPlanes) - 1u;
constexpr uint32_t kSparse = 32;   // bottom-up round with |F| < n / kSparse: frontier bitmap filter
}  // namespace

// Per-round list sizes; round r reads slot r % 4 and fills slot (r + 1) % 4.
struct MsCount {
    unsigned F;               // frontier list size
    unsigned T;               // touched list size (top-down rounds)
    unsigned U;               // unfinished list size (bottom-up rounds)
    unsigned pad;
    unsigned long long E;     // out-degree sum of the frontier
    unsigned long long pad2[2];
};

struct PgMsbfsWork {
    unsigned long long *seen, *visit[2], *next;
    unsigned long long *planes;  // [kPlanes][n]
    uint32_t *front[2], *unfin[2], *touched;
    uint32_t *flev;              // round whose frontier a vertex last joined (its visit word's age)
    uint32_t *fbits;             // frontier bitmap of a sparse bottom-up round, ceil(n / 32) words
    MsCount *cnt;                // [4]
    uint32_t n;
    uint2 *chunks[2];            // (vertex, first edge) per chunk: out-lists, in-lists
    uint32_t nchunks[2];
    uint32_t chunk_len;          // edges per chunk the lists were built for
};

void pg_msbfs_release(pg_graph *g) {
    if (g && g->msbfs) {
        cudaFree(g->msbfs->seen);
        cudaFree(g->msbfs->front[0]);
        cudaFree(g->msbfs->cnt);
        cudaFree(g->msbfs->fbits);
        cudaFree(g->msbfs->chunks[0]);
        if (g->msbfs->chunks[1] != g->msbfs->chunks[0]) cudaFree(g->msbfs->chunks[1]);
        delete g->msbfs;
        g->msbfs = nullptr;
    }
}

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// chunks of each heavy vertex: cnt[v] = ceil(deg / clen) when deg >= kHeavy
__global__ void k_chunk_count(const uint32_t *off, uint32_t n, uint32_t clen, uint32_t *cnt) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        uint32_t c = 0;
        if (v < n) {
            const uint32_t d = off[v + 1] - off[v];
            c = d >= kHeavy ? (d + clen - 1) / clen : 0u;
        }
        cnt[v] = c;
    }
}

__global__ void k_chunk_fill(const uint32_t *off, uint32_t n, uint32_t clen, const uint32_t *pos,
                             uint2 *chunks) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t b = off[v], d = off[v + 1] - b;
        if (d < kHeavy) continue;
        const uint32_t c = (d + clen - 1) / clen;
        for (uint32_t i = 0; i < c; i++) chunks[pos[v] + i] = make_uint2(v, b + i * clen);
    }
}

struct MsArgs {
    PgGraphDev G;
    const uint2 *chunks_out, *chunks_in;
    uint32_t nchunks_out, nchunks_in;
    PgCtrl *ctrl;
    MsCount *cnt;
    unsigned long long *seen, *visit0, *visit1, *next, *planes;
    uint32_t *front0, *front1, *unfin0, *unfin1, *touched;
    uint32_t *flev;
    uint32_t *fbits;      // ceil(n / 32) words, all zero between rounds
    uint32_t *dist;       // k * n, source-major
    uint32_t k;
    uint32_t sources[64];
    uint32_t alpha, beta, allow_pull, direction;
    unsigned long long timeout_ns;
    uint32_t max_rounds, stall_block;
    uint32_t clen;        // edges per chunk of a heavy vertex
};

__device__ __forceinline__ unsigned long long wsum(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Warp-collective append of the lanes' `go` ids to list[] with one atomic on
// *size; returns nothing (the list capacity is n, and every id is appended at
// most once per round, so it cannot overflow).
__device__ __forceinline__ void list_append(uint32_t *list, unsigned *size, bool go, uint32_t id,
                                            int lane) {
    const unsigned bal = __ballot_sync(kFull, go);
    if (!bal) return;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(size, (unsigned)__popc(bal));
    pos = __shfl_sync(kFull, pos, 0);
    if (go) list[pos + __popc(bal & pg_lanemask_lt())] = id;
}

// New bits nb of vertex w at distance dnew: visit word of the next round,
// distance planes (or the output directly from round 31 on).
__device__ __forceinline__ void record_bits(const MsArgs &A, unsigned long long *visit_nxt, uint32_t w,
                                            unsigned long long nb, uint32_t dnew) {
    visit_nxt[w] = nb;
    A.flev[w] = dnew;
    const uint32_t n = A.G.n;
    const uint32_t code = dnew >= kDirect ? kDirect : dnew;
#pragma unroll
    for (uint32_t b = 0; b < kPlanes; b++)
        if ((code >> b) & 1u) A.planes[(size_t)b * n + w] |= nb;
    if (code == kDirect) {
        for (uint32_t j = 0; j < A.k; j++)
            if ((nb >> j) & 1ull) A.dist[(size_t)j * n + w] = dnew;
    }
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

    // init: sources at distance 0 (all-zero planes), every other word 0
    for (uint32_t v = gtid; v < n; v += gthreads) {
        unsigned long long b = 0;
        for (uint32_t j = 0; j < k; j++)
            if (A.sources[j] == v) b |= 1ull << j;
        A.seen[v] = b;
        A.visit0[v] = b;
        A.visit1[v] = 0;
        A.next[v] = 0;
        A.flev[v] = 0;
        for (uint32_t p = 0; p < kPlanes; p++) A.planes[(size_t)p * n + v] = 0;
    }
    const uint32_t nw = (n + 31u) >> 5;  // frontier bitmap words
    for (uint32_t i = gtid; i < nw; i += gthreads) A.fbits[i] = 0;

    if (gtid == 0) {
        // the first frontier: the distinct sources
        uint32_t F = 0;
        unsigned long long E = 0;
        for (uint32_t j = 0; j < k; j++) {
            const uint32_t v = A.sources[j];
            bool dup = false;
            for (uint32_t i = 0; i < j; i++) dup |= (A.sources[i] == v);
            if (dup) continue;
            A.front0[F++] = v;
            E += A.G.off[v + 1] - A.G.off[v];
        }
        A.cnt[0].F = F;
        A.cnt[0].E = E;
    }
    if (A.stall_block == blockIdx.x) return;  // fault injection: never arrive
    if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) return;

    unsigned long long edges_seen = 0;
    const unsigned long long t_deadline = pg_gtimer() + 16ull * A.timeout_ns;
    bool bottom_up = false;
    bool uall = true;          // no bottom-up round yet: every vertex is unfinished
    bool fdirty = false;       // the bitmap holds the last sparse round's frontier
    uint32_t up = 0, Ucur = 0; // current unfinished list and its size
    uint32_t L = 0, pulls = 0;
    for (;; L++) {
        MsCount *cc = &A.cnt[L & 3u];
        MsCount *cn = &A.cnt[(L + 1u) & 3u];
        const uint32_t F = __ldcg(&cc->F);
        const unsigned long long E = pg_ldcg64(&cc->E);
        if (F == 0) break;
        if (A.max_rounds && L >= A.max_rounds) {
            if (gtid == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        if (gtid == 0) {
            MsCount *cr = &A.cnt[(L + 2u) & 3u];  // neither read nor filled in this round
            cr->F = 0;
            cr->T = 0;
            cr->U = 0;
            cr->E = 0;
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
        const uint32_t cur = L & 1u;
        const unsigned long long *visit_cur = cur ? A.visit1 : A.visit0;
        unsigned long long *visit_nxt = cur ? A.visit0 : A.visit1;
        const uint32_t *front_cur = cur ? A.front1 : A.front0;
        uint32_t *front_nxt = cur ? A.front0 : A.front1;
        const uint32_t dnew = L + 1u;
        unsigned long long ne = 0;  // out-degree sum of the next frontier
        // A sparse bottom-up round marks its frontier in a bitmap (n / 8
        // bytes, resident in L2), and a gather reads an in-neighbour's visit
        // word only when its bit is set: the other words hold no bit of this
        // round.  The bitmap is cleared in the round after its use.
        const bool sparse = bottom_up && (unsigned long long)F * kSparse < (unsigned long long)n;
        const bool cleared = fdirty;
        if (fdirty) {
            for (uint32_t i = gtid; i < nw; i += gthreads) A.fbits[i] = 0;
            fdirty = false;
        }
        if (sparse) {
            if (cleared && !pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
            for (uint32_t i = gtid; i < F; i += gthreads) {
                const uint32_t v = __ldcg(front_cur + i);
                atomicOr(A.fbits + (v >> 5), 1u << (v & 31u));
            }
            if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
            fdirty = true;
        }
        if (bottom_up) {
            pulls++;
            const uint32_t *ulist = up ? A.unfin1 : A.unfin0;
            uint32_t *unext = up ? A.unfin0 : A.unfin1;
            const uint32_t U = uall ? n : Ucur;
            // light vertices: one thread each, kGather gathers in flight,
            // stopping at the first step that completes the vertex; warps
            // take consecutive list positions (whole-warp appends).  The
            // in-list indices are read once per round: streaming loads keep
            // them from displacing the visit words in L2.
            for (uint32_t b0 = gwarp * 32u; b0 < U; b0 += nwarps * 32u) {
                const uint32_t i = b0 + (uint32_t)lane;
                uint32_t w = PG_NONE, b = 0, e = 0;
                if (i < U) w = uall ? i : __ldcg(ulist + i);
                unsigned long long s = 0, need = 0, acc = 0, nb = 0;
                bool keep = false, light = false;
                if (w != PG_NONE) {
                    s = A.seen[w];
                    need = full & ~s;
                    if (need) {
                        b = __ldg(A.G.toff + w);
                        e = __ldg(A.G.toff + w + 1);
                        // heavy vertices are updated (and listed) by the chunk pass
                        light = e - b < kHeavy;
                    }
                }
                if (light) {
                    if (sparse) {
                        // bitmap first: a visit word only for a frontier neighbour
                        for (uint32_t q = b; q < e; q += kGatherSparse) {
                            uint32_t u[kGatherSparse], bw[kGatherSparse];
#pragma unroll
                            for (int t = 0; t < (int)kGatherSparse; t++)
                                u[t] = (q + t < e) ? __ldcs(A.G.tidx + q + t) : PG_NONE;
#pragma unroll
                            for (int t = 0; t < (int)kGatherSparse; t++)
                                bw[t] = (u[t] != PG_NONE) ? __ldcg(A.fbits + (u[t] >> 5)) : 0u;
#pragma unroll
                            for (int t = 0; t < (int)kGatherSparse; t++)
                                if ((bw[t] >> (u[t] & 31u)) & 1u) acc |= __ldcg(visit_cur + u[t]);
                            if ((acc & need) == need) break;
                        }
                    } else {
                        for (uint32_t q = b; q < e; q += kGather) {
                            uint32_t u[kGather];
#pragma unroll
                            for (int t = 0; t < (int)kGather; t++)
                                u[t] = (q + t < e) ? __ldcs(A.G.tidx + q + t) : PG_NONE;
#pragma unroll
                            for (int t = 0; t < (int)kGather; t++)
                                if (u[t] != PG_NONE) acc |= __ldcg(visit_cur + u[t]);
                            if ((acc & need) == need) break;
                        }
                    }
                }
                if (light) {
                    nb = acc & need;
                    if (nb) {
                        A.seen[w] = s | nb;
                        record_bits(A, visit_nxt, w, nb, dnew);
                        ne += __ldg(A.G.off + w + 1) - __ldg(A.G.off + w);
                    }
                    keep = nb != need && e > b;  // still missing bits, reachable
                }
                list_append(front_nxt, &cn->F, light && nb != 0, w, lane);
                list_append(unext, &cn->U, keep, w, lane);
            }
            // heavy vertices: one warp per chunk of in-edges
            for (uint32_t c = gwarp; c < A.nchunks_in; c += nwarps) {
                const uint2 ch = A.chunks_in[c];
                const uint32_t w = ch.x;
                const unsigned long long need = full & ~__ldcg(A.seen + w);
                if (!need) continue;
                const uint32_t e = min(ch.y + A.clen, __ldg(A.G.toff + w + 1));
                // kChunkSteps steps of 32 edges per pass: every index read of
                // the pass, then every gather, one warp OR per pass
                unsigned long long acc = 0;
                for (uint32_t q0 = ch.y; q0 < e; q0 += 32u * kChunkSteps) {
                    uint32_t u[kChunkSteps];
#pragma unroll
                    for (int t = 0; t < (int)kChunkSteps; t++) {
                        const uint32_t q = q0 + 32u * (uint32_t)t + (uint32_t)lane;
                        u[t] = (q < e) ? __ldcs(A.G.tidx + q) : PG_NONE;
                    }
                    if (sparse) {
#pragma unroll
                        for (int t = 0; t < (int)kChunkSteps; t++)
                            if (u[t] != PG_NONE && !((__ldcg(A.fbits + (u[t] >> 5)) >> (u[t] & 31u)) & 1u))
                                u[t] = PG_NONE;
                    }
#pragma unroll
                    for (int t = 0; t < (int)kChunkSteps; t++)
                        if (u[t] != PG_NONE) acc |= __ldcg(visit_cur + u[t]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc |= __shfl_xor_sync(kFull, acc, o);
                    if ((acc & need) == need) break;
                }
                if (lane == 0 && (acc & need)) atomicOr(A.next + w, acc & need);
            }
            if (A.nchunks_in) {
                if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
                // update of the heavy vertices (each at its first chunk)
                for (uint32_t c0 = gwarp * 32u; c0 < A.nchunks_in; c0 += nwarps * 32u) {
                    const uint32_t c = c0 + (uint32_t)lane;
                    uint32_t w = PG_NONE;
                    bool grew = false, keep = false;
                    if (c < A.nchunks_in) {
                        const uint2 ch = A.chunks_in[c];
                        if (ch.y == __ldg(A.G.toff + ch.x)) w = ch.x;
                    }
                    if (w != PG_NONE) {
                        const unsigned long long s = A.seen[w];
                        if ((s & full) != full) {
                            const unsigned long long nx = __ldcg(A.next + w);
                            const unsigned long long nb = nx & ~s & full;
                            if (nx) A.next[w] = 0;
                            if (nb) {
                                A.seen[w] = s | nb;
                                record_bits(A, visit_nxt, w, nb, dnew);
                                ne += __ldg(A.G.off + w + 1) - __ldg(A.G.off + w);
                                grew = true;
                            }
                            keep = ((s | nb) & full) != full;
                        }
                    }
                    list_append(front_nxt, &cn->F, grew, w, lane);
                    list_append(unext, &cn->U, keep, w, lane);
                }
            }
        } else {
            // top-down: warps take 32 consecutive frontier entries and expand
            // their edges cooperatively (32 edges per step)
            for (uint32_t b0 = gwarp * 32u; b0 < F; b0 += nwarps * 32u) {
                const uint32_t i = b0 + (uint32_t)lane;
                unsigned long long bits = 0;
                uint32_t beg = 0, deg = 0;
                if (i < F) {
                    const uint32_t v = __ldcg(front_cur + i);
                    bits = __ldcg(visit_cur + v);
                    beg = __ldg(A.G.off + v);
                    deg = __ldg(A.G.off + v + 1) - beg;
                    if (deg >= kHeavy) deg = 0;  // in the chunk list
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
                for (uint32_t j0 = 0; j0 < total; j0 += 32u) {
                    const uint32_t j = j0 + (uint32_t)lane;
                    uint32_t w = 0;
                    bool first = false;
                    if (j < total) {
                        uint32_t o = 0;
#pragma unroll
                        for (uint32_t step = 16; step >= 1; step >>= 1)
                            if (s_incl[wib][o + step - 1] <= j) o += step;
                        const uint32_t e = s_base[wib][o] + j;  // u32 sum (the base may wrap)
                        w = __ldg(A.G.idx + e);
                        first = atomicOr(A.next + w, s_bits[wib][o]) == 0ull;
                    }
                    list_append(A.touched, &cn->T, first, w, lane);
                }
                __syncwarp();
            }
            // heavy frontier vertices: one warp per chunk of out-edges (only
            // the vertices that joined this round's frontier)
            for (uint32_t c = gwarp; c < A.nchunks_out; c += nwarps) {
                const uint2 ch = A.chunks_out[c];
                if (__ldcg(A.flev + ch.x) != L) continue;
                const unsigned long long bits = __ldcg(visit_cur + ch.x);
                if (!bits) continue;
                const uint32_t e = min(ch.y + A.clen, __ldg(A.G.off + ch.x + 1));
                for (uint32_t q0 = ch.y; q0 < e; q0 += 32u) {
                    const uint32_t q = q0 + (uint32_t)lane;
                    uint32_t w = 0;
                    bool first = false;
                    if (q < e) {
                        w = __ldg(A.G.idx + q);
                        first = atomicOr(A.next + w, bits) == 0ull;
                    }
                    list_append(A.touched, &cn->T, first, w, lane);
                }
            }
            if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
            // update of the touched vertices
            const uint32_t T = __ldcg(&cn->T);
            for (uint32_t b0 = gwarp * 32u; b0 < T; b0 += nwarps * 32u) {
                const uint32_t i = b0 + (uint32_t)lane;
                uint32_t w = 0;
                bool grew = false;
                if (i < T) {
                    w = __ldcg(A.touched + i);
                    const unsigned long long nx = __ldcg(A.next + w);
                    A.next[w] = 0;
                    const unsigned long long s = A.seen[w];
                    const unsigned long long nb = nx & ~s & full;
                    if (nb) {
                        A.seen[w] = s | nb;
                        record_bits(A, visit_nxt, w, nb, dnew);
                        ne += __ldg(A.G.off + w + 1) - __ldg(A.G.off + w);
                        grew = true;
                    }
                }
                list_append(front_nxt, &cn->F, grew, w, lane);
            }
        }
        ne = wsum(ne);
        if (lane == 0 && ne) atomicAdd(&cn->E, ne);
        if (!pg_grid_sync(ctrl, gridDim.x, gen, A.timeout_ns, &s_flag)) break;
        if (bottom_up) {
            Ucur = __ldcg(&cn->U);
            up ^= 1u;
            uall = false;
        }
    }
    if (gtid == 0) {
        ctrl->rounds = L;
        ctrl->pull_rounds = pulls;
    }
}

// Distances from the planes: dist[j * n + v] for every source j (coalesced
// over v); 0xFFFFFFFF where bit j never arrived; code 31 was written directly.
// The planes of a vertex that no bit reached are all zero: not read.
__global__ void k_msbfs_decode(const unsigned long long *seen, const unsigned long long *planes,
                               uint32_t n, uint32_t k, uint32_t *dist) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long s = seen[v];
        unsigned long long p[kPlanes];
#pragma unroll
        for (uint32_t b = 0; b < kPlanes; b++) p[b] = s ? planes[(size_t)b * n + v] : 0ull;
        for (uint32_t j = 0; j < k; j++) {
            uint32_t code = 0;
#pragma unroll
            for (uint32_t b = 0; b < kPlanes; b++) code |= (uint32_t)((p[b] >> j) & 1ull) << b;
            if (!((s >> j) & 1ull)) dist[(size_t)j * n + v] = PG_INF;
            else if (code != kDirect) dist[(size_t)j * n + v] = code;
        }
    }
}

// The same for four consecutive vertices per thread with 16-byte loads and
// stores (n a multiple of 4 and a 16-byte aligned output): one store
// instruction per source for four vertices.
__global__ void k_msbfs_decode4(const unsigned long long *seen, const unsigned long long *planes,
                                uint32_t n, uint32_t k, uint32_t *dist) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < (n >> 2); q += stride) {
        const uint32_t v = q << 2;
        const ulonglong2 s01 = *reinterpret_cast<const ulonglong2 *>(seen + v);
        const ulonglong2 s23 = *reinterpret_cast<const ulonglong2 *>(seen + v + 2);
        const unsigned long long s[4] = {s01.x, s01.y, s23.x, s23.y};
        unsigned long long p[kPlanes][4];
#pragma unroll
        for (uint32_t b = 0; b < kPlanes; b++)
#pragma unroll
            for (int i = 0; i < 4; i++) p[b][i] = 0ull;
        if (s[0] | s[1] | s[2] | s[3]) {
#pragma unroll
            for (uint32_t b = 0; b < kPlanes; b++) {
                const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(planes + (size_t)b * n + v);
                const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(planes + (size_t)b * n + v + 2);
                p[b][0] = a.x;
                p[b][1] = a.y;
                p[b][2] = c.x;
                p[b][3] = c.y;
            }
        }
        for (uint32_t j = 0; j < k; j++) {
            uint32_t d[4];
            bool direct = false;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                uint32_t code = 0;
#pragma unroll
                for (uint32_t b = 0; b < kPlanes; b++) code |= (uint32_t)((p[b][i] >> j) & 1ull) << b;
                const bool hit = (s[i] >> j) & 1ull;
                d[i] = hit ? code : PG_INF;
                direct |= hit && code == kDirect;
            }
            uint32_t *o = dist + (size_t)j * n + v;
            if (!direct) {
                *reinterpret_cast<uint4 *>(o) = make_uint4(d[0], d[1], d[2], d[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (d[i] != kDirect) o[i] = d[i];
            }
        }
    }
}

}  // namespace

// The chunk list of one direction (built once per graph, on first use).
static pg_status build_chunks(pg_graph *g, const uint32_t *off, uint32_t clen, uint2 **out,
                              uint32_t *count, cudaStream_t s) {
    const uint32_t n = g->n;
    *out = nullptr;
    *count = 0;
    uint32_t *cnt = nullptr;
    PG_CK(cudaMallocAsync(&cnt, ((size_t)n + 1) * 2 * sizeof(uint32_t), s));
    uint32_t *pos = cnt + n + 1;
    k_chunk_count<<<g->num_sms * 4, 256, 0, s>>>(off, n, clen, cnt);
    PG_CK(cudaGetLastError());
    pg_status st = pg_exclusive_scan(cnt, pos, n + 1, s);
    if (st) return st;
    uint32_t total = 0;
    PG_CK(cudaMemcpyAsync(&total, pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    uint2 *ch = nullptr;
    PG_CK(cudaMalloc(&ch, (size_t)(total ? total : 1) * sizeof(uint2)));
    if (total) k_chunk_fill<<<g->num_sms * 4, 256, 0, s>>>(off, n, clen, pos, ch);
    PG_CK(cudaGetLastError());
    PG_CK(cudaFreeAsync(cnt, s));
    *out = ch;
    *count = total;
    return PG_OK;
}

pg_status pg_launch_msbfs(pg_graph *g, PgLaunch &L, const uint32_t *sources, uint32_t k,
                          uint32_t chunk_len, uint32_t *dist, cudaStream_t s) {
    const uint32_t clen = chunk_len ? chunk_len : kChunkDefault;
    if (g->msbfs && g->msbfs->chunk_len != clen) {
        // another chunk length: rebuild the chunk lists (the words are kept)
        PgMsbfsWork &W = *g->msbfs;
        PG_CK(cudaStreamSynchronize(s));
        cudaFree(W.chunks[0]);
        if (W.chunks[1] != W.chunks[0]) cudaFree(W.chunks[1]);
        W.chunks[0] = W.chunks[1] = nullptr;
        W.nchunks[0] = W.nchunks[1] = 0;
        W.chunk_len = 0;
    }
    if (!g->msbfs) {
        PgMsbfsWork *W = new PgMsbfsWork();
        memset(W, 0, sizeof(PgMsbfsWork));
        const size_t n = g->n;
        unsigned long long *p = nullptr;
        uint32_t *q = nullptr;
        cudaError_t e = cudaMalloc(&p, (4 + kPlanes) * n * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&q, 6 * n * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&W->cnt, 4 * sizeof(MsCount));
        if (e == cudaSuccess) e = cudaMalloc(&W->fbits, ((n + 31) / 32) * sizeof(uint32_t));
        if (e != cudaSuccess) {
            cudaFree(p);
            cudaFree(q);
            cudaFree(W->cnt);
            delete W;
            return pg_cuda_error(e, "cudaMalloc(batched BFS words)");
        }
        W->seen = p;
        W->visit[0] = p + n;
        W->visit[1] = p + 2 * n;
        W->next = p + 3 * n;
        W->planes = p + 4 * n;
        W->front[0] = q;
        W->front[1] = q + n;
        W->unfin[0] = q + 2 * n;
        W->unfin[1] = q + 3 * n;
        W->touched = q + 4 * n;
        W->flev = q + 5 * n;
        W->n = g->n;
        g->msbfs = W;
    }
    if (g->msbfs->chunk_len == 0) {
        PgMsbfsWork *W = g->msbfs;
        const bool self = g->transpose_is_self || !g->d_toff;
        for (int d = 0; d < (self ? 1 : 2); d++) {
            pg_status st = build_chunks(g, d ? g->d_toff : g->d_off, clen, &W->chunks[d], &W->nchunks[d], s);
            if (st) {
                pg_msbfs_release(g);
                return st;
            }
        }
        if (self) {
            W->chunks[1] = W->chunks[0];
            W->nchunks[1] = W->nchunks[0];
        }
        W->chunk_len = clen;
    }
    PgMsbfsWork &W = *g->msbfs;
    MsArgs A;
    memset(&A, 0, sizeof(A));
    A.G.off = g->d_off;
    A.G.idx = g->d_idx;
    A.G.toff = g->d_toff ? g->d_toff : g->d_off;
    A.G.tidx = g->d_tidx ? g->d_tidx : g->d_idx;
    A.G.n = g->n;
    A.G.m = g->m;
    A.chunks_out = W.chunks[0];
    A.nchunks_out = W.nchunks[0];
    A.chunks_in = W.chunks[1];
    A.nchunks_in = g->has_transpose ? W.nchunks[1] : 0u;
    A.ctrl = g->d_ctrl;
    A.cnt = W.cnt;
    A.seen = W.seen;
    A.visit0 = W.visit[0];
    A.visit1 = W.visit[1];
    A.next = W.next;
    A.planes = W.planes;
    A.front0 = W.front[0];
    A.front1 = W.front[1];
    A.unfin0 = W.unfin[0];
    A.unfin1 = W.unfin[1];
    A.touched = W.touched;
    A.flev = W.flev;
    A.fbits = W.fbits;
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
    A.clen = clen;
    const uint32_t threads = 512;
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pg_msbfs_kernel, threads, 0));
    if (per_sm < 1) return pg_set_error(PG_ERR_CUDA, "batched BFS kernel does not fit an SM");
    uint32_t bps = L.blocks ? min((uint32_t)per_sm, L.blocks) : (uint32_t)per_sm;
    L.blocks = bps;
    L.threads = threads;
    PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
    PG_CK(cudaMemsetAsync(W.cnt, 0, 4 * sizeof(MsCount), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaEventRecord(g->ev0, s));
    PG_CK(cudaLaunchCooperativeKernel((const void *)pg_msbfs_kernel, dim3(bps * g->num_sms),
                                      dim3(threads), args, 0, s));
    if ((g->n & 3u) == 0 && ((uintptr_t)dist & 15u) == 0)
        k_msbfs_decode4<<<g->num_sms * 8, 256, 0, s>>>(W.seen, W.planes, g->n, k, dist);
    else
        k_msbfs_decode<<<g->num_sms * 8, 256, 0, s>>>(W.seen, W.planes, g->n, k, dist);
    PG_CK(cudaGetLastError());
    PG_CK(cudaEventRecord(g->ev1, s));
    return PG_OK;
}

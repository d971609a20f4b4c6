// pg_traverse.cu -- persistent frontier traversal for sm_103a.
//
// One cooperative launch runs every round of Algorithm 1 (frontier-based
// traversal) without returning to the host.  Two instantiations:
//   BFS   (Sec. 2.2): value = uint32 hop distance, relax = atomicMin(d + 1);
//   REACH (Sec. 2.1): value = uint64 source bitmask, relax = atomicOr(mask),
//                     forward (G) and backward (G^T) searches share the rounds.
// Vertical granularity control (Sec. 2.1) is a per-warp local search: a warp
// that takes a chunk of c frontier entries may expand up to c*(tau-1)
// further vertices it improves, held in a shared-memory FIFO, before new
// improvements spill to the next frontier bag.  Any vertex whose value
// improves is expanded again later (label-correcting, Sec. 2.2), so the
// result is the exact fixpoint for every tau and every push/pull sequence.
//
// Frontier bags (the paper's hash bag, Sec. 2.1 "Data Structure Design",
// rethought for the GPU): a flat array per round parity with a global tail
// and warp-aggregated appends, de-duplicated by a per-vertex round tag.
// Vertices of out-degree >= hub_degree are also listed as hubs when
// appended; their edges are split into fixed chunks taken by any warp.
// Pull rounds (direction optimisation [Beamer12], Sec. 2.2) run at the
// settled level L = smallest tentative distance among active vertices.
#include <cstdio>

#include "pg_internal.cuh"

namespace {

constexpr int kU = 4;                 // 32-edge batches in flight per step
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr unsigned long long kMask40 = (1ull << 40) - 1;

struct TravArgs {
    PgGraphDev G;
    PgCtrl *ctrl;
    uint32_t *bag;        // [2][cap]
    uint32_t cap;
    uint32_t *stamp;      // [2n]
    PgHub *hubs;          // [2][hcap]
    uint32_t hcap;
    uint32_t *dist;       // BFS output
    unsigned long long *mask[2];  // REACH outputs (fwd, bwd)
    uint32_t src;
    uint32_t k, dir;
    uint32_t sources[64];
    PgLaunch L;
};

struct WarpSm {
    uint32_t *lq;            // local queue [qcap]
    uint32_t *s_incl;        // [32] inclusive degree prefix of the wave
    uint32_t *s_base;        // [32] row start - exclusive prefix
    uint32_t *s_dir;         // [32] direction of the owner (REACH)
    unsigned long long *s_val;  // [32] value to propagate (BFS: d + 1)
};

struct Round {
    uint32_t cur, nxt;       // storage parity
    PgSlot *sc, *sn;         // counters of the bag read / filled
    uint32_t tag;            // round tag of the bag being filled
    uint32_t tau;
    uint32_t F;
};

struct Counters {
    unsigned long long expansions = 0, pushes = 0;
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ uint32_t warp_min(uint32_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(kFull, x, o));
    return x;
}

template <bool kReach>
__device__ __forceinline__ const uint32_t *row_off(const TravArgs &A, uint32_t dir) {
    return (kReach && dir) ? A.G.toff : A.G.off;
}
template <bool kReach>
__device__ __forceinline__ const uint32_t *row_idx(const TravArgs &A, uint32_t dir) {
    return (kReach && dir) ? A.G.tidx : A.G.idx;
}

// Append the lanes' improved vertices (go[u]) to the next bag.  Warp-
// collective: every lane calls it with the same control flow.
//   - de-duplication: atomicExch of the round tag into stamp[key]
//   - one atomicAdd on the bag tail per warp call
//   - out-degree sum for the schedule statistics, hub registration
//   - BFS: min tentative distance over all attempted pushes (kept even when
//     the push was de-duplicated), which defines the settled level.
template <bool kReach>
__device__ void push_global(const TravArgs &A, const Round &R, const uint32_t (&w)[kU],
                            const uint32_t (&dirv)[kU], const uint32_t (&nd)[kU],
                            const bool (&go)[kU], int lane, Counters &C) {
    bool keep[kU];
    uint32_t deg[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
        keep[u] = false;
        deg[u] = 0;
        if (go[u]) {
            const uint32_t key = w[u] + ((kReach && dirv[u]) ? A.G.n : 0u);
            keep[u] = atomicExch(&A.stamp[key], R.tag) != R.tag;
        }
    }
#pragma unroll
    for (int u = 0; u < kU; u++) {
        if (go[u]) {
            const uint32_t *o = row_off<kReach>(A, dirv[u]);
            deg[u] = __ldg(o + w[u] + 1) - __ldg(o + w[u]);
        }
    }
    unsigned bal[kU];
    uint32_t before[kU];
    uint32_t total = 0;
#pragma unroll
    for (int u = 0; u < kU; u++) {
        bal[u] = __ballot_sync(kFull, keep[u]);
        before[u] = total;
        total += __popc(bal[u]);
    }
    if (!kReach) {
        uint32_t mn = PG_INF;
#pragma unroll
        for (int u = 0; u < kU; u++)
            if (go[u]) mn = min(mn, nd[u]);
        mn = warp_min(mn);
        if (lane == 0 && mn != PG_INF) atomicMin(&R.sn->min_level, mn);
    }
    if (total == 0) return;
    uint32_t pos = 0;
    if (lane == 0) pos = atomicAdd(&R.sn->size, total);
    pos = __shfl_sync(kFull, pos, 0);
    const unsigned lt = pg_lanemask_lt();
    unsigned long long dsum = 0;
#pragma unroll
    for (int u = 0; u < kU; u++) {
        if (keep[u]) {
            const uint32_t p = pos + before[u] + __popc(bal[u] & lt);
            const uint32_t entry = kReach ? (w[u] | (dirv[u] << 31)) : w[u];
            if (p < A.cap) {
                A.bag[(size_t)R.nxt * A.cap + p] = entry;
            } else {
                atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
            }
            dsum += deg[u];
            if (deg[u] >= A.L.hub_degree) {
                const unsigned long long pk =
                    atomicAdd(&R.sn->hub_pack, (1ull << 40) | (unsigned long long)deg[u]);
                const uint32_t hi = (uint32_t)(pk >> 40);
                if (hi < A.hcap) {
                    PgHub h;
                    h.v = entry;
                    h.start = (uint32_t)(pk & kMask40);
                    A.hubs[(size_t)R.nxt * A.hcap + hi] = h;
                } else {
                    atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
                }
            }
        }
    }
    dsum = warp_sum64(dsum);
    if (lane == 0) atomicAdd(&R.sn->out_edges, dsum);
    C.pushes += (lane == 0) ? total : 0;
}

// Value a vertex propagates: BFS d+1 (INF stays INF), REACH its mask.
template <bool kReach>
__device__ __forceinline__ unsigned long long load_prop(const TravArgs &A, uint32_t v,
                                                        uint32_t dir) {
    if (kReach) return pg_ldcg64(A.mask[dir] + v);
    const uint32_t d = pg_ldcg(A.dist + v);
    return d == PG_INF ? (unsigned long long)PG_INF : (unsigned long long)(d + 1);
}

// Relax arc (.., w) with propagated value p; returns true if w improved.
template <bool kReach>
__device__ __forceinline__ bool relax(const TravArgs &A, uint32_t w, uint32_t dir,
                                      unsigned long long p) {
    if (kReach) {
        const unsigned long long old = atomicOr(A.mask[dir] + w, p);
        return (p & ~old) != 0ull;
    }
    const uint32_t nd = (uint32_t)p;
    return nd < atomicMin(A.dist + w, nd);
}

// Expand one wave (<= 32 vertices, one per lane) cooperatively: the wave's
// out-edges are laid end to end and dealt 32 per step to the lanes, with
// kU steps in flight.  Improved vertices go to the warp's local queue while
// the VGC budget and queue space last, otherwise to the next bag.
template <bool kReach>
__device__ void expand_wave(const TravArgs &A, const Round &R, const WarpSm &S, uint32_t entry,
                            bool from_bag, uint32_t &budget, uint32_t &qhead, uint32_t &qtail,
                            int lane, Counters &C) {
    const uint32_t qmask = A.L.qcap - 1;
    uint32_t v = PG_NONE, dir = 0;
    if (entry != PG_NONE) {
        v = kReach ? (entry & 0x7FFFFFFFu) : entry;
        dir = kReach ? (entry >> 31) : 0u;
    }
    unsigned long long prop = 0;
    uint32_t beg = 0, deg = 0;
    bool hub_repush = false;
    if (v != PG_NONE) {
        const uint32_t *o = row_off<kReach>(A, dir);
        beg = __ldg(o + v);
        deg = __ldg(o + v + 1) - beg;
        prop = load_prop<kReach>(A, v, dir);
        if (deg >= A.L.hub_degree) {
            // hubs from the bag are expanded through the hub list; a hub met
            // by a local search is sent to the next bag (listed there)
            hub_repush = !from_bag;
            deg = 0;
        } else if (!kReach && prop == (unsigned long long)PG_INF) {
            deg = 0;
        } else {
            C.expansions++;
        }
    }
    {
        const bool any = __any_sync(kFull, hub_repush);
        if (any) {
            uint32_t w1[kU] = {v, 0, 0, 0}, d1[kU] = {dir, 0, 0, 0};
            uint32_t n1[kU] = {(uint32_t)(prop - 1), 0, 0, 0};
            bool g1[kU] = {hub_repush, false, false, false};
            push_global<kReach>(A, R, w1, d1, n1, g1, lane, C);
        }
    }
    const uint32_t incl = warp_incl_scan(deg, lane);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    S.s_incl[lane] = incl;
    S.s_base[lane] = beg - (incl - deg);
    S.s_val[lane] = prop;
    S.s_dir[lane] = dir;
    __syncwarp();
    const unsigned lt = pg_lanemask_lt();
    for (uint32_t base = 0; base < total; base += 32u * kU) {
        uint32_t w[kU], wd[kU], nd[kU];
        unsigned long long pv[kU];
        bool ok[kU], imp[kU], go[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t j = base + (uint32_t)u * 32u + (uint32_t)lane;
            ok[u] = j < total;
            w[u] = 0; wd[u] = 0; pv[u] = 0;
            if (ok[u]) {
                uint32_t o = 0;
#pragma unroll
                for (uint32_t step = 16; step >= 1; step >>= 1)
                    if (S.s_incl[o + step - 1] <= j) o += step;
                const uint32_t e = S.s_base[o] + j;
                wd[u] = S.s_dir[o];
                pv[u] = S.s_val[o];
                w[u] = __ldg(row_idx<kReach>(A, wd[u]) + e);
            }
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            imp[u] = ok[u] && relax<kReach>(A, w[u], wd[u], pv[u]);
            nd[u] = (uint32_t)pv[u];
        }
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const unsigned b = __ballot_sync(kFull, imp[u]);
            go[u] = false;
            if (b) {
                const uint32_t cnt = __popc(b);
                const uint32_t rank = __popc(b & lt);
                const uint32_t space = min(A.L.qcap - (qtail - qhead), budget);
                const uint32_t nloc = min(cnt, space);
                if (imp[u]) {
                    if (rank < nloc) {
                        S.lq[(qtail + rank) & qmask] = kReach ? (w[u] | (wd[u] << 31)) : w[u];
                    } else {
                        go[u] = true;
                    }
                }
                qtail += nloc;
                budget -= nloc;
            }
        }
        push_global<kReach>(A, R, w, wd, nd, go, lane, C);
    }
    __syncwarp();
}

// One warp task: c frontier entries plus the local search they start.
template <bool kReach>
__device__ void run_task(const TravArgs &A, const Round &R, const WarpSm &S, uint32_t entry,
                         uint32_t c, int lane, Counters &C) {
    uint32_t budget = c * (R.tau - 1u);
    uint32_t qhead = 0, qtail = 0;
    bool from_bag = true;
    for (;;) {
        expand_wave<kReach>(A, R, S, entry, from_bag, budget, qhead, qtail, lane, C);
        const uint32_t avail = qtail - qhead;
        if (avail == 0) break;
        const uint32_t take = min(32u, avail);
        __syncwarp();
        entry = ((uint32_t)lane < take) ? S.lq[(qhead + lane) & (A.L.qcap - 1)] : PG_NONE;
        qhead += take;
        from_bag = false;
        __syncwarp();
    }
}

// Edges of listed hubs, dealt in chunks of `hch` edges (hch <= hub_degree, so
// a chunk touches at most two hubs).  Improvements go straight to the bag.
template <bool kReach>
__device__ void hub_edges(const TravArgs &A, const Round &R, int lane, Counters &C) {
    const unsigned long long hp = pg_ldcg64(&R.sc->hub_pack);
    const uint32_t hcount = min((uint32_t)(hp >> 40), A.hcap);
    const uint32_t hedges = (uint32_t)(hp & kMask40);
    if (hcount == 0) return;
    const uint32_t hch = min(1024u, A.L.hub_degree);
    const PgHub *H = A.hubs + (size_t)R.cur * A.hcap;
    for (;;) {
        uint32_t a = 0;
        if (lane == 0) a = atomicAdd(&R.sc->hub_cursor, hch);
        a = __shfl_sync(kFull, a, 0);
        if (a >= hedges) break;
        const uint32_t len = min(hch, hedges - a);
        uint32_t lo = 0, hi = hcount;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldcg(&H[mid].start) <= a) lo = mid; else hi = mid;
        }
        uint32_t hv[2], hs[2], hb[2], hd[2], hdeg[2];
        unsigned long long hpv[2];
        for (int t = 0; t < 2; t++) {
            hs[t] = PG_INF; hv[t] = 0; hb[t] = 0; hd[t] = 0; hpv[t] = 0; hdeg[t] = 0;
            const uint32_t i = lo + t;
            if (i < hcount) {
                const uint32_t e = __ldcg(&H[i].v);
                hs[t] = __ldcg(&H[i].start);
                hv[t] = kReach ? (e & 0x7FFFFFFFu) : e;
                hd[t] = kReach ? (e >> 31) : 0u;
                hb[t] = __ldg(row_off<kReach>(A, hd[t]) + hv[t]);
                hdeg[t] = __ldg(row_off<kReach>(A, hd[t]) + hv[t] + 1) - hb[t];
                hpv[t] = load_prop<kReach>(A, hv[t], hd[t]);
            }
        }
        if (lane == 0) C.expansions += (hs[1] < a + len) ? 2 : 1;
        for (uint32_t t0 = 0; t0 < len; t0 += 32u * kU) {
            uint32_t w[kU], wd[kU], nd[kU];
            unsigned long long pv[kU];
            bool go[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const uint32_t j = a + t0 + (uint32_t)u * 32u + (uint32_t)lane;
                go[u] = false;
                w[u] = 0; wd[u] = 0; pv[u] = 0;
                if (j < a + len) {
                    const int t = (j >= hs[1]) ? 1 : 0;
                    const uint32_t rel = j - hs[t];
                    if (rel < hdeg[t]) {
                        wd[u] = hd[t];
                        pv[u] = hpv[t];
                        w[u] = __ldg(row_idx<kReach>(A, hd[t]) + hb[t] + rel);
                        go[u] = !(!kReach && pv[u] == (unsigned long long)PG_INF);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                go[u] = go[u] && relax<kReach>(A, w[u], wd[u], pv[u]);
                nd[u] = (uint32_t)pv[u];
            }
            push_global<kReach>(A, R, w, wd, nd, go, lane, C);
        }
    }
}

// Bottom-up round at settled level L (BFS only): every vertex with
// dist > L+1 looks for an in-neighbour at distance L (first match wins) and
// takes L+1; bag entries still above L stay active.
__device__ void pull_round(const TravArgs &A, const Round &R, uint32_t Lvl, int lane,
                           uint32_t gwarp, uint32_t nwarps, Counters &C) {
    const uint32_t n = A.G.n;
    const uint32_t target = Lvl + 1u;
    for (uint32_t base = gwarp * 32u; base < n; base += nwarps * 32u) {
        const uint32_t v = base + lane;
        bool found = false;
        if (v < n) {
            const uint32_t d = pg_ldcg(A.dist + v);
            if (d > target) {
                const uint32_t b = __ldg(A.G.toff + v), e = __ldg(A.G.toff + v + 1);
                for (uint32_t q = b; q < e; q++) {
                    const uint32_t u = __ldg(A.G.tidx + q);
                    if (pg_ldcg(A.dist + u) == Lvl) { found = true; break; }
                }
                if (found) A.dist[v] = target;
            }
        }
        uint32_t w[kU] = {v, 0, 0, 0}, wd[kU] = {0, 0, 0, 0}, nd[kU] = {target, 0, 0, 0};
        bool go[kU] = {found, false, false, false};
        if (__any_sync(kFull, found)) push_global<false>(A, R, w, wd, nd, go, lane, C);
    }
    for (uint32_t base = gwarp * 32u; base < R.F; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        uint32_t v = 0, d = 0;
        bool keep = false;
        if (i < R.F) {
            v = __ldcg(A.bag + (size_t)R.cur * A.cap + i);
            d = pg_ldcg(A.dist + v);
            keep = d > Lvl;
        }
        uint32_t w[kU] = {v, 0, 0, 0}, wd[kU] = {0, 0, 0, 0}, nd[kU] = {d, 0, 0, 0};
        bool go[kU] = {keep, false, false, false};
        if (__any_sync(kFull, keep)) push_global<false>(A, R, w, wd, nd, go, lane, C);
    }
}

__device__ __forceinline__ void reset_slot(PgSlot *s) {
    s->size = 0;
    s->head = 0;
    s->hub_cursor = 0;
    s->min_level = PG_INF;
    s->out_edges = 0;
    s->hub_pack = 0;
    s->settled = 0;
    s->expansions = 0;
}

__device__ __forceinline__ uint32_t mix32(uint32_t a, uint32_t b) {
    unsigned long long z = ((unsigned long long)a << 32) ^ b ^ 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (uint32_t)(z ^ (z >> 31));
}

// Schedule-MLP inference on one warp; weights in shared memory.  Returns
// the arg-max action among the allowed ones (ties -> lowest index).
__device__ uint32_t mlp_decide(const float *W, const float (&x)[5], bool allow_pull, int lane) {
    const float *W1 = W, *b1 = W + 160, *W2 = W + 192, *b2 = W + 1216, *W3 = W + 1248,
                *b3 = W + 1504;
    float h1 = b1[lane];
#pragma unroll
    for (int i = 0; i < 5; i++) h1 = fmaf(W1[lane * 5 + i], x[i], h1);
    h1 = fmaxf(h1, 0.f);
    float h2 = b2[lane];
#pragma unroll
    for (int i = 0; i < 32; i++) h2 = fmaf(W2[lane * 32 + i], __shfl_sync(kFull, h1, i), h2);
    h2 = fmaxf(h2, 0.f);
    const int a = lane & 7;
    float y = b3[a];
#pragma unroll
    for (int i = 0; i < 32; i++) y = fmaf(W3[a * 32 + i], __shfl_sync(kFull, h2, i), y);
    uint32_t best = 0;
    float by = __shfl_sync(kFull, y, 0);
    for (int t = 1; t < (int)PG_NUM_ACTIONS; t++) {
        const float yt = __shfl_sync(kFull, y, t);
        if ((uint32_t)t == PG_ACTION_PULL && !allow_pull) continue;
        if (yt > by) { by = yt; best = (uint32_t)t; }
    }
    return best;
}

__device__ __forceinline__ float flog2p1(float x) { return log2f(1.0f + x); }

template <bool kReach>
__global__ void __launch_bounds__(512) pg_traverse_kernel(const TravArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    __shared__ uint32_t s_action;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwib = blockDim.x >> 5;
    const uint32_t gwarp = blockIdx.x * nwib + wib;
    const uint32_t nwarps = gridDim.x * nwib;
    const uint32_t nblocks = gridDim.x;

    // shared memory carve-up
    float *s_w = reinterpret_cast<float *>(smem);                       // 1512 floats
    unsigned long long *s_val_all =
        reinterpret_cast<unsigned long long *>(smem + 6144);            // [nwib][32]
    uint32_t *s_u32 = reinterpret_cast<uint32_t *>(smem + 6144 + nwib * 256);
    WarpSm S;
    S.s_val = s_val_all + wib * 32;
    S.s_incl = s_u32 + wib * 96;
    S.s_base = S.s_incl + 32;
    S.s_dir = S.s_incl + 64;
    S.lq = s_u32 + nwib * 96 + (size_t)wib * A.L.qcap;

    if (A.L.schedule == PG_SCHED_LEARNED)
        for (int i = threadIdx.x; i < (int)PG_MLP_NPARAMS; i += blockDim.x) s_w[i] = A.L.weights[i];

    PgCtrl *ctrl = A.ctrl;
    unsigned gen = 0;
    const unsigned long long tmo = A.L.timeout_ns;
    const uint32_t n = A.G.n;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t gthreads = gridDim.x * blockDim.x;

    // ---- init: values, first bag (Algorithm 1: F_0)
    if (!kReach) {
        for (uint32_t v = gtid; v < n; v += gthreads) A.dist[v] = (v == A.src) ? 0u : PG_INF;
    } else {
        for (uint32_t v = gtid; v < n; v += gthreads) {
            unsigned long long bits = 0;
            for (uint32_t j = 0; j < A.k; j++)
                if (A.sources[j] == v) bits |= 1ull << j;
            if (A.dir & PG_FWD) A.mask[0][v] = bits;
            if (A.dir & PG_BWD) A.mask[1][v] = bits;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int s = 0; s < PG_NUM_SLOTS; s++) reset_slot(&ctrl->slot[s]);
        PgSlot *s0 = &ctrl->slot[0];
        const uint32_t tag0 = A.L.epoch;
        uint32_t cnt = 0;
        unsigned long long oe = 0;
        const uint32_t ndir = kReach ? 2 : 1;
        for (uint32_t d = 0; d < ndir; d++) {
            if (kReach && !(A.dir & (d ? PG_BWD : PG_FWD))) continue;
            const uint32_t ksrc = kReach ? A.k : 1;
            for (uint32_t j = 0; j < ksrc; j++) {
                const uint32_t v = kReach ? A.sources[j] : A.src;
                const uint32_t key = v + (d ? n : 0u);
                if (A.stamp[key] == tag0) continue;
                A.stamp[key] = tag0;
                const uint32_t *o = d ? A.G.toff : A.G.off;
                const uint32_t dg = o[v + 1] - o[v];
                const uint32_t entry = kReach ? (v | (d << 31)) : v;
                A.bag[cnt++] = entry;
                oe += dg;
                if (dg >= A.L.hub_degree) {
                    const unsigned long long pk = s0->hub_pack;
                    PgHub h;
                    h.v = entry;
                    h.start = (uint32_t)(pk & kMask40);
                    A.hubs[pk >> 40] = h;
                    s0->hub_pack = pk + ((1ull << 40) | dg);
                }
            }
        }
        s0->size = cnt;
        s0->min_level = 0;
        s0->out_edges = oe;
    }
    if (A.L.stall_block == blockIdx.x) return;  // fault injection: never arrive
    if (!pg_grid_sync(ctrl, nblocks, gen, tmo, &s_flag)) return;

    Counters C;
    unsigned long long t_begin = __ldcg(&ctrl->t_release);
    // whole-launch limit: 16 x the per-wait limit, checked once per round
    const unsigned long long t_deadline = t_begin + 16ull * tmo;
    unsigned long long prev_ns = 0;
    unsigned long long edges_seen = 0;
    bool pull_state = false;
    uint32_t pull_rounds = 0;
    uint32_t r = 0;
    bool ok = true;
    for (;; r++) {
        Round R;
        R.cur = r & 1u;
        R.nxt = R.cur ^ 1u;
        R.sc = &ctrl->slot[r % PG_NUM_SLOTS];
        R.sn = &ctrl->slot[(r + 1) % PG_NUM_SLOTS];
        R.tag = A.L.epoch + r + 1u;
        R.F = __ldcg(&R.sc->size);
        if (R.F == 0) break;
        if ((A.L.max_rounds && r >= A.L.max_rounds) || R.tag == 0u) {
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        if (R.F > A.cap) {
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        const unsigned long long E = pg_ldcg64(&R.sc->out_edges);
        const uint32_t Lvl = __ldcg(&R.sc->min_level);
        float x[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (A.L.schedule == PG_SCHED_LEARNED || A.L.trace != nullptr) {
            x[0] = flog2p1((float)R.F) / 24.f;
            x[1] = flog2p1((float)E) / 32.f;
            x[2] = flog2p1((float)E / (float)R.F) / 8.f;
            x[3] = flog2p1((float)r) / 24.f;
            x[4] = flog2p1((float)prev_ns * 1e-3f) / 16.f;
        }

        // ---- schedule decision (identical in every CTA)
        const bool can_pull = (!kReach) && A.L.allow_pull && Lvl != PG_INF;
        uint32_t action;
        if (A.L.schedule == PG_SCHED_LEARNED) {
            if (wib == 0) {
                const uint32_t a = mlp_decide(s_w, x, can_pull, lane);
                if (lane == 0) s_action = a;
            }
            __syncthreads();
            action = s_action;
        } else if (A.L.schedule == PG_SCHED_RANDOM) {
            const uint32_t na = can_pull ? PG_NUM_ACTIONS : PG_NUM_ACTIONS - 1u;
            action = mix32(A.L.seed, r) % na;
        } else if (A.L.schedule == PG_SCHED_SCRIPT) {
            action = A.L.script[r % A.L.script_len];
            if (action >= PG_NUM_ACTIONS) action = 0;
        } else {
            if (can_pull && A.L.direction == PG_DIR_AUTO) {
                const unsigned long long unexplored =
                    (unsigned long long)A.G.m > edges_seen ? (unsigned long long)A.G.m - edges_seen
                                                           : 0ull;
                if (!pull_state) {
                    if (E > unexplored / A.L.alpha) pull_state = true;
                } else if ((unsigned long long)R.F < (unsigned long long)n / A.L.beta) {
                    pull_state = false;
                }
            } else {
                pull_state = false;
            }
            action = PG_NUM_ACTIONS;  // marker: fixed tau
        }
        bool pull;
        if (action == PG_NUM_ACTIONS) {
            pull = pull_state;
            R.tau = A.L.tau;
        } else if (action == PG_ACTION_PULL) {
            pull = can_pull;
            R.tau = 1;
        } else {
            pull = false;
            R.tau = 1u << action;
        }
        if (!pull && A.L.schedule == PG_SCHED_FIXED) R.tau = A.L.tau;
        edges_seen += E;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            reset_slot(&ctrl->slot[(r + 2) % PG_NUM_SLOTS]);
            if (pg_gtimer() > t_deadline) atomicOr(&ctrl->status, PG_DEV_TIMEOUT);
        }

        // ---- round work
        if (pull) {
            pull_round(A, R, Lvl, lane, gwarp, nwarps, C);
            pull_rounds++;
        } else {
            for (;;) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&R.sc->head, A.L.chunk);
                base = __shfl_sync(kFull, base, 0);
                if (base >= R.F) break;
                const uint32_t c = min(A.L.chunk, R.F - base);
                const uint32_t entry =
                    ((uint32_t)lane < c) ? __ldcg(A.bag + (size_t)R.cur * A.cap + base + lane)
                                         : PG_NONE;
                run_task<kReach>(A, R, S, entry, c, lane, C);
            }
            hub_edges<kReach>(A, R, lane, C);
        }
        ok = pg_grid_sync(ctrl, nblocks, gen, tmo, &s_flag);
        if (!ok) break;
        const unsigned long long t_end = __ldcg(&ctrl->t_release);

        // ---- training traces: vertices already at their final distance
        unsigned long long settled = 0;
        if (!kReach && A.L.ref_dist != nullptr && A.L.trace != nullptr && r < A.L.trace_cap) {
            unsigned long long cnt = 0;
            for (uint32_t v = gtid; v < n; v += gthreads)
                cnt += (pg_ldcg(A.dist + v) == __ldg(A.L.ref_dist + v)) ? 1u : 0u;
            cnt = warp_sum64(cnt);
            if (lane == 0 && cnt) atomicAdd(&R.sc->settled, cnt);
            ok = pg_grid_sync(ctrl, nblocks, gen, tmo, &s_flag);
            if (!ok) break;
            settled = pg_ldcg64(&R.sc->settled);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && A.L.trace != nullptr && r < A.L.trace_cap) {
            pg_round_trace tr;
            tr.round = r;
            tr.action = pull ? PG_ACTION_PULL
                             : (uint32_t)(31 - __clz((int)max(R.tau, 1u)));
            tr.frontier = R.F;
            tr.min_level = Lvl;
            tr.out_edges = E;
            tr.t_begin_ns = t_begin;
            tr.t_end_ns = t_end;
            tr.settled = settled;
            for (int i = 0; i < 5; i++) tr.features[i] = x[i];
            tr.reserved = 0;
            A.L.trace[r] = tr;
        }
        prev_ns = t_end - t_begin;
        t_begin = __ldcg(&ctrl->t_release);
    }
    // ---- totals
    unsigned long long e = C.expansions, p = C.pushes;
    e = warp_sum64(e);
    p = warp_sum64(p);
    if (lane == 0) {
        if (e) atomicAdd(&ctrl->expansions, e);
        if (p) atomicAdd(&ctrl->pushes, p);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->rounds = r;
        ctrl->pull_rounds = pull_rounds;
    }
}

template <bool kReach>
size_t traverse_smem(uint32_t threads, uint32_t qcap) {
    const uint32_t nw = threads / 32;
    return 6144 + (size_t)nw * 256 + (size_t)nw * 96 * 4 + (size_t)nw * qcap * 4;
}

template <bool kReach>
pg_status launch_impl(pg_graph *g, PgLaunch &L, TravArgs &A, cudaStream_t s) {
    auto kern = pg_traverse_kernel<kReach>;
    const size_t smem = traverse_smem<kReach>(L.threads, L.qcap);
    int maxopt = 0;
    PG_CK(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
    if (smem > (size_t)maxopt)
        return pg_set_error(PG_ERR_INVALID_ARG,
                            "launch shape needs %zu B shared memory > %d (threads=%u, local_queue=%u)",
                            smem, maxopt, L.threads, L.qcap);
    PG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)L.threads, smem));
    if (per_sm < 1)
        return pg_set_error(PG_ERR_INVALID_ARG,
                            "launch shape does not fit an SM (threads=%u, local_queue=%u)",
                            L.threads, L.qcap);
    uint32_t bps = L.blocks ? min((uint32_t)per_sm, L.blocks) : (uint32_t)per_sm;
    const uint32_t grid = bps * (uint32_t)g->num_sms;
    L.blocks = bps;
    A.L = L;
    PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(L.threads), args, smem,
                                      s));
    return PG_OK;
}

}  // namespace

pg_status pg_launch_traverse(pg_graph *g, PgLaunch &L, int kind, uint32_t src,
                             const uint32_t *sources, uint32_t k, uint32_t dir, uint32_t *dist,
                             unsigned long long *fwd, unsigned long long *bwd, cudaStream_t s) {
    TravArgs A;
    memset(&A, 0, sizeof(A));
    A.G.off = g->d_off;
    A.G.idx = g->d_idx;
    A.G.toff = g->d_toff ? g->d_toff : g->d_off;
    A.G.tidx = g->d_tidx ? g->d_tidx : g->d_idx;
    A.G.n = g->n;
    A.G.m = g->m;
    A.ctrl = g->d_ctrl;
    A.bag = g->d_bag;
    A.cap = g->bag_cap;
    A.stamp = g->d_stamp;
    A.hubs = g->d_hubs;
    A.hcap = g->hub_cap;
    A.dist = dist;
    A.mask[0] = fwd;
    A.mask[1] = bwd;
    A.src = src;
    A.k = k;
    A.dir = dir;
    for (uint32_t j = 0; j < k && j < 64; j++) A.sources[j] = sources[j];
    if (kind == 0) return launch_impl<false>(g, L, A, s);
    return launch_impl<true>(g, L, A, s);
}

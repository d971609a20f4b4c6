// pg_traverse.cu -- persistent frontier traversal for sm_103a.
//
// One cooperative launch runs every round of Algorithm 1 (frontier-based
// traversal) without returning to the host.  Two instantiations:
//   BFS   (Sec. 2.2): value = uint32 hop distance, relax = atomicMin(d + 1);
//   REACH (Sec. 2.1): value = uint64 source bitmask, relax = atomicOr(mask),
//                     forward (G) and backward (G^T) searches share the rounds.
//
// Vertical granularity control (Sec. 2.1) on the GPU is a tau-hop local
// search: a task keeps expanding the vertices it improves as long as they
// lie within tau hops of the round's frontier (BFS: new distance < L + tau,
// L = smallest distance in the frontier; REACH: hop count < tau); other
// improvements spill to the next frontier bag.  By default (PG_VGC_CTA) a
// task is a CTA's share of the bag, searched level by level in shared
// memory with all warps splitting each level; with padded rows a level is
// cut into slot-parallel waves (one lane per vertex and row slot).  The
// alternative (PG_VGC_WARP) is a warp's chunk of entries with a
// shared-memory FIFO and a per-task budget.
// A vertex whose value improves is always expanded again later (Sec. 2.2:
// a vertex can be visited multiple times), so the result is the exact
// fixpoint for every tau and every push/pull sequence.
//
// Frontier bags (the hash bag of Sec. 2.1, rethought): a flat array per
// round parity with a global tail; spills are staged per warp in shared
// memory and appended 128 at a time with one atomicAdd, de-duplicated by a
// per-vertex round tag (skipped in level-pure plain rounds, where every
// vertex can only improve once).
// Neighbour lists come from padded rows (4/8/16 ids per vertex, one to four
// 16-byte loads, no offsets lookup) when the graph's degrees are low, else
// from the CSR with a warp-cooperative edge deal.  Vertices of out-degree
// >= hub_degree are listed as hubs when appended and their edges are split
// into fixed chunks that any warp takes.
// Pull rounds (direction optimisation [Beamer12], Sec. 2.2) run at the
// settled level L, the smallest tentative distance among active vertices:
// every vertex with true distance <= L already holds it, so a bottom-up
// sweep at L yields exactly level L + 1.
#include <cstdio>

#include "pg_internal.cuh"

namespace {

constexpr int kU = 4;                   // 32-wide batches in flight per step
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr unsigned long long kMask40 = (1ull << 40) - 1;
constexpr uint32_t kSpillCap = 32u * kU;  // per-warp spill staging entries
constexpr uint32_t kMaxW = 16;            // widest padded row
// Settled-vertex filter of the CTA BFS local search: 2^kVtLog2 shared-memory
// slots of (distance, vertex), direct-mapped; only with CTA level buffers of
// at most kVtMaxQueue entries (so that both fit in shared memory).
constexpr uint32_t kVtLog2 = 11;
constexpr uint32_t kVtMaxQueue = 4096;

struct TravArgs {
    PgGraphDev G;
    const uint32_t *ell0, *ell1;  // padded rows (forward, reverse) or null
    uint32_t ellw0, ellw1;        // their widths
    PgCtrl *ctrl;
    uint32_t *bag;        // [2][cap]
    uint32_t cap;
    uint32_t *stamp;      // [2n]
    PgHub *hubs;          // [2][hcap]
    uint32_t hcap;
    uint32_t *dist;       // BFS output
    unsigned long long *mask0, *mask1;  // REACH outputs (forward, backward)
    uint32_t src;
    uint32_t k, dir;
    uint32_t need_deg;       // exact out-degree sums at append time (Beamer test)
    uint32_t hubs_possible;  // some out-degree >= hub_degree
    uint32_t sources[64];
    PgLaunch L;
};

// Self-checking builds (-DPG_DEBUG_BOUNDS): every vertex id that enters a
// wave (bag entry, local-queue entry, padded-row slot, CSR index) is checked
// against n; the first bad one is recorded in the control block with its
// site code and the id is replaced by "no vertex", so nothing out of range
// is ever dereferenced.
#ifdef PG_DEBUG_BOUNDS
__device__ __forceinline__ uint32_t dbg_id(const TravArgs &A, uint32_t ent, uint32_t site, bool is_entry,
                                          bool reach) {
    if (ent == PG_NONE) return ent;
    const uint32_t v = reach ? (ent & 0x7FFFFFFFu) : ent;
    if (v < A.G.n) return ent;
    if (atomicCAS(&A.ctrl->dbg_site, 0u, site) == 0u) {
        A.ctrl->dbg_value = ent;
        A.ctrl->dbg_round = A.ctrl->rounds;
    }
    return is_entry ? PG_NONE : PG_NONE;
}
#define PG_DBG_ENTRY(A, e, site, reach) dbg_id(A, e, site, true, reach)
#define PG_DBG_ID(A, e, site, reach) dbg_id(A, e, site, false, reach)
#else
#define PG_DBG_ENTRY(A, e, site, reach) (e)
#define PG_DBG_ID(A, e, site, reach) (e)
#endif

struct WarpSm {
    uint32_t *lq, *lqa;      // local FIFO [qcap]: entry, aux (BFS: distance, REACH: hops)
    uint32_t *sp, *spa;      // spill staging [kSpillCap]: entry, aux
    uint32_t *s_incl, *s_base, *s_dir, *s_aux;  // [32] CSR wave bookkeeping
    unsigned long long *s_val;                  // [32]
};

// Per-CTA aggregates of one round, in shared memory: warps add to them with
// shared-memory atomics, and thread 0 adds them to the global counters once
// per round inside the round barrier (pg_grid_sync_then), so the global
// counters see one atomic per CTA instead of one per warp.
struct CtaStat {
    unsigned long long exp_edges;  // edges expanded in the round
    unsigned long long out_edges;  // out-degree sum of the entries appended to the next bag
    unsigned exp_verts;            // vertices expanded in the round
    unsigned min_level, max_level; // BFS: distance range of attempted appends
    unsigned pad;
};

struct Round {
    uint32_t cur, nxt;       // storage parity
    PgSlot *sc, *sn;         // counters of the bag read / filled
    CtaStat *cs;             // this CTA's aggregates of the round
    uint32_t tag;            // round tag of the bag being filled
    uint32_t tau;
    uint32_t F;
    uint32_t Lbase;          // smallest distance pushed into the bag read
    bool dedupe;             // false only in level-pure plain push rounds
    unsigned long long hub_pack;
};

struct Task {
    uint32_t qhead, qtail;   // local FIFO cursors (warp-uniform)
    uint32_t budget;         // local enqueues left
    uint32_t nsp;            // staged spills
    // CTA level-synchronous local search: when cta_n is set, local children
    // go to the CTA's next-level buffer instead of the warp FIFO
    uint32_t *cta_ent, *cta_aux;
    unsigned *cta_n;
    uint32_t cta_cap;
};

__device__ __forceinline__ void task_init(Task &T, uint32_t budget) {
    T.qhead = T.qtail = 0;
    T.nsp = 0;
    T.budget = budget;
    T.cta_ent = T.cta_aux = nullptr;
    T.cta_n = nullptr;
    T.cta_cap = 0;
}

// Shared-memory level buffers of the CTA local search.
struct CtaSm {
    uint32_t *ent[3], *aux[3];  // three level buffers, rotating
    unsigned long long *vt;     // settled-vertex filter (BFS), or null
    unsigned *n;                // [3] level sizes
    unsigned *task;             // grabbed task base
    unsigned *wcnt;             // [warps + 1] spill counts / offsets of a CTA flush
};

struct Counters {
    unsigned long long expansions = 0, pushes = 0, exp_edges = 0;
    unsigned exp_verts = 0;
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

__device__ __forceinline__ uint32_t warp_max(uint32_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
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

// Append up to kU*32 entries (lane-major batches) to the next bag.  Warp-
// collective: every lane calls it with the same control flow.
//   - de-duplication: atomicExch of the round tag into stamp[key] (skipped
//     when the round cannot produce duplicates)
//   - one atomicAdd on the bag tail per call; with kCta, the call is
//     CTA-collective (every thread of the CTA makes it, wcnt = [warps + 1]
//     shared words) and thread 0 makes one reservation for all warps, so the
//     bag tail sees one atomic per CTA instead of one per warp
//   - out-degree sum (schedule statistics) and hub registration when needed
//   - BFS: min / max distance over all attempted appends (kept even when the
//     append was de-duplicated); the min defines the settled level.
template <bool kReach, bool kCta = false>
__device__ void push_global(const TravArgs &A, const Round &R, const uint32_t (&ent)[kU],
                            const uint32_t (&nd)[kU], const bool (&go)[kU], int lane,
                            Counters &C, unsigned *wcnt = nullptr) {
    bool keep[kU];
    uint32_t deg[kU], prev[kU];
    const bool want_deg = A.need_deg || A.hubs_possible;
    // all tag exchanges in flight before any result is compared
#pragma unroll
    for (int u = 0; u < kU; u++) {
        deg[u] = 0;
        prev[u] = 0;
        if (go[u] && R.dedupe) {
            const uint32_t w = kReach ? (ent[u] & 0x7FFFFFFFu) : ent[u];
            const uint32_t key = w + ((kReach && (ent[u] >> 31)) ? A.G.n : 0u);
            prev[u] = atomicExch(&A.stamp[key], R.tag);
        }
    }
#pragma unroll
    for (int u = 0; u < kU; u++) keep[u] = go[u] && (!R.dedupe || prev[u] != R.tag);
    if (want_deg) {
#pragma unroll
        for (int u = 0; u < kU; u++) {
            if (go[u]) {
                const uint32_t w = kReach ? (ent[u] & 0x7FFFFFFFu) : ent[u];
                const uint32_t *o = row_off<kReach>(A, kReach ? (ent[u] >> 31) : 0u);
                deg[u] = __ldg(o + w + 1) - __ldg(o + w);
            }
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
        uint32_t mn = PG_INF, mx = 0;
#pragma unroll
        for (int u = 0; u < kU; u++)
            if (go[u]) { mn = min(mn, nd[u]); mx = max(mx, nd[u]); }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0 && mn != PG_INF) {
            atomicMin(&R.cs->min_level, mn);
            atomicMax(&R.cs->max_level, mx);
        }
    }
    uint32_t pos = 0;
    if (kCta) {
        const int wib = threadIdx.x >> 5, nwib = blockDim.x >> 5;
        if (lane == 0) wcnt[wib] = total;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t sum = 0;
            for (int w = 0; w < nwib; w++) {
                const uint32_t c = wcnt[w];
                wcnt[w] = sum;
                sum += c;
            }
            wcnt[nwib] = sum ? atomicAdd(&R.sn->size, sum) : 0u;
        }
        __syncthreads();
        pos = wcnt[nwib] + wcnt[wib];
        if (total == 0) return;
    } else {
        if (total == 0) return;
        if (lane == 0) pos = atomicAdd(&R.sn->size, total);
        pos = __shfl_sync(kFull, pos, 0);
    }
    const unsigned lt = pg_lanemask_lt();
    unsigned long long dsum = 0;
#pragma unroll
    for (int u = 0; u < kU; u++) {
        if (keep[u]) {
            const uint32_t p = pos + before[u] + __popc(bal[u] & lt);
            if (p < A.cap) {
                A.bag[(size_t)R.nxt * A.cap + p] = ent[u];
            } else {
                atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
            }
            dsum += deg[u];
            if (A.hubs_possible && deg[u] >= A.L.hub_degree) {
                const unsigned long long pk =
                    atomicAdd(&R.sn->hub_pack, (1ull << 40) | (unsigned long long)deg[u]);
                const uint32_t hi = (uint32_t)(pk >> 40);
                if (hi < A.hcap) {
                    PgHub h;
                    h.v = ent[u];
                    h.start = (uint32_t)(pk & kMask40);
                    A.hubs[(size_t)R.nxt * A.hcap + hi] = h;
                } else {
                    atomicOr(&A.ctrl->status, PG_DEV_OVERFLOW);
                }
            }
        }
    }
    if (want_deg) {
        dsum = warp_sum64(dsum);
        if (lane == 0 && dsum) atomicAdd(&R.cs->out_edges, dsum);
    }
    C.pushes += (lane == 0) ? total : 0;
}

// Append every staged spill of this warp to the next bag.
template <bool kReach>
__device__ void flush_spill(const TravArgs &A, const Round &R, const WarpSm &S, Task &T, int lane,
                            Counters &C) {
    __syncwarp();
    for (uint32_t base = 0; base < T.nsp; base += kSpillCap) {
        uint32_t ent[kU], nd[kU];
        bool go[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t i = base + (uint32_t)u * 32u + (uint32_t)lane;
            go[u] = i < T.nsp;
            ent[u] = go[u] ? S.sp[i] : 0u;
            nd[u] = go[u] ? S.spa[i] : 0u;
        }
        push_global<kReach>(A, R, ent, nd, go, lane, C);
    }
    T.nsp = 0;
    __syncwarp();
}

// End-of-task flush of the CTA local search: every warp's staged spills (at
// most kSpillCap each, one batch) with one bag reservation for the CTA.
// CTA-collective.
template <bool kReach>
__device__ void flush_spill_cta(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                                unsigned *wcnt, int lane, Counters &C) {
    __syncwarp();
    uint32_t ent[kU], nd[kU];
    bool go[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
        const uint32_t i = (uint32_t)u * 32u + (uint32_t)lane;
        go[u] = i < T.nsp;
        ent[u] = go[u] ? S.sp[i] : 0u;
        nd[u] = go[u] ? S.spa[i] : 0u;
    }
    push_global<kReach, true>(A, R, ent, nd, go, lane, C, wcnt);
    T.nsp = 0;
    __syncwarp();
}

// Route one improved entry per lane: into the local FIFO if it is eligible
// and there is room and budget, else into the spill staging.
template <bool kReach>
__device__ __forceinline__ void stage(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                                      bool imp, uint32_t ent, uint32_t aux, bool eligible,
                                      int lane, Counters &C) {
    const unsigned lt = pg_lanemask_lt();
    const bool want = imp && eligible;
    const unsigned bl = __ballot_sync(kFull, want);
    bool to_local = false;
    if (bl && T.cta_n != nullptr) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(T.cta_n, (unsigned)__popc(bl));
        base = __shfl_sync(kFull, base, 0);
        const uint32_t p = base + __popc(bl & lt);
        to_local = want && p < T.cta_cap;
        if (to_local) {
            T.cta_ent[p] = ent;
            T.cta_aux[p] = aux;
        }
    } else if (bl) {
        const uint32_t room = min(A.L.qcap - (T.qtail - T.qhead), T.budget);
        const uint32_t nl = min((uint32_t)__popc(bl), room);
        const uint32_t rank = __popc(bl & lt);
        to_local = want && rank < nl;
        if (to_local) {
            const uint32_t p = (T.qtail + rank) & (A.L.qcap - 1);
            S.lq[p] = ent;
            S.lqa[p] = aux;
        }
        T.qtail += nl;
        T.budget -= nl;
    }
    const bool to_spill = imp && !to_local;
    const unsigned bs = __ballot_sync(kFull, to_spill);
    if (bs) {
        if (T.nsp + (uint32_t)__popc(bs) > kSpillCap) flush_spill<kReach>(A, R, S, T, lane, C);
        if (to_spill) {
            const uint32_t p = T.nsp + __popc(bs & lt);
            S.sp[p] = ent;
            S.spa[p] = aux;
        }
        T.nsp += __popc(bs);
    }
}

// Route a whole padded-row wave at once (CTA local search): one warp scan
// and one shared-memory atomic reserve the lanes' local slots; the rest go
// to the spill staging.  Children of one lane share eligibility (same
// parent).  If the spills do not fit the staging even after a flush, they
// are routed one slot at a time through stage().
template <bool kReach>
__device__ void stage_rows(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                           const bool (&imp)[kMaxW], const uint32_t (&row)[kMaxW], uint32_t dir,
                           uint32_t caux, bool ok_local, uint32_t wmax, int lane, Counters &C) {
    uint32_t mask = 0;
#pragma unroll
    for (int j = 0; j < (int)kMaxW; j++)
        if (imp[j]) mask |= 1u << j;
    const uint32_t cnt = __popc(mask);
    const uint32_t want = ok_local ? cnt : 0u;
    const uint32_t incl = warp_incl_scan(want, lane);
    const uint32_t tot = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (lane == 0 && tot) base = atomicAdd(T.cta_n, tot);
    base = __shfl_sync(kFull, base, 0);
    const uint32_t p0 = base + incl - want;
    const uint32_t nfit = (p0 < T.cta_cap) ? min(want, T.cta_cap - p0) : 0u;
    const uint32_t nsl = cnt - nfit;
    // inside the window nothing spills: skip the second scan
    const bool any_sl = __any_sync(kFull, nsl != 0u);
    const uint32_t sincl = any_sl ? warp_incl_scan(nsl, lane) : 0u;
    const uint32_t stot = any_sl ? __shfl_sync(kFull, sincl, 31) : 0u;
    if (stot && T.nsp + stot > kSpillCap) flush_spill<kReach>(A, R, S, T, lane, C);
    const bool batch_spill = stot <= kSpillCap;
    uint32_t k = 0, q = T.nsp + sincl - nsl;
#pragma unroll
    for (int j = 0; j < (int)kMaxW; j++) {
        if ((mask >> j) & 1u) {
            const uint32_t ent = kReach ? (row[j] | (dir << 31)) : row[j];
            if (k < nfit) {
                T.cta_ent[p0 + k] = ent;
                T.cta_aux[p0 + k] = caux;
            } else if (batch_spill) {
                S.sp[q] = ent;
                S.spa[q] = caux;
                q++;
            }
            k++;
        }
    }
    if (batch_spill) {
        T.nsp += stot;
        return;
    }
    // rare: more spills than the staging holds -- slot by slot
    uint32_t seen = 0;
#pragma unroll
    for (int j = 0; j < (int)kMaxW; j++) {
        const bool bit = (mask >> j) & 1u;
        const bool sp = bit && seen >= nfit;
        seen += bit ? 1u : 0u;
        if ((uint32_t)j < wmax)
            stage<kReach>(A, R, S, T, sp, kReach ? (row[j] | (dir << 31)) : row[j], caux, false,
                          lane, C);
    }
}

// Value a vertex propagates: BFS d + 1 (INF stays INF), REACH its mask.
template <bool kReach>
__device__ __forceinline__ unsigned long long load_prop(const TravArgs &A, uint32_t v,
                                                        uint32_t dir) {
    if (kReach) return pg_ldcg64((dir ? A.mask1 : A.mask0) + v);
    const uint32_t d = pg_ldcg(A.dist + v);
    return d == PG_INF ? (unsigned long long)PG_INF : (unsigned long long)(d + 1);
}

// Relax arc (.., w) with propagated value p, in two halves so that a
// warp issues all of its atomics before it waits for any result:
// relax_issue returns the old value (a "no improvement" value when !ok),
// improved() compares.
template <bool kReach>
__device__ __forceinline__ unsigned long long relax_issue(const TravArgs &A, uint32_t w,
                                                          uint32_t dir, unsigned long long p,
                                                          bool ok) {
    if (kReach) return ok ? atomicOr((dir ? A.mask1 : A.mask0) + w, p) : ~0ull;
    return ok ? (unsigned long long)atomicMin(A.dist + w, (uint32_t)p) : 0ull;
}
template <bool kReach>
__device__ __forceinline__ bool improved(unsigned long long p, unsigned long long old) {
    if (kReach) return (p & ~old) != 0ull;
    return (uint32_t)p < (uint32_t)old;
}

// Local eligibility of a child with aux value `caux` (BFS: its distance,
// REACH: its hop count).
template <bool kReach>
__device__ __forceinline__ bool eligible(const Round &R, uint32_t caux) {
    return kReach ? (caux < R.tau) : (caux < R.Lbase + R.tau);
}

// Expand one wave (<= 32 vertices, one per lane).
template <bool kReach>
__device__ void expand_wave(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                            uint32_t entry, uint32_t aux, bool from_bag, int lane, Counters &C) {
    uint32_t v = PG_NONE, dir = 0;
    const bool valid = entry != PG_NONE;
    if (valid) {
        v = kReach ? (entry & 0x7FFFFFFFu) : entry;
        dir = kReach ? (entry >> 31) : 0u;
    }
    const uint32_t *ell = dir ? A.ell1 : A.ell0;
    const uint32_t W = dir ? A.ellw1 : A.ellw0;
    // fetch: value and padded row in parallel
    unsigned long long prop = 0;
    uint32_t row[kMaxW];
#pragma unroll
    for (int j = 0; j < (int)kMaxW; j++) row[j] = PG_NONE;
    bool use_row = false;
    if (valid) {
        // BFS entries of a local search carry the distance they were given
        // (aux); a later decrease by another task re-queues the vertex there,
        // so expanding with this value is exact and saves a dependent load
        prop = (!kReach && !from_bag) ? (unsigned long long)(aux + 1u) : load_prop<kReach>(A, v, dir);
        if (ell != nullptr) {
            use_row = true;
            const uint4 *rp = reinterpret_cast<const uint4 *>(ell + (size_t)v * W);
#pragma unroll
            for (int q = 0; q < (int)(kMaxW / 4); q++) {
                if ((uint32_t)q * 4u < W) {
                    const uint4 t = __ldg(rp + q);
                    row[4 * q] = t.x; row[4 * q + 1] = t.y; row[4 * q + 2] = t.z; row[4 * q + 3] = t.w;
                }
            }
#ifdef PG_DEBUG_BOUNDS
            for (int j = 0; j < (int)kMaxW; j++)
                if (row[j] < 0x80000000u) row[j] = PG_DBG_ID(A, row[j], 3u, false);
#endif
        }
    }
    const bool dead = !kReach && prop == (unsigned long long)PG_INF;
    const bool is_long = valid && !dead && (!use_row || row[0] == PG_ELL_LONG);
    // CSR row for long lanes (dependent load, rare when padded rows exist)
    uint32_t beg = 0, deg = 0;
    bool hub_repush = false;
    if (is_long) {
        const uint32_t *o = row_off<kReach>(A, dir);
        beg = __ldg(o + v);
        deg = __ldg(o + v + 1) - beg;
        if (A.hubs_possible && deg >= A.L.hub_degree) {
            hub_repush = !from_bag;  // a hub met by a local search goes to the next bag
            deg = 0;
        }
    }
    const uint32_t caux = kReach ? aux + 1u : (uint32_t)prop;
    const bool ok_local = eligible<kReach>(R, caux);
    // padded rows: relax every slot (all atomics in flight), then stage
    const bool row_lane = use_row && valid && !dead && !is_long;
    if (__any_sync(kFull, row_lane)) {
        bool imp[kMaxW];
        unsigned long long old[kMaxW];
        uint32_t nvalid = 0;
#pragma unroll
        for (int j = 0; j < (int)kMaxW; j++) {
            const bool ok = row_lane && (uint32_t)j < W && row[j] < 0x80000000u;
            nvalid += ok ? 1u : 0u;
            old[j] = relax_issue<kReach>(A, row[j], dir, prop, ok);
        }
        // children inside the window are expanded next by this SM: start
        // fetching their padded rows while the atomics are in flight
        if (row_lane && ok_local) {
#pragma unroll
            for (int j = 0; j < (int)kMaxW; j++)
                if ((uint32_t)j < W && row[j] < 0x80000000u) pg_prefetch_l1(ell + (size_t)row[j] * W);
        }
#pragma unroll
        for (int j = 0; j < (int)kMaxW; j++) imp[j] = improved<kReach>(prop, old[j]);
        if (row_lane) { C.expansions++; C.exp_verts++; C.exp_edges += nvalid; }
        const uint32_t wmax = max(A.ellw0, A.ellw1);
        if (T.cta_n != nullptr) {
            stage_rows<kReach>(A, R, S, T, imp, row, dir, caux, ok_local, wmax, lane, C);
        } else {
#pragma unroll
            for (int j = 0; j < (int)kMaxW; j++) {
                if ((uint32_t)j < wmax)
                    stage<kReach>(A, R, S, T, imp[j], kReach ? (row[j] | (dir << 31)) : row[j],
                                  caux, ok_local, lane, C);
            }
        }
    }
    if (__any_sync(kFull, hub_repush))
        stage<kReach>(A, R, S, T, hub_repush, entry, kReach ? aux : (uint32_t)(prop - 1), false,
                      lane, C);
    // CSR rows: the wave's edges laid end to end, dealt 32 per step
    if (!__any_sync(kFull, deg != 0u)) return;
    const uint32_t incl = warp_incl_scan(deg, lane);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    if (deg) { C.expansions++; C.exp_verts++; C.exp_edges += deg; }
    __syncwarp();
    S.s_incl[lane] = incl;
    S.s_base[lane] = beg - (incl - deg);
    S.s_val[lane] = prop;
    S.s_dir[lane] = dir;
    S.s_aux[lane] = caux;
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32u * kU) {
        uint32_t w[kU], wd[kU], ca[kU];
        unsigned long long pv[kU];
        bool ok[kU], imp[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) {
            const uint32_t j = base + (uint32_t)u * 32u + (uint32_t)lane;
            ok[u] = j < total;
            w[u] = 0; wd[u] = 0; pv[u] = 0; ca[u] = 0;
            if (ok[u]) {
                uint32_t o = 0;
#pragma unroll
                for (uint32_t step = 16; step >= 1; step >>= 1)
                    if (S.s_incl[o + step - 1] <= j) o += step;
                wd[u] = S.s_dir[o];
                pv[u] = S.s_val[o];
                ca[u] = S.s_aux[o];
                // u32 sum first: s_base = row start - prefix may wrap
                const uint32_t e = S.s_base[o] + j;
                w[u] = __ldg(row_idx<kReach>(A, wd[u]) + e);
#ifdef PG_DEBUG_BOUNDS
                if (PG_DBG_ID(A, w[u], 4u, false) == PG_NONE) { ok[u] = false; w[u] = 0; }
#endif
            }
        }
        unsigned long long old[kU];
#pragma unroll
        for (int u = 0; u < kU; u++) old[u] = relax_issue<kReach>(A, w[u], wd[u], pv[u], ok[u]);
#pragma unroll
        for (int u = 0; u < kU; u++) imp[u] = ok[u] && improved<kReach>(pv[u], old[u]);
#pragma unroll
        for (int u = 0; u < kU; u++)
            stage<kReach>(A, R, S, T, imp[u], kReach ? (w[u] | (wd[u] << 31)) : w[u], ca[u],
                          eligible<kReach>(R, ca[u]), lane, C);
    }
    __syncwarp();
}

// Padded-row wave with one lane per (entry, slot): 32 / W entries per wave,
// entry i0 + lane / W reads slot lane % W of its row (W = the widest row of
// the two directions; a narrower direction leaves its upper slots idle).
// Each lane relaxes at most one arc and stages at most one child, so a
// sparse level costs a short path instead of W unrolled slots per lane.
// Entries whose list is in the CSR (long rows, or a direction without rows)
// are expanded afterwards, one per lane, by expand_wave.
template <bool kReach>
__device__ void expand_rows_sp(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                               const uint32_t *ents, const uint32_t *auxs, uint32_t i0,
                               uint32_t cnt, uint32_t lw, bool from_bag, int lane, Counters &C) {
    const uint32_t j = (uint32_t)lane & ((1u << lw) - 1u);
    const uint32_t i = i0 + ((uint32_t)lane >> lw);
    const bool valid = i < cnt;
    uint32_t ent = PG_NONE, aux = 0;
    if (valid) {
        ent = PG_DBG_ENTRY(A, ents[i], 8u, kReach);
        aux = auxs[i];
    }
    const bool live = ent != PG_NONE;
    const uint32_t v = kReach ? (ent & 0x7FFFFFFFu) : ent;
    const uint32_t dir = kReach ? (ent >> 31) : 0u;
    const uint32_t *ell = dir ? A.ell1 : A.ell0;
    const uint32_t Wd = dir ? A.ellw1 : A.ellw0;
    const bool has_rows = live && ell != nullptr;
    unsigned long long prop = 0;
    uint32_t x = PG_NONE;
    if (live) {
        prop = (!kReach && !from_bag) ? (unsigned long long)(aux + 1u) : load_prop<kReach>(A, v, dir);
        if (has_rows && j < Wd) x = __ldg(ell + (size_t)v * Wd + j);
#ifdef PG_DEBUG_BOUNDS
        if (x < 0x80000000u) x = PG_DBG_ID(A, x, 9u, false);
#endif
    }
    const bool dead = !kReach && prop == (unsigned long long)PG_INF;
    const bool lead = live && !dead && j == 0u;
    const bool is_long = lead && (!has_rows || x == PG_ELL_LONG);
    const uint32_t caux = kReach ? aux + 1u : (uint32_t)prop;
    const bool ok_local = eligible<kReach>(R, caux);
    const bool arc = live && !dead && x < 0x80000000u;
    const unsigned long long old = relax_issue<kReach>(A, x, dir, prop, arc);
    if (arc && ok_local) pg_prefetch_l1(ell + (size_t)x * Wd);
    const bool imp = arc && improved<kReach>(prop, old);
    if (lead && !is_long) { C.expansions++; C.exp_verts++; }
    if (arc) C.exp_edges++;
    stage<kReach>(A, R, S, T, imp, kReach ? (x | (dir << 31)) : x, caux, ok_local, lane, C);
    // rows kept in the CSR: lane t takes the t-th such entry
    const unsigned bl = __ballot_sync(kFull, is_long);
    if (bl) {
        unsigned mm = bl;
        for (int q = 0; q < lane && mm; q++) mm &= mm - 1u;
        const int src = mm ? __ffs(mm) - 1 : 0;
        const uint32_t e2 = __shfl_sync(kFull, ent, src);
        const uint32_t a2 = __shfl_sync(kFull, aux, src);
        expand_wave<kReach>(A, R, S, T, mm ? e2 : PG_NONE, a2, from_bag, lane, C);
    }
}

// One level of the CTA's reachability search over padded rows: the
// slot-parallel wave of expand_rows_sp (lane l takes entry l / W and slot
// l % W, W = the widest row of the two directions), with U groups of
// 32 / W entries per warp in flight: every mask and row read of the pass is
// issued before the first atomicOr, and every atomicOr before the first
// result is used.  Entries whose list is in the CSR (long rows, or a
// direction without rows) are expanded afterwards, one per lane, by
// expand_wave.
template <uint32_t LW, uint32_t U>
__device__ void reach_rows_level(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                                 const uint32_t *ents, const uint32_t *auxs, uint32_t ncur,
                                 bool from_bag, int lane, int wib, int nwib, Counters &C) {
    constexpr uint32_t W = 1u << LW, G = 32u >> LW;
    const uint32_t j = (uint32_t)lane & (W - 1u);
    const uint32_t gstride = (uint32_t)nwib * G;
    for (uint32_t w0 = (uint32_t)wib * G; w0 < ncur; w0 += gstride * U) {
        uint32_t ent[U], aux[U], x[U];
        unsigned long long prop[U], old[U];
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            const uint32_t i = w0 + u * gstride + ((uint32_t)lane >> LW);
            ent[u] = PG_NONE;
            aux[u] = 0;
            if (i < ncur) {
                ent[u] = PG_DBG_ENTRY(A, ents[i], 8u, true);
                aux[u] = auxs[i];
            }
        }
        // every mask and row read of the pass
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            prop[u] = 0;
            x[u] = PG_NONE;
            if (ent[u] != PG_NONE) {
                const uint32_t v = ent[u] & 0x7FFFFFFFu, dir = ent[u] >> 31;
                const uint32_t *ell = dir ? A.ell1 : A.ell0;
                const uint32_t Wd = dir ? A.ellw1 : A.ellw0;
                prop[u] = load_prop<true>(A, v, dir);
                if (ell != nullptr && j < Wd) x[u] = __ldg(ell + (size_t)v * Wd + j);
#ifdef PG_DEBUG_BOUNDS
                if (x[u] < 0x80000000u) x[u] = PG_DBG_ID(A, x[u], 9u, false);
#endif
            }
        }
        // every atomicOr of the pass
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            const bool arc = ent[u] != PG_NONE && x[u] < 0x80000000u;
            const uint32_t dir = ent[u] >> 31;
            old[u] = relax_issue<true>(A, x[u], dir, prop[u], arc);
            if (arc && aux[u] + 1u < R.tau) {
                const uint32_t *ell = dir ? A.ell1 : A.ell0;
                const uint32_t Wd = dir ? A.ellw1 : A.ellw0;
                pg_prefetch_l1(ell + (size_t)x[u] * Wd);
            }
        }
        // stage the improved children, then the lists kept in the CSR
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            const bool live = ent[u] != PG_NONE;
            const uint32_t dir = ent[u] >> 31;
            const bool has_rows = live && (dir ? A.ell1 : A.ell0) != nullptr;
            const bool lead = live && j == 0u;
            const bool is_long = lead && (!has_rows || x[u] == PG_ELL_LONG);
            const uint32_t caux = aux[u] + 1u;
            const bool arc = live && x[u] < 0x80000000u;
            const bool imp = arc && improved<true>(prop[u], old[u]);
            if (lead && !is_long) { C.expansions++; C.exp_verts++; }
            if (arc) C.exp_edges++;
            stage<true>(A, R, S, T, imp, x[u] | (dir << 31), caux, eligible<true>(R, caux), lane, C);
            const unsigned bl = __ballot_sync(kFull, is_long);
            if (bl) {
                unsigned mm = bl;
                for (int q = 0; q < lane && mm; q++) mm &= mm - 1u;
                const int src = mm ? __ffs(mm) - 1 : 0;
                const uint32_t e2 = __shfl_sync(kFull, ent[u], src);
                const uint32_t a2 = __shfl_sync(kFull, aux[u], src);
                expand_wave<true>(A, R, S, T, mm ? e2 : PG_NONE, a2, from_bag, lane, C);
            }
        }
    }
}

__device__ __forceinline__ uint32_t vt_slot(uint32_t v) { return (v * 0x9E3779B1u) >> (32u - kVtLog2); }
__device__ __forceinline__ unsigned long long vt_pack(uint32_t d, uint32_t v) {
    return ((unsigned long long)d << 32) | v;
}
// Filter slots are read and written by the CTA's threads concurrently, so
// both sides are relaxed CTA-scope accesses: single-copy atomic, a reader
// sees one whole (distance, vertex) pair, never halves of two.
__device__ __forceinline__ unsigned long long vt_get(const unsigned long long *vt, uint32_t v) {
    unsigned long long e;
    asm volatile("ld.relaxed.cta.shared.u64 %0, [%1];"
                 : "=l"(e)
                 : "r"((unsigned)__cvta_generic_to_shared(vt + vt_slot(v))));
    return e;
}
__device__ __forceinline__ void vt_put(unsigned long long *vt, uint32_t v, uint32_t d) {
    asm volatile("st.relaxed.cta.shared.u64 [%0], %1;"
                 :
                 : "r"((unsigned)__cvta_generic_to_shared(vt + vt_slot(v))), "l"(vt_pack(d, v))
                 : "memory");
}

// One level of the CTA's BFS local search over forward padded rows of width
// W = 2^LW.  Its latency is one dependent chain per warp pass: entry (shared
// memory), row read, atomicMin, append.  To keep the passes few, an entry
// takes NL = 2^LS lanes (NL <= W; lane j reads slots j, j + NL, ... of the
// row, coalesced), and a warp holds U groups of 32 / NL entries in flight:
// every row read of the pass is issued before the first atomicMin and every
// atomicMin before the first result is used, so a pass over up to
// U * 32 / NL entries per warp costs about one row read and one atomic round
// trip.  The children inside the window go to the CTA's next level with one
// warp scan and one shared-memory atomic per pass; the others go to the
// warp's spill staging.  Entries whose list is in the CSR (every slot marked
// PG_ELL_LONG) are expanded afterwards, one per lane, by expand_wave.
template <uint32_t LW, uint32_t LS, uint32_t U>
__device__ void bfs_rows_level(const TravArgs &A, const Round &R, const WarpSm &S, Task &T,
                               const uint32_t *ents, const uint32_t *auxs, uint32_t ncur,
                               bool from_bag, int lane, int wib, int nwib, Counters &C,
                               unsigned long long *vt) {
    constexpr uint32_t W = 1u << LW, NL = 1u << LS, SL = W >> LS, G = 32u >> LS;
    static_assert(LS <= LW && SL * U <= 8u, "at most 8 arcs per lane and pass");
    const uint32_t j = (uint32_t)lane & (NL - 1u);
    const uint32_t win = R.Lbase + R.tau;  // children at distance < win stay in the CTA
    const uint32_t *ell = A.ell0;
    const uint32_t gstride = (uint32_t)nwib * G;  // entries per CTA-wide group
    for (uint32_t w0 = (uint32_t)wib * G; w0 < ncur; w0 += gstride * U) {
        uint32_t v[U], nd[U], aux[U];
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            const uint32_t i = w0 + u * gstride + ((uint32_t)lane >> LS);
            v[u] = PG_NONE;
            aux[u] = 0;
            nd[u] = PG_INF;
            if (i < ncur) {
                v[u] = PG_DBG_ENTRY(A, ents[i], 10u, false);
                aux[u] = auxs[i];
            }
        }
#pragma unroll
        for (uint32_t u = 0; u < U; u++)
            if (v[u] != PG_NONE) {
                // a local-search entry carries its distance; a bag entry reads it
                const uint32_t d = from_bag ? pg_ldcg(A.dist + v[u]) : aux[u];
                nd[u] = (d == PG_INF) ? PG_INF : d + 1u;
                if (from_bag && vt && d != PG_INF) vt_put(vt, v[u], d);
            }
        // every row read of the pass, then every atomicMin
        uint32_t x[U][SL];
#pragma unroll
        for (uint32_t u = 0; u < U; u++)
#pragma unroll
            for (uint32_t s = 0; s < SL; s++) {
                x[u][s] = PG_NONE;
                if (nd[u] != PG_INF) x[u][s] = __ldg(ell + (size_t)v[u] * W + s * NL + j);
#ifdef PG_DEBUG_BOUNDS
                if (x[u][s] < 0x80000000u) x[u][s] = PG_DBG_ID(A, x[u][s], 11u, false);
#endif
            }
        // an arc into a vertex this CTA settled at a distance <= nd cannot
        // improve it (distances only decrease): no atomic
        bool go[U][SL];
#pragma unroll
        for (uint32_t u = 0; u < U; u++)
#pragma unroll
            for (uint32_t s = 0; s < SL; s++) {
                go[u][s] = x[u][s] < 0x80000000u;  // not padding, not a CSR-row marker
                if (vt && go[u][s]) {
                    const unsigned long long e = vt_get(vt, x[u][s]);
                    go[u][s] = !((uint32_t)e == x[u][s] && (uint32_t)(e >> 32) <= nd[u]);
                }
            }
        uint32_t old[U][SL];
#pragma unroll
        for (uint32_t u = 0; u < U; u++)
#pragma unroll
            for (uint32_t s = 0; s < SL; s++) {
                old[u][s] = 0;
                if (go[u][s]) {
                    old[u][s] = atomicMin(A.dist + x[u][s], nd[u]);
                    if (nd[u] < win) pg_prefetch_l1(ell + (size_t)x[u][s] * W);
                }
            }
        // improved children: inside the window -> next level, else spill.
        // Bit k = u * SL + s of a lane's masks is arc (u, s); one ballot per
        // bit gives every arc's rank, and one shared-memory atomic per pass
        // reserves the warp's places in the next level.
        constexpr uint32_t K = U * SL;
        const unsigned lt = pg_lanemask_lt();
        uint32_t locm = 0, impm = 0;
        bool is_long[U];
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            const bool live = nd[u] != PG_INF;
            is_long[u] = live && j == 0u && x[u][0] == PG_ELL_LONG;
            if (live && j == 0u && !is_long[u]) { C.expansions++; C.exp_verts++; }
#pragma unroll
            for (uint32_t s = 0; s < SL; s++) {
                const bool arc = x[u][s] < 0x80000000u;
                if (arc) C.exp_edges++;
                const bool imp = arc && nd[u] < old[u][s];
                if (imp && vt) vt_put(vt, x[u][s], nd[u]);
                impm |= (imp ? 1u : 0u) << (u * SL + s);
                locm |= (imp && nd[u] < win ? 1u : 0u) << (u * SL + s);
            }
        }
        unsigned bal[K];
        uint32_t tot = 0;
#pragma unroll
        for (uint32_t k = 0; k < K; k++) {
            bal[k] = __ballot_sync(kFull, (locm >> k) & 1u);
            tot += (uint32_t)__popc(bal[k]);
        }
        uint32_t spm = impm & ~locm;  // spilled arcs of this lane
        if (tot) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(T.cta_n, tot);
            base = __shfl_sync(kFull, base, 0);
#pragma unroll
            for (uint32_t k = 0; k < K; k++) {
                if ((locm >> k) & 1u) {
                    const uint32_t p = base + (uint32_t)__popc(bal[k] & lt);
                    if (p < T.cta_cap) {
                        T.cta_ent[p] = x[k / SL][k % SL];
                        T.cta_aux[p] = nd[k / SL];
                    } else {
                        spm |= 1u << k;  // the level buffer is full
                    }
                }
                base += (uint32_t)__popc(bal[k]);
            }
        }
        // children beyond the window (or overflow): the warp's spill staging
        if (__any_sync(kFull, spm != 0u)) {
            unsigned sb[K];
            uint32_t stot = 0;
#pragma unroll
            for (uint32_t k = 0; k < K; k++) {
                sb[k] = __ballot_sync(kFull, (spm >> k) & 1u);
                stot += (uint32_t)__popc(sb[k]);
            }
            if (T.nsp + stot > kSpillCap) flush_spill<false>(A, R, S, T, lane, C);
            uint32_t q = T.nsp;
#pragma unroll
            for (uint32_t k = 0; k < K; k++) {
                if ((spm >> k) & 1u) {
                    const uint32_t p = q + (uint32_t)__popc(sb[k] & lt);
                    S.sp[p] = x[k / SL][k % SL];
                    S.spa[p] = nd[k / SL];
                }
                q += (uint32_t)__popc(sb[k]);
            }
            T.nsp = q;
        }
        // lists kept in the CSR: lane t takes the t-th such entry
#pragma unroll
        for (uint32_t u = 0; u < U; u++) {
            const unsigned bll = __ballot_sync(kFull, is_long[u]);
            if (bll) {
                unsigned mm = bll;
                for (int q = 0; q < lane && mm; q++) mm &= mm - 1u;
                const int src = mm ? __ffs(mm) - 1 : 0;
                const uint32_t e2 = __shfl_sync(kFull, v[u], src);
                const uint32_t a2 = __shfl_sync(kFull, aux[u], src);
                expand_wave<false>(A, R, S, T, mm ? e2 : PG_NONE, a2, from_bag, lane, C);
            }
        }
    }
}

// One warp task: c frontier entries plus the local search they start.
template <bool kReach>
__device__ void run_task(const TravArgs &A, const Round &R, const WarpSm &S, uint32_t entry,
                         uint32_t c, int lane, Counters &C) {
    Task T;
    task_init(T, (R.tau > 1u) ? c * R.tau * 8u : 0u);
    uint32_t aux = 0;
    bool from_bag = true;
    for (;;) {
        expand_wave<kReach>(A, R, S, T, entry, aux, from_bag, lane, C);
        const uint32_t avail = T.qtail - T.qhead;
        if (avail == 0) break;
        const uint32_t take = min(32u, avail);
        __syncwarp();
        const uint32_t p = (T.qhead + lane) & (A.L.qcap - 1);
        entry = ((uint32_t)lane < take) ? S.lq[p] : PG_NONE;
        entry = PG_DBG_ENTRY(A, entry, 2u, kReach);
        aux = ((uint32_t)lane < take) ? S.lqa[p] : 0u;
        T.qhead += take;
        from_bag = false;
        __syncwarp();
    }
    flush_spill<kReach>(A, R, S, T, lane, C);
}

// CTA-cooperative local search for one round (tau > 1): the CTA takes a
// share of the frontier (static first, then grabbed), and runs it level by
// level for up to tau levels: all warps split each level, children inside
// the window go to the CTA's next-level buffer in shared memory, the rest
// (and any overflow) spill to the next bag.  Levels are separated by a CTA
// barrier, so the CTA's local search is itself breadth-first.
//
// Multiple frontiers (PG_VGC_BUCKETS; Sec. 2.2, the BFS paragraph): the
// CTA's level buffer at depth 2^i is its frontier i, the vertices 2^i hops
// from the round's frontier.  The round's local search is cut into phases
// at depths 1, 2, 4, ... < tau with a grid barrier between phases, so no
// frontier i is expanded before every CTA has finished the frontiers
// nearer than it: a CTA can run ahead of the slowest one by at most the
// current phase's width, which limits the vertices expanded with a distance
// that another CTA then shortens ("unready" vertices).  Every CTA takes at
// most one share (rounds with more entries than the CTAs' level buffers run
// unphased) and passes every phase barrier, with or without entries.
// Returns false when a barrier gave up (timeout).
template <bool kReach>
__device__ bool cta_round(const TravArgs &A, const Round &R, const WarpSm &S, const CtaSm &Q,
                          int lane, int wib, int nwib, Counters &C, unsigned &gen, int *s_flag) {
    const uint32_t nb = gridDim.x;
    const uint32_t QC = A.L.cta_queue;
    // slot-parallel waves when padded rows exist: log2 of the widest row
    const uint32_t wmax = max(A.ellw0, A.ellw1);
    const uint32_t lw = wmax >= 16u ? 4u : (wmax >= 8u ? 3u : (wmax >= 4u ? 2u : 0u));
    uint32_t cc = (R.F + nb - 1) / nb;
    cc = max(1u, min(cc, QC / 2));
    const uint32_t span = nb * cc;
    const bool phased = A.L.vgc == PG_VGC_BUCKETS && R.F <= span;
    bool ok = true;
    Task T;
    task_init(T, 0);
    for (uint32_t base = blockIdx.x * cc;;) {
        if (base >= R.F && !phased) break;
        const uint32_t c = (base < R.F) ? min(cc, R.F - base) : 0u;
        for (uint32_t i = threadIdx.x; i < c; i += blockDim.x) {
            uint32_t e = __ldcg(A.bag + (size_t)R.cur * A.cap + base + i);
            e = PG_DBG_ENTRY(A, e, 7u, kReach);
            Q.ent[0][i] = e;
            Q.aux[0][i] = 0u;
        }
        if (threadIdx.x == 0) {
            Q.n[0] = c;
            Q.n[1] = 0;
            Q.n[2] = 0;
        }
        __syncthreads();
        // level h reads buffer h%3 and appends to (h+1)%3; buffer (h+2)%3 was
        // last touched in level h-1, so it is cleared here for level h+1,
        // and one CTA barrier per level suffices
        for (uint32_t h = 0;; h++) {
            // phases: every CTA passes the barriers at depths 1, 2, 4, ... < tau
            const bool in_phases = phased && h < R.tau;
            if (in_phases && h > 0u && (h & (h - 1u)) == 0u &&
                !pg_grid_sync(A.ctrl, gridDim.x, gen, A.L.timeout_ns, s_flag)) {
                ok = false;
                break;
            }
            const uint32_t cl = h % 3u, nl = (h + 1u) % 3u, ql = (h + 2u) % 3u;
            const uint32_t ncur = min(Q.n[cl], QC);
            if (ncur == 0 && !in_phases) break;
            T.cta_ent = Q.ent[nl];
            T.cta_aux = Q.aux[nl];
            T.cta_n = &Q.n[nl];
            T.cta_cap = QC;
            if (!kReach && A.ellw0 != 0u) {
                // BFS reads the forward rows only: the lean level of width ellw0
                // one group in flight per warp when that covers the level
                const bool one = ncur <= (uint32_t)nwib * (32u >> (A.ellw0 == 4u ? 2u : 3u));
                if (A.ellw0 == 4u) {
                    if (one) bfs_rows_level<2, 2, 1>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C, Q.vt);
                    else bfs_rows_level<2, 2, 2>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C, Q.vt);
                } else if (A.ellw0 == 8u) {
                    if (one) bfs_rows_level<3, 3, 1>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C, Q.vt);
                    else bfs_rows_level<3, 3, 2>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C, Q.vt);
                } else {
                    if (one) bfs_rows_level<4, 3, 1>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C, Q.vt);
                    else bfs_rows_level<4, 3, 2>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C, Q.vt);
                }
            } else if (kReach && lw) {
                // reachability: two entry groups in flight per warp
                if (lw == 2u)
                    reach_rows_level<2, 2>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C);
                else if (lw == 3u)
                    reach_rows_level<3, 2>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C);
                else
                    reach_rows_level<4, 2>(A, R, S, T, Q.ent[cl], Q.aux[cl], ncur, h == 0, lane, wib, nwib, C);
            } else if (lw) {
                const uint32_t G = 32u >> lw;  // entries per slot-parallel wave
                for (uint32_t w0 = (uint32_t)wib * G; w0 < ncur; w0 += (uint32_t)nwib * G)
                    expand_rows_sp<kReach>(A, R, S, T, Q.ent[cl], Q.aux[cl], w0, ncur, lw, h == 0, lane, C);
            } else {
                for (uint32_t w0 = (uint32_t)wib * 32u; w0 < ncur; w0 += (uint32_t)nwib * 32u) {
                    const uint32_t i = w0 + lane;
                    const uint32_t e = (i < ncur) ? Q.ent[cl][i] : PG_NONE;
                    const uint32_t ax = (i < ncur) ? Q.aux[cl][i] : 0u;
                    expand_wave<kReach>(A, R, S, T, e, ax, h == 0, lane, C);
                }
            }
            if (threadIdx.x == 0) Q.n[ql] = 0;
            __syncthreads();
        }
        T.cta_n = nullptr;
        flush_spill_cta<kReach>(A, R, S, T, Q.wcnt, lane, C);
        if (R.F <= span || !ok) break;
        if (threadIdx.x == 0) *Q.task = span + atomicAdd(&R.sc->head, cc);
        __syncthreads();
        base = *Q.task;
        __syncthreads();
    }
    return ok;
}

// Edges of listed hubs, dealt in chunks of `hch` edges (hch <= hub_degree, so
// a chunk touches at most two hubs).  Improvements go to the next bag.
template <bool kReach>
__device__ void hub_edges(const TravArgs &A, const Round &R, const WarpSm &S, int lane,
                          Counters &C) {
    const unsigned long long hp = R.hub_pack;
    const uint32_t hcount = min((uint32_t)(hp >> 40), A.hcap);
    const uint32_t hedges = (uint32_t)(hp & kMask40);
    if (hcount == 0) return;
    const uint32_t hch = min(1024u, A.L.hub_degree);
    const PgHub *H = A.hubs + (size_t)R.cur * A.hcap;
    Task T;
    task_init(T, 0);
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
        uint32_t hs[2], hb[2], hd[2], hdeg[2];
        unsigned long long hpv[2];
        for (int t = 0; t < 2; t++) {
            hs[t] = PG_INF; hb[t] = 0; hd[t] = 0; hpv[t] = 0; hdeg[t] = 0;
            const uint32_t i = lo + t;
            if (i < hcount) {
                const uint32_t e = __ldcg(&H[i].v);
                hs[t] = __ldcg(&H[i].start);
                const uint32_t hv = kReach ? (e & 0x7FFFFFFFu) : e;
                hd[t] = kReach ? (e >> 31) : 0u;
                hb[t] = __ldg(row_off<kReach>(A, hd[t]) + hv);
                hdeg[t] = __ldg(row_off<kReach>(A, hd[t]) + hv + 1) - hb[t];
                hpv[t] = load_prop<kReach>(A, hv, hd[t]);
            }
        }
        if (lane == 0) C.expansions += (hs[1] < a + len) ? 2 : 1;
        for (uint32_t t0 = 0; t0 < len; t0 += 32u * kU) {
            uint32_t w[kU], wd[kU];
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
#ifdef PG_DEBUG_BOUNDS
                        if (PG_DBG_ID(A, w[u], 5u, false) == PG_NONE) { go[u] = false; w[u] = 0; }
#endif
                    }
                }
            }
            unsigned long long old[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) old[u] = relax_issue<kReach>(A, w[u], wd[u], pv[u], go[u]);
#pragma unroll
            for (int u = 0; u < kU; u++) go[u] = go[u] && improved<kReach>(pv[u], old[u]);
#pragma unroll
            for (int u = 0; u < kU; u++)
                stage<kReach>(A, R, S, T, go[u], kReach ? (w[u] | (wd[u] << 31)) : w[u],
                              kReach ? 1u : (uint32_t)pv[u], false, lane, C);
        }
    }
    flush_spill<kReach>(A, R, S, T, lane, C);
}

// Bottom-up round at settled level L (BFS only): every vertex with
// dist > L + 1 looks for an in-neighbour at distance L and takes L + 1;
// bag entries still above L stay active.
__device__ void pull_round(const TravArgs &A, const Round &R, const WarpSm &S, uint32_t Lvl,
                           int lane, uint32_t gwarp, uint32_t nwarps, Counters &C) {
    const uint32_t n = A.G.n;
    const uint32_t target = Lvl + 1u;
    Task T;
    task_init(T, 0);
    const uint32_t W = A.ellw1;
    for (uint32_t base = gwarp * 32u; base < n; base += nwarps * 32u) {
        const uint32_t v = base + lane;
        bool found = false;
        if (v < n) {
            const uint32_t d = pg_ldcg(A.dist + v);
            if (d > target) {
                bool use_csr = true;
                if (A.ell1 != nullptr) {
                    const uint4 *rp = reinterpret_cast<const uint4 *>(A.ell1 + (size_t)v * W);
                    uint32_t row[kMaxW];
#pragma unroll
                    for (int j = 0; j < (int)kMaxW; j++) row[j] = PG_NONE;
#pragma unroll
                    for (int q = 0; q < (int)(kMaxW / 4); q++) {
                        if ((uint32_t)q * 4u < W) {
                            const uint4 t = __ldg(rp + q);
                            row[4 * q] = t.x; row[4 * q + 1] = t.y; row[4 * q + 2] = t.z;
                            row[4 * q + 3] = t.w;
                        }
                    }
                    if (row[0] != PG_ELL_LONG) {
                        use_csr = false;
#pragma unroll
                        for (int j = 0; j < (int)kMaxW; j++)
                            if ((uint32_t)j < W && row[j] < 0x80000000u &&
                                pg_ldcg(A.dist + row[j]) == Lvl)
                                found = true;
                    }
                }
                if (use_csr) {
                    const uint32_t b = __ldg(A.G.toff + v), e = __ldg(A.G.toff + v + 1);
                    for (uint32_t q = b; q < e; q++) {
                        if (pg_ldcg(A.dist + __ldg(A.G.tidx + q)) == Lvl) { found = true; break; }
                    }
                }
                if (found) A.dist[v] = target;
            }
        }
        if (__any_sync(kFull, found)) stage<false>(A, R, S, T, found, v, target, false, lane, C);
    }
    for (uint32_t base = gwarp * 32u; base < R.F; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        uint32_t v = 0, d = 0;
        bool keep = false;
        if (i < R.F) {
            v = __ldcg(A.bag + (size_t)R.cur * A.cap + i);
            v = PG_DBG_ENTRY(A, v, 6u, false);
            if (v != PG_NONE) {
                d = pg_ldcg(A.dist + v);
                keep = d > Lvl;
            } else {
                v = 0;
            }
        }
        if (__any_sync(kFull, keep)) stage<false>(A, R, S, T, keep, v, d, false, lane, C);
    }
    flush_spill<false>(A, R, S, T, lane, C);
}

__device__ __forceinline__ void reset_slot(PgSlot *s) {
    s->size = 0;
    s->head = 0;
    s->hub_cursor = 0;
    s->min_level = PG_INF;
    s->max_level = 0;
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
// The network's choice, judged against the fixed-tau push action a_fix: the
// network overrides it only when its predicted gain (standardised log2
// kernel-time units) exceeds a margin, so near-ties keep the fixed heuristic.
// Raising tau or pulling needs kJudgeUp; lowering tau, which adds rounds,
// needs the stronger evidence kJudgeDown.
constexpr float kJudgeUp = 0.1f;
constexpr float kJudgeDown = 0.3f;

__device__ uint32_t mlp_decide(const float *W, const float (&x)[5], bool allow_pull, uint32_t a_fix,
                               int lane) {
    // packed order W1 (32 x 5), b1, W2 (32 x 32), b2, W3 (8 x 32), b3; W2 and
    // W3 were stored transposed when the CTA loaded them
    const float *W1 = W, *b1 = W + 160, *W2t = W + 192, *b2 = W + 1216, *W3t = W + 1248,
                *b3 = W + 1504;
    float h1 = b1[lane];
#pragma unroll
    for (int i = 0; i < 5; i++) h1 = fmaf(W1[lane * 5 + i], x[i], h1);
    h1 = fmaxf(h1, 0.f);
    float h2 = b2[lane];
#pragma unroll
    for (int i = 0; i < 32; i++) h2 = fmaf(W2t[i * 32 + lane], __shfl_sync(kFull, h1, i), h2);
    h2 = fmaxf(h2, 0.f);
    const int a = lane & 7;
    float y = b3[a];
#pragma unroll
    for (int i = 0; i < 32; i++) y = fmaf(W3t[i * 8 + a], __shfl_sync(kFull, h2, i), y);
    uint32_t best = 0;
    float by = __shfl_sync(kFull, y, 0);
    for (int t = 1; t < (int)PG_NUM_ACTIONS; t++) {
        const float yt = __shfl_sync(kFull, y, t);
        if ((uint32_t)t == PG_ACTION_PULL && !allow_pull) continue;
        if (yt > by) { by = yt; best = (uint32_t)t; }
    }
    const float yf = __shfl_sync(kFull, y, (int)a_fix);
    return (by - yf > (best < a_fix ? kJudgeDown : kJudgeUp)) ? best : a_fix;
}

__device__ __forceinline__ float flog2p1(float x) { return log2f(1.0f + x); }

// The round-index feature saturates at 2^14 rounds: the training states never
// go further (strips are sampled up to about 17k rounds), and the network is
// not evaluated outside that range.
constexpr uint32_t kRoundFeatureCap = 1u << 14;

// Whether the settled-vertex filter has room beside the CTA level buffers.
__host__ __device__ __forceinline__ bool vt_enabled(const PgLaunch &L) {
    return L.vgc != PG_VGC_WARP && L.cta_queue <= kVtMaxQueue;
}

// Per-warp FIFO words (entry + aux per slot): only the warp local search
// uses the FIFO, so the CTA local search leaves it out of shared memory.
__host__ __device__ __forceinline__ uint32_t warp_fifo_words(const PgLaunch &L) {
    return L.vgc == PG_VGC_WARP ? L.qcap : 0u;
}

template <bool kReach>
__global__ void __launch_bounds__(512, 1) pg_traverse_kernel(const TravArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int nwib = blockDim.x >> 5;
    const uint32_t gwarp = blockIdx.x * nwib + wib;
    const uint32_t nwarps = gridDim.x * nwib;
    const uint32_t nblocks = gridDim.x;

    // shared memory: MLP weights, then per warp: s_val[32] (u64), 4 x [32]
    // u32 wave arrays, spill staging 2 x [kSpillCap], local FIFO 2 x [qcap]
    // (the per-warp FIFO is used by the warp local search only)
    float *s_w = reinterpret_cast<float *>(smem);
    unsigned long long *s_val_all = reinterpret_cast<unsigned long long *>(smem + 6144);
    uint32_t *s_u32 = reinterpret_cast<uint32_t *>(smem + 6144 + nwib * 256);
    const uint32_t per_warp = 4u * 32u + 2u * kSpillCap + 2u * warp_fifo_words(A.L);
    uint32_t *mine = s_u32 + (size_t)wib * per_warp;
    WarpSm S;
    S.s_val = s_val_all + wib * 32;
    S.s_incl = mine;
    S.s_base = mine + 32;
    S.s_dir = mine + 64;
    S.s_aux = mine + 96;
    S.sp = mine + 128;
    S.spa = S.sp + kSpillCap;
    S.lq = S.spa + kSpillCap;
    S.lqa = S.lq + A.L.qcap;
    CtaSm Q;
    {
        uint32_t *cta = s_u32 + (size_t)nwib * per_warp;
        for (int b = 0; b < 3; b++) {
            Q.ent[b] = cta + (uint32_t)(2 * b) * A.L.cta_queue;
            Q.aux[b] = cta + (uint32_t)(2 * b + 1) * A.L.cta_queue;
        }
        Q.n = cta + 6u * A.L.cta_queue;
        Q.task = Q.n + 3;
        // the filter follows the level buffers (8-byte aligned: every region
        // before it is a multiple of 8 bytes)
        Q.vt = (!kReach && A.ellw0 != 0u && vt_enabled(A.L))
                   ? reinterpret_cast<unsigned long long *>(Q.n + 4) : nullptr;
        if (Q.vt)
            for (uint32_t i = threadIdx.x; i < (1u << kVtLog2); i += blockDim.x) Q.vt[i] = ~0ull;
    }
    __shared__ unsigned s_wcnt[17];
    Q.wcnt = s_wcnt;
    __shared__ CtaStat s_cs;
    if (threadIdx.x == 0) {
        s_cs.exp_edges = 0;
        s_cs.out_edges = 0;
        s_cs.exp_verts = 0;
        s_cs.min_level = PG_INF;
        s_cs.max_level = 0;
    }

    // the network runs in CTA 0 only (see the round-end decision below)
    if (A.L.schedule == PG_SCHED_LEARNED && blockIdx.x == 0)
        for (int i = threadIdx.x; i < (int)PG_MLP_NPARAMS; i += blockDim.x) {
            // W2 (32 x 32) and W3 (8 x 32) are stored transposed, so that in
            // mlp_decide the lanes read consecutive words (no bank conflicts)
            int j = i;
            if (i >= 192 && i < 1216) j = 192 + ((i - 192) & 31) * 32 + (i - 192) / 32;
            else if (i >= 1248 && i < 1504) j = 1248 + ((i - 1248) & 31) * 8 + (i - 1248) / 32;
            s_w[j] = A.L.weights[i];
        }

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
            if (A.dir & PG_FWD) A.mask0[v] = bits;
            if (A.dir & PG_BWD) A.mask1[v] = bits;
        }
    }
    // the fixed schedule's push action: tau = 2^a_fix (rounded down, at most 64)
    const uint32_t a_fix = min(31u - (uint32_t)__clz((int)max(A.L.tau, 1u)), 6u);
    __shared__ unsigned long long s_init[2];  // CTA 0: size and out-edges of the first bag
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
                if (A.hubs_possible && dg >= A.L.hub_degree) {
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
        s0->max_level = 0;
        s0->out_edges = oe;
        s_init[0] = cnt;
        s_init[1] = oe;
    }
    // learned schedule, round 0: CTA 0 built the first bag, so it knows round
    // 0's inputs already and picks round 0's action before the first barrier
    // (later rounds: at the end of the previous round, below)
    if (A.L.schedule == PG_SCHED_LEARNED && blockIdx.x == 0) {
        __syncthreads();
        if (wib == 0) {
            const float F0 = (float)s_init[0], E0 = (float)s_init[1];
            const float x0[5] = {flog2p1(F0) / 24.f, flog2p1(E0) / 32.f, flog2p1(E0 / F0) / 8.f,
                                 flog2p1(0.f) / 24.f, flog2p1(0.f) / 16.f};
            const uint32_t a = mlp_decide(s_w, x0, (!kReach) && A.L.allow_pull, a_fix, lane);
            if (lane == 0) ctrl->next_action = a;
        }
    }
    if (A.L.stall_block == blockIdx.x) return;  // fault injection: never arrive
    if (!pg_grid_sync(ctrl, nblocks, gen, tmo, &s_flag)) return;

    Counters C;
    const unsigned long long t_start = pg_gtimer();
    // whole-launch limit: 16 x the per-wait limit, checked once per round
    const unsigned long long t_deadline = t_start + 16ull * tmo;
    const float avg_deg = (float)A.G.m / (float)max(n, 1u);
    unsigned long long edges_seen = 0;
    bool pull_state = false;
    bool prev_plain = true;   // the initial bag is a single level
    uint32_t pull_rounds = 0;
    uint32_t r = 0;
    unsigned long long t_round = 0;
    // the round's control words, read once per CTA (thread 0) and shared
    __shared__ unsigned long long s_in[5];
    __shared__ uint32_t s_in32[5];
    for (;; r++) {
        Round R;
        R.cur = r & 1u;
        R.nxt = R.cur ^ 1u;
        R.sc = &ctrl->slot[r % PG_NUM_SLOTS];
        R.sn = &ctrl->slot[(r + 1) % PG_NUM_SLOTS];
        R.cs = &s_cs;
        R.tag = A.L.epoch + r + 1u;
        if (threadIdx.x == 0) {
            s_in32[0] = __ldcg(&R.sc->size);
            s_in32[1] = __ldcg(&R.sc->min_level);
            s_in32[2] = __ldcg(&R.sc->max_level);
            s_in[0] = pg_ldcg64(&R.sc->out_edges);
            s_in[1] = pg_ldcg64(&R.sc->hub_pack);
            s_in32[3] = (r > 0) ? __ldcg(&ctrl->exp_verts[(r - 1) & 3]) : 0u;
            s_in32[4] = __ldcg(&ctrl->next_action);
            s_in[2] = (r > 0) ? pg_ldcg64(&ctrl->exp_edges[(r - 1) & 3]) : 0ull;
            s_in[3] = (r >= 2) ? pg_ldcg64(&ctrl->round_t[(r - 1) & 3]) : 0ull;
            s_in[4] = (r >= 2) ? pg_ldcg64(&ctrl->round_t[(r - 2) & 3]) : 0ull;
        }
        __syncthreads();
        R.F = s_in32[0];
        const unsigned long long E_exact = s_in[0];
        const uint32_t Lvl = s_in32[1];
        const uint32_t Lmax = s_in32[2];
        R.hub_pack = s_in[1];
        R.Lbase = Lvl;
        if (R.F == 0) break;
        if ((A.L.max_rounds && r >= A.L.max_rounds) || R.tag == 0u || R.F > A.cap) {
            if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&ctrl->status, PG_DEV_OVERFLOW);
            break;
        }
        // out-edges of F: exact when counted at append time, else F times the
        // mean degree of the vertices expanded in the previous round
        unsigned long long E = E_exact;
        if (!A.need_deg && r > 0) {
            const unsigned ev = s_in32[3];
            const unsigned long long ee = s_in[2];
            const float md = ev ? (float)ee / (float)ev : avg_deg;
            E = (unsigned long long)((float)R.F * md + 0.5f);
        }
        // previous-round time as published by CTA 0 (visible one round late)
        const unsigned long long prev_ns = (r >= 2) ? s_in[3] - s_in[4] : 0ull;
        float x[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if ((A.L.schedule == PG_SCHED_LEARNED || A.L.trace != nullptr) && blockIdx.x == 0) {
            x[0] = flog2p1((float)R.F) / 24.f;
            x[1] = flog2p1((float)E) / 32.f;
            x[2] = flog2p1((float)E / (float)R.F) / 8.f;
            x[3] = flog2p1((float)min(r, kRoundFeatureCap)) / 24.f;
            x[4] = flog2p1((float)prev_ns * 1e-3f) / 16.f;
        }

        // ---- schedule decision (identical in every CTA)
        const bool can_pull = (!kReach) && A.L.allow_pull && Lvl != PG_INF;
        uint32_t action;
        if (A.L.schedule == PG_SCHED_LEARNED) {
            // chosen by CTA 0 at the end of the previous round from that
            // round's features (round 0: from round 0's, before the first barrier)
            action = s_in32[4];
            if (action >= PG_NUM_ACTIONS || (action == PG_ACTION_PULL && !can_pull)) action = a_fix;
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
        // A plain push round on a bag whose entries all carry the same
        // distance, right after a plain push round, improves each vertex at
        // most once: no de-duplication tags needed.
        const bool plain_now = !pull && R.tau == 1u;
        R.dedupe = kReach || !(plain_now && prev_plain && Lvl == Lmax);
        prev_plain = plain_now;
        edges_seen += E;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            reset_slot(&ctrl->slot[(r + 2) % PG_NUM_SLOTS]);
            ctrl->exp_edges[(r + 2) & 3] = 0;
            ctrl->exp_verts[(r + 2) & 3] = 0;
            t_round = pg_gtimer();
            ctrl->round_t[r & 3] = t_round;
            if (t_round > t_deadline) atomicOr(&ctrl->status, PG_DEV_TIMEOUT);
        }

        // ---- round work
        if (pull) {
            pull_round(A, R, S, Lvl, lane, gwarp, nwarps, C);
            pull_rounds++;
        } else if (R.tau > 1u && A.L.vgc != PG_VGC_WARP) {
            if (!cta_round<kReach>(A, R, S, Q, lane, wib, nwib, C, gen, &s_flag)) break;
            hub_edges<kReach>(A, R, S, lane, C);
        } else {
            // first task of every warp assigned statically, the rest grabbed
            const uint32_t span = nwarps * A.L.chunk;
            for (uint32_t base = gwarp * A.L.chunk;;) {
                if (base >= R.F) break;
                const uint32_t c = min(A.L.chunk, R.F - base);
                uint32_t entry =
                    ((uint32_t)lane < c) ? __ldcg(A.bag + (size_t)R.cur * A.cap + base + lane)
                                         : PG_NONE;
                entry = PG_DBG_ENTRY(A, entry, 1u, kReach);
                run_task<kReach>(A, R, S, entry, c, lane, C);
                if (R.F <= span) break;
                uint32_t b = 0;
                if (lane == 0) b = atomicAdd(&R.sc->head, A.L.chunk);
                base = span + __shfl_sync(kFull, b, 0);
            }
            hub_edges<kReach>(A, R, S, lane, C);
        }
        // expansion statistics of this round (mean degree for the next round)
        {
            const unsigned long long ee = warp_sum64(C.exp_edges);
            const unsigned long long ev = warp_sum64((unsigned long long)C.exp_verts);
            if (lane == 0 && ev) {
                atomicAdd(&s_cs.exp_edges, ee);
                atomicAdd(&s_cs.exp_verts, (unsigned)ev);
            }
            C.exp_edges = 0;
            C.exp_verts = 0;
        }
        // learned schedule: CTA 0's warp 0 picks the next round's action from
        // this round's features while it waits for the slowest CTA; the
        // barrier below publishes it with the round's other control words
        if (A.L.schedule == PG_SCHED_LEARNED && blockIdx.x == 0 && wib == 0) {
            const uint32_t a = mlp_decide(s_w, x, (!kReach) && A.L.allow_pull, a_fix, lane);
            if (lane == 0) ctrl->next_action = a;
        }
        // the CTA's aggregates reach the global counters before its arrival
        PgSlot *sn = R.sn;
        const uint32_t rr = r & 3;
        const bool ok = pg_grid_sync_then(ctrl, nblocks, gen, tmo, &s_flag, [&] {
            if (s_cs.exp_verts) {
                atomicAdd(&ctrl->exp_edges[rr], s_cs.exp_edges);
                atomicAdd(&ctrl->exp_verts[rr], s_cs.exp_verts);
            }
            if (s_cs.out_edges) atomicAdd(&sn->out_edges, s_cs.out_edges);
            if (s_cs.min_level != PG_INF) {
                atomicMin(&sn->min_level, s_cs.min_level);
                atomicMax(&sn->max_level, s_cs.max_level);
            }
            s_cs.exp_edges = 0;
            s_cs.out_edges = 0;
            s_cs.exp_verts = 0;
            s_cs.min_level = PG_INF;
            s_cs.max_level = 0;
        });
        if (!ok) break;
        const unsigned long long t_end = pg_gtimer();

        // ---- training traces: vertices already at their final distance
        unsigned long long settled = 0;
        if (!kReach && A.L.ref_dist != nullptr && A.L.trace != nullptr && r < A.L.trace_cap) {
            unsigned long long cnt = 0;
            for (uint32_t v = gtid; v < n; v += gthreads)
                cnt += (pg_ldcg(A.dist + v) == __ldg(A.L.ref_dist + v)) ? 1u : 0u;
            cnt = warp_sum64(cnt);
            if (lane == 0 && cnt) atomicAdd(&R.sc->settled, cnt);
            if (!pg_grid_sync(ctrl, nblocks, gen, tmo, &s_flag)) break;
            settled = pg_ldcg64(&R.sc->settled);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && A.L.trace != nullptr && r < A.L.trace_cap) {
            pg_round_trace tr;
            tr.round = r;
            tr.action = pull ? PG_ACTION_PULL : (uint32_t)(31 - __clz((int)max(R.tau, 1u)));
            tr.frontier = R.F;
            tr.min_level = Lvl;
            tr.out_edges = E;
            tr.t_begin_ns = t_round;
            tr.t_end_ns = t_end;
            tr.settled = settled;
            for (int i = 0; i < 5; i++) tr.features[i] = x[i];
            tr.reserved = 0;
            A.L.trace[r] = tr;
        }
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

size_t traverse_smem(const PgLaunch &L) {
    const uint32_t nw = L.threads / 32;
    return 6144 + (size_t)nw * 256 +
           (size_t)nw * (4u * 32u + 2u * kSpillCap + 2u * warp_fifo_words(L)) * 4u +
           (size_t)(6u * L.cta_queue + 4u) * 4u + (vt_enabled(L) ? (8u << kVtLog2) : 0u);
}

template <bool kReach>
pg_status launch_impl(pg_graph *g, PgLaunch &L, TravArgs &A, cudaStream_t s) {
    auto kern = pg_traverse_kernel<kReach>;
    const size_t smem = traverse_smem(L);
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
    const uint32_t bps = L.blocks ? min((uint32_t)per_sm, L.blocks) : (uint32_t)per_sm;
    const uint32_t grid = bps * (uint32_t)g->num_sms;
    L.blocks = bps;
    A.L = L;
    PG_CK(cudaMemsetAsync(g->d_ctrl, 0, sizeof(PgCtrl), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaEventRecord(g->ev0, s));
    PG_CK(cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(L.threads), args, smem,
                                      s));
    PG_CK(cudaEventRecord(g->ev1, s));
    return PG_OK;
}

void fill_traverse_args(TravArgs &A, const pg_graph *g, const PgLaunch &L, int kind,
                        uint32_t src, const uint32_t *sources, uint32_t k, uint32_t dir,
                        uint32_t *dist, unsigned long long *fwd, unsigned long long *bwd) {
    memset(&A, 0, sizeof(A));
    A.G.off = g->d_off;
    A.G.idx = g->d_idx;
    A.G.toff = g->d_toff ? g->d_toff : g->d_off;
    A.G.tidx = g->d_tidx ? g->d_tidx : g->d_idx;
    A.G.n = g->n;
    A.G.m = g->m;
    A.ell0 = g->d_ell[0];
    A.ellw0 = g->d_ell[0] ? g->ellw[0] : 0u;
    A.ell1 = g->d_ell[1];
    A.ellw1 = g->d_ell[1] ? g->ellw[1] : 0u;
    A.ctrl = g->d_ctrl;
    A.bag = g->d_bag;
    A.cap = g->bag_cap;
    A.stamp = g->d_stamp;
    A.hubs = g->d_hubs;
    A.hcap = g->hub_cap;
    A.dist = dist;
    A.mask0 = fwd;
    A.mask1 = bwd;
    A.src = src;
    A.k = k;
    A.dir = dir;
    A.need_deg = (kind == 0 && L.schedule == PG_SCHED_FIXED && L.direction == PG_DIR_AUTO &&
                  L.allow_pull) ? 1u : 0u;
    const uint32_t md =
        (kind == 1 && (dir & PG_BWD)) ? max(g->maxdeg[0], g->maxdeg[1]) : g->maxdeg[0];
    A.hubs_possible = md >= L.hub_degree ? 1u : 0u;
    for (uint32_t j = 0; j < k && j < 64; j++) A.sources[j] = sources[j];
}

}  // namespace

// The two instantiations of the kernel are compiled in separate translation
// units (this file for BFS, pg_traverse_reach.cu for reachability, which
// includes it with PG_TRAVERSE_REACH_TU defined), so that they build in
// parallel; each unit emits device code only for the kernel it launches.
#ifndef PG_TRAVERSE_REACH_TU

pg_status pg_launch_bfs_raw(const PgRawBfs &w, PgLaunch &L, cudaStream_t s) {
    TravArgs A;
    memset(&A, 0, sizeof(A));
    A.G.off = w.off;
    A.G.idx = w.idx;
    A.G.toff = w.off;   // push only: the reverse lists are never read
    A.G.tidx = w.idx;
    A.G.n = w.n;
    A.G.m = w.m;
    A.ctrl = w.ctrl;
    A.bag = w.bag;
    A.cap = w.cap;
    A.stamp = w.stamp;
    A.hubs = nullptr;
    A.hcap = 0;
    A.dist = w.dist;
    A.src = w.src;
    A.need_deg = 0;
    A.hubs_possible = 0;
    auto kern = pg_traverse_kernel<false>;
    const size_t smem = traverse_smem(L);
    int maxopt = 0;
    PG_CK(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, w.device));
    if (smem > (size_t)maxopt)
        return pg_set_error(PG_ERR_INVALID_ARG,
                            "launch shape needs %zu B shared memory > %d (threads=%u, local_queue=%u)",
                            smem, maxopt, L.threads, L.qcap);
    PG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)L.threads, smem));
    if (per_sm < 1)
        return pg_set_error(PG_ERR_INVALID_ARG, "launch shape does not fit an SM (threads=%u, local_queue=%u)",
                            L.threads, L.qcap);
    const uint32_t bps = L.blocks ? min((uint32_t)per_sm, L.blocks) : (uint32_t)per_sm;
    L.blocks = bps;
    A.L = L;
    PG_CK(cudaMemsetAsync(w.ctrl, 0, sizeof(PgCtrl), s));
    void *args[] = {(void *)&A};
    PG_CK(cudaLaunchCooperativeKernel((const void *)kern, dim3(bps * (uint32_t)w.num_sms),
                                      dim3(L.threads), args, smem, s));
    return PG_OK;
}

pg_status pg_launch_traverse(pg_graph *g, PgLaunch &L, int kind, uint32_t src,
                             const uint32_t *sources, uint32_t k, uint32_t dir, uint32_t *dist,
                             unsigned long long *fwd, unsigned long long *bwd, cudaStream_t s) {
    if (kind != 0) return pg_launch_traverse_reach(g, L, kind, src, sources, k, dir, dist, fwd, bwd, s);
    TravArgs A;
    fill_traverse_args(A, g, L, kind, src, sources, k, dir, dist, fwd, bwd);
    return launch_impl<false>(g, L, A, s);
}

#else

pg_status pg_launch_traverse_reach(pg_graph *g, PgLaunch &L, int kind, uint32_t src,
                                   const uint32_t *sources, uint32_t k, uint32_t dir,
                                   uint32_t *dist, unsigned long long *fwd,
                                   unsigned long long *bwd, cudaStream_t s) {
    TravArgs A;
    fill_traverse_args(A, g, L, kind, src, sources, k, dir, dist, fwd, bwd);
    return launch_impl<true>(g, L, A, s);
}

#endif  // PG_TRAVERSE_REACH_TU

// pg_internal.cuh -- internal types and device primitives of the sm_103a
// traversal library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pasgal.h"

#define PG_INF 0xFFFFFFFFu
#define PG_NONE 0xFFFFFFFFu

// device status bits (Ctrl::status)
#define PG_DEV_TIMEOUT 1u
#define PG_DEV_OVERFLOW 2u
#define PG_DEV_STALLED 4u

#define PG_NUM_SLOTS 3

// Per-round counters of one frontier bag.  Three of them form a ring: the
// bag being read (round i), the one being filled (round i + 1) and the one
// being reset for round i + 2, so no reset ever races with a use.
struct alignas(128) PgSlot {
    unsigned size;                 // entries appended to the bag
    unsigned head;                 // grab cursor over regular entries
    unsigned hub_cursor;           // grab cursor over concatenated hub edges
    unsigned min_level;            // min tentative distance pushed (incl. de-duplicated pushes)
    unsigned max_level;            // max tentative distance pushed
    unsigned long long out_edges;  // sum of out-degrees of appended entries
    unsigned long long hub_pack;   // (hub count << 40) | hub edge total
    unsigned long long settled;    // trace: vertices equal to the reference after the round
    unsigned long long expansions; // vertex expansions during the round that reads this bag
    unsigned pad[2];
};

#define PG_ELL_LONG 0xFFFFFFFEu  // padded-row marker: the vertex's list is in the CSR

struct alignas(128) PgCtrl {
    unsigned bar_cnt;              // grid-barrier arrivals (monotone, wraps)
    unsigned pad0[31];
    unsigned status;               // PG_DEV_* bits
    unsigned rounds;               // rounds executed
    unsigned pull_rounds;
    unsigned next_action;          // learned schedule: the action CTA 0 chose for the next round
    unsigned long long pushes;
    unsigned long long expansions;
    unsigned long long round_t[4];   // CTA 0's clock at the start of round r (entry r % 4)
    unsigned long long exp_edges[4]; // edges expanded in round r (entry r % 4)
    unsigned exp_verts[4];           // vertices expanded in round r (entry r % 4)
    unsigned dbg_site, dbg_value, dbg_round;  // PG_DEBUG_BOUNDS builds: first bad index
    unsigned pad2[9];
    PgSlot slot[PG_NUM_SLOTS];
};

struct PgHub {
    uint32_t v;      // vertex with out-degree >= hub_degree
    uint32_t start;  // start of its edges in the concatenated hub-edge space (< 2^40 packed)
};

// ------------------------------------------------------------ primitives

__device__ __forceinline__ unsigned long long pg_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned pg_ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned pg_ld_volatile(const unsigned *p) {
    return *(const volatile unsigned *)p;
}

__device__ __forceinline__ void pg_st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// L2-coherent load (bypasses the non-coherent L1) for data other SMs update.
__device__ __forceinline__ uint32_t pg_ldcg(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long pg_ldcg64(const unsigned long long *p) {
    return __ldcg(p);
}

// Fire-and-forget fetch of the line holding p into this SM's L1 (and L2).
__device__ __forceinline__ void pg_prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned pg_lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Grid-wide barrier for a persistent, co-resident grid.  Thread 0 of every
// CTA adds 1 to one monotone counter with release semantics and polls it
// with relaxed loads until it reaches (generation + 1) * nblocks, then
// fences (acquire).  Measured on GB300 at ~1.2 us for 152 CTAs, about half
// a flag-array or arrive-and-flip barrier.  Every wait is bounded: after
// `timeout_ns` (or an iteration cap) the waiter sets PG_DEV_TIMEOUT and
// leaves; a waiter that sees the status set leaves at once.  Returns false
// when the traversal must stop.
__device__ __forceinline__ unsigned pg_ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// pg_grid_sync_then: the same barrier, with `pre()` run by thread 0 after the
// CTA's threads have all arrived and before the CTA's arrival is released,
// so that per-CTA aggregates (built in shared memory during the round) reach
// global memory with one atomic per CTA and are visible to every CTA after
// the barrier, at no extra CTA barrier.
template <class Pre>
__device__ __forceinline__ bool pg_grid_sync_then(PgCtrl *c, unsigned nblocks, unsigned &gen,
                                                  unsigned long long timeout_ns, int *s_flag,
                                                  Pre pre) {
    __syncthreads();
    if (threadIdx.x == 0) {
        pre();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&c->bar_cnt) : "memory");
        const unsigned target = (gen + 1u) * nblocks;
        const unsigned long long t0 = pg_gtimer();
        unsigned long long it = 0;
        while ((int)(pg_ld_relaxed(&c->bar_cnt) - target) < 0) {
            if ((++it & 31ull) == 0) {
                if (pg_ld_volatile(&c->status) != 0u) break;
                if (pg_gtimer() - t0 > timeout_ns || it > (1ull << 34)) {
                    atomicOr(&c->status, PG_DEV_TIMEOUT);
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        *s_flag = (pg_ld_volatile(&c->status) != 0u);
    }
    gen++;
    __syncthreads();
    return *s_flag == 0;
}

__device__ __forceinline__ bool pg_grid_sync(PgCtrl *c, unsigned nblocks, unsigned &gen,
                                             unsigned long long timeout_ns, int *s_flag) {
    return pg_grid_sync_then(c, nblocks, gen, timeout_ns, s_flag, [] {});
}

// ------------------------------------------------------------ host side

struct PgGraphDev {
    const uint32_t *off, *idx;    // forward CSR
    const uint32_t *toff, *tidx;  // reversed CSR (== forward for undirected)
    uint32_t n, m;
};

// Internal helpers shared by the host translation units.
pg_status pg_set_error(pg_status st, const char *fmt, ...);
pg_status pg_cuda_error(cudaError_t e, const char *what);
int pg_device_sms(int dev);

#define PG_CK(call)                                                  \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return pg_cuda_error(e_, #call);      \
    } while (0)

struct PgMsbfsWork;  // batched BFS buffers (pg_msbfs.cu)
struct PgSccWork;    // SCC buffers (pg_scc.cu)
struct PgSsspWork;   // arc weights and SSSP counters (pg_sssp.cu)
void pg_scc_release(pg_graph *g);
void pg_sssp_release(pg_graph *g);
void pg_msbfs_release(pg_graph *g);  // frees them; rebuilt on the next batched call

struct pg_graph {
    int device;
    uint32_t n, m, flags;
    bool has_transpose, transpose_is_self;
    uint32_t *d_off, *d_idx, *d_toff, *d_tidx;
    uint32_t *d_ell[2];   // padded adjacency rows (forward, reverse) or null
    uint32_t ellw[2];     // their width: 4, 8 or 16 neighbour slots, 0 = none
    uint32_t maxdeg[2];   // largest out-degree (forward, reverse)
    // traversal workspace
    uint32_t *d_bag;      // 2 * bag_cap
    uint32_t bag_cap;
    uint32_t *d_stamp;    // 2n round tags (de-duplication)
    PgHub *d_hubs;        // 2 * hub_cap
    uint32_t hub_cap;
    uint32_t hub_degree_alloc;  // hub degree the hub capacity was sized for
    PgCtrl *d_ctrl;
    PgCtrl *h_ctrl;       // pinned host copy for status/statistics
    uint32_t epoch;       // round-tag base for d_stamp
    void *d_stage;        // staging for host-memory outputs
    size_t stage_bytes;
    pg_round_trace *d_trace;
    uint32_t trace_cap;
    uint8_t *d_script;
    uint32_t script_cap;
    float *d_weights;
    bool has_weights;
    PgMsbfsWork *msbfs;
    PgSccWork *scc;
    PgSsspWork *sssp;
    int num_sms;
    cudaEvent_t ev0, ev1;  // bracket the traversal kernel of the last call
};

// per-call launch parameters resolved from pg_config
struct PgLaunch {
    uint32_t schedule, tau, direction, alpha, beta;
    uint32_t blocks, threads, qcap, chunk, hub_degree;
    unsigned long long timeout_ns;
    uint32_t max_rounds, seed, script_len, trace_cap, stall_block;
    const uint8_t *script;       // device
    pg_round_trace *trace;       // device
    const uint32_t *ref_dist;    // device
    const float *weights;        // device
    uint32_t epoch;
    uint32_t allow_pull;
    uint32_t vgc;        // PG_VGC_CTA / PG_VGC_WARP
    uint32_t cta_queue;  // CTA level-buffer capacity
};

pg_status pg_resolve_config(pg_graph *g, const pg_config *cfg, PgLaunch *L, cudaStream_t s);
pg_status pg_stage(pg_graph *g, size_t bytes, void **dev, cudaStream_t s);
// out[i] = in[0] + ... + in[i-1] for i < len (device arrays, stream-ordered)
pg_status pg_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t len, cudaStream_t s);
bool pg_is_device_ptr(const void *p);
pg_status pg_ensure_trace(pg_graph *g, const pg_config *cfg, PgLaunch *L, cudaStream_t s);
pg_status pg_finish_call(pg_graph *g, const PgLaunch &L, const pg_config *cfg,
                         pg_stats *stats, cudaStream_t s);

// kernels launched from the API translation unit
pg_status pg_launch_traverse(pg_graph *g, PgLaunch &L, int kind, uint32_t src,
                             const uint32_t *sources, uint32_t k, uint32_t dir,
                             uint32_t *dist, unsigned long long *fwd, unsigned long long *bwd,
                             cudaStream_t s);
// kind != 0 of pg_launch_traverse (reachability), defined in its own
// translation unit (pg_traverse_reach.cu)
pg_status pg_launch_traverse_reach(pg_graph *g, PgLaunch &L, int kind, uint32_t src,
                                   const uint32_t *sources, uint32_t k, uint32_t dir,
                                   uint32_t *dist, unsigned long long *fwd,
                                   unsigned long long *bwd, cudaStream_t s);
pg_status pg_launch_msbfs(pg_graph *g, PgLaunch &L, const uint32_t *sources, uint32_t k,
                          uint32_t chunk_len, uint32_t *dist, cudaStream_t s);

// BFS launch on caller-provided workspace (used by the allocation-free entry
// point): CSR, output and every scratch buffer are given as raw pointers.
struct PgRawBfs {
    const uint32_t *off, *idx;
    uint32_t n, m, src;
    uint32_t *dist;
    PgCtrl *ctrl;
    uint32_t *bag;    // 2 * cap entries
    uint32_t cap;
    uint32_t *stamp;  // n entries
    int device, num_sms;
};
pg_status pg_launch_bfs_raw(const PgRawBfs &w, PgLaunch &L, cudaStream_t s);

/*
 * pasgal.h -- C ABI of the GB300 (sm_103a) frontier-traversal library.
 *
 * The library computes exact BFS hop distances and multi-source
 * reachability with the frontier-based scheme of Algorithm 1 of the paper
 * (PASGAL, arXiv 2404.17101), made faster by vertical granularity control
 * (VGC, Sec. 2.1): each task runs a bounded local search over several hops,
 * and a vertex is queued again whenever its distance improves (Sec. 2.2),
 * so the result is the exact fixpoint whatever the schedule.
 *
 * Conventions shared by every entry point
 *  - Vertex ids and CSR offsets/indices are uint32; n < 2^31, m < 2^32.
 *  - Every call returns a pg_status; PG_OK is 0.  On failure a message is
 *    stored for the calling thread and can be read with pg_last_error().
 *    No entry point aborts, throws or prints.
 *  - Device buffers are plain device pointers (e.g. the data pointer of a
 *    contiguous torch tensor).  `stream` is a cudaStream_t passed as void*
 *    (NULL = legacy default stream).  Work is enqueued on that stream; the
 *    traversal entry points then wait for their own 16-byte status word, so
 *    when they return PG_OK the output is complete and valid.
 *  - "Unreachable" is 0xFFFFFFFF in distance outputs and bit 0 in masks.
 */
#ifndef PASGAL_GB300_H
#define PASGAL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pg_status {
    PG_OK = 0,
    PG_ERR_INVALID_ARG = 1,   /* bad pointer, size or id; nothing was launched */
    PG_ERR_INVALID_GRAPH = 2, /* CSR failed validation at upload */
    PG_ERR_OOM = 3,           /* device allocation failed */
    PG_ERR_CUDA = 4,          /* a CUDA runtime call failed (message has the name) */
    PG_ERR_TIMEOUT = 5,       /* a device wait exceeded cfg->timeout_ms; outputs undefined */
    PG_ERR_UNSUPPORTED = 6,   /* e.g. pull without a transpose, no device */
    PG_ERR_OVERFLOW = 7       /* a device queue overflowed (should not happen) */
} pg_status;

/* pg_graph_upload flags */
#define PG_DIRECTED 1u        /* arcs as given; otherwise the CSR must be symmetric */
#define PG_BUILD_TRANSPOSE 2u /* build the reversed CSR on the device (pull, backward reach) */
#define PG_SKIP_VALIDATE 4u   /* trust the CSR (skips the validation kernel) */
#define PG_ELL 8u             /* also build padded adjacency rows (see pg_graph_upload) */

/* pg_reach_multi directions */
#define PG_FWD 1u
#define PG_BWD 2u

/* schedules (pg_config.schedule) */
#define PG_SCHED_FIXED 0u   /* fixed tau; push/pull by the Beamer test if direction = AUTO */
#define PG_SCHED_LEARNED 1u /* per-round action from the schedule MLP (weights required), judged
                               against the fixed push action tau = cfg->tau: the network's choice
                               is taken only when its predicted gain exceeds a margin.  Round r's
                               action comes from round r-1's inputs (the network is evaluated by
                               one warp while the round-end barrier waits); round 0's from its
                               own inputs, known before the first barrier */
#define PG_SCHED_RANDOM 2u  /* uniformly random action per round (trace collection) */
#define PG_SCHED_SCRIPT 3u  /* per-round action read from cfg->script (tests) */

/* local-search organisation (pg_config.vgc_mode), for rounds with tau > 1:
 * PG_VGC_CTA: a CTA takes a share of the frontier and runs a level-by-level
 *   local search of up to tau levels in shared memory, all its warps
 *   splitting each level (levels separated by a CTA barrier);
 * PG_VGC_WARP: every warp runs its own FIFO local search from a chunk of
 *   `chunk` frontier entries;
 * PG_VGC_BUCKETS: PG_VGC_CTA with the paper's multiple frontiers (Sec. 2.2,
 *   BFS): the CTA's vertices at depth 2^i form frontier i, and a round's
 *   local search runs in phases at depths 1, 2, 4, ... < tau separated by
 *   grid barriers, so no CTA expands frontier i before every CTA has
 *   finished the nearer ones (fewer vertices expanded before their distance
 *   is final, at the price of log2(tau) barriers per round). */
#define PG_VGC_CTA 0u
#define PG_VGC_WARP 1u
#define PG_VGC_BUCKETS 2u

/* direction policy for PG_SCHED_FIXED */
#define PG_DIR_PUSH 0u
#define PG_DIR_AUTO 1u

/* Actions of the per-round schedule: a in 0..6 is a push round with
 * tau = 2^a; a = 7 is a pull (bottom-up) round. */
#define PG_NUM_ACTIONS 8u
#define PG_ACTION_PULL 7u

/* Schedule MLP: 5 inputs -> 32 ReLU -> 32 ReLU -> 8 outputs, fp32,
 * packed W1[32][5], b1[32], W2[32][32], b2[32], W3[8][32], b3[8].
 * Inputs of round r (F = frontier entries, E = their out-edges, t = the
 * previous round's time in microseconds): log2(1+F)/24, log2(1+E)/32,
 * log2(1+E/F)/8, log2(1+min(r, 2^14))/24, log2(1+t)/16.  Outputs: one score
 * per action (higher = faster predicted). */
#define PG_MLP_IN 5u
#define PG_MLP_HID 32u
#define PG_MLP_NPARAMS 1512u

typedef struct pg_graph pg_graph; /* opaque, library-owned device graph */

/* One record per traversal round (filled when cfg->trace_out != NULL). */
typedef struct pg_round_trace {
    uint32_t round;      /* round index i of Algorithm 1 */
    uint32_t action;     /* action taken (see PG_NUM_ACTIONS) */
    uint32_t frontier;   /* |F_i|: entries in the frontier bag */
    uint32_t min_level;  /* smallest tentative distance pushed into F_i */
    uint64_t out_edges;  /* sum of out-degrees of F_i */
    uint64_t t_begin_ns; /* device %globaltimer at round start */
    uint64_t t_end_ns;   /* device %globaltimer after the round's barrier */
    uint64_t settled;    /* vertices whose distance equals cfg->ref_dist after the round (0 if none) */
    float features[5];   /* schedule-MLP inputs of this round */
    uint32_t reserved;
} pg_round_trace;        /* 72 bytes */

typedef struct pg_config {
    uint32_t struct_size;       /* sizeof(pg_config) */
    uint32_t schedule;          /* PG_SCHED_* */
    uint32_t tau;               /* VGC window: a task's local search expands vertices within tau hops of the
                                   round's frontier (BFS: distance < L + tau; reach: hops < tau); 1 = plain BFS */
    uint32_t direction;         /* PG_DIR_PUSH or PG_DIR_AUTO (fixed schedule only) */
    uint32_t alpha;             /* push -> pull when out_edges(F) > unexplored_edges / alpha */
    uint32_t beta;              /* pull -> push when |F| < n / beta */
    uint32_t blocks_per_sm;     /* persistent CTAs per SM; 0 = as many as fit */
    uint32_t threads_per_block; /* 64..512, multiple of 32; 0 = 512 */
    uint32_t local_queue;       /* per-warp shared-memory queue entries, power of two 32..4096; 0 = 512 */
    uint32_t chunk;             /* frontier entries one warp takes per task (1..32); 0 = 2 */
    uint32_t hub_degree;        /* out-degree from which a vertex's edges are split across warps; 0 = 2048 */
    uint32_t timeout_ms;        /* limit for every device-side wait; 0 = 5000 */
    uint32_t max_rounds;        /* 0 = unlimited */
    uint32_t seed;              /* PG_SCHED_RANDOM stream */
    uint32_t script_len;        /* entries in script */
    uint32_t trace_cap;         /* records available in trace_out */
    uint32_t test_stall_block;  /* fault injection: this CTA never arrives at the grid barrier; 0xFFFFFFFF = off */
    uint32_t vgc_mode;          /* local search for tau > 1: PG_VGC_CTA (default), PG_VGC_WARP or PG_VGC_BUCKETS */
    uint32_t cta_queue;         /* PG_VGC_CTA: vertices per level a CTA keeps locally (64..8192); 0 = 2048 */
    uint32_t delta;             /* pg_sssp: step width of a round's distance threshold; 0 = 8 x mean weight */
    const uint8_t *script;      /* host: action per round for PG_SCHED_SCRIPT (round i uses script[i % len]) */
    pg_round_trace *trace_out;  /* host buffer for per-round records, or NULL */
    const uint32_t *ref_dist;   /* device: known final distances (training traces), or NULL */
} pg_config;

typedef struct pg_stats {
    uint32_t rounds;       /* rounds executed */
    uint32_t pull_rounds;  /* of which bottom-up */
    uint32_t blocks;       /* persistent CTAs launched */
    uint32_t threads;      /* threads per CTA */
    uint64_t expansions;   /* vertex expansions (>= reached vertices; the excess is VGC re-work) */
    uint64_t pushes;       /* entries appended to frontier bags */
    float kernel_ms;       /* CUDA-event time of the traversal kernel launch itself */
    uint32_t reserved;
} pg_stats;

/* Fill *cfg with defaults (fixed schedule, tau = 16, chunk 2, push only, alpha 15, beta 18). */
void pg_config_default(pg_config *cfg);

/*
 * Upload a graph (Sec. 2 preliminaries: G = (V, E), n = |V|, m = |E|).
 *  offsets[n+1], indices[m]: CSR, host or device memory (detected); copied,
 *    so the caller may free them afterwards.  Lists need not be sorted.
 *  flags: PG_DIRECTED, PG_BUILD_TRANSPOSE, PG_SKIP_VALIDATE, PG_ELL.
 *  PG_ELL: when at most 0.1% of the vertices have more than 16
 *    out-neighbours, also keep padded rows (4, 8 or 16 ids per vertex, the
 *    smallest width that 99.9% of the vertices fit) so that a traversal step
 *    reads a neighbour list with 16-byte loads and no offsets lookup; longer
 *    lists stay in the CSR.  Measured slower than the CSR path on GB300 for
 *    now (more instructions per step than the saved offsets load), so it is
 *    opt-in.
 *  Validation (unless skipped): offsets[0] = 0, non-decreasing, offsets[n] = m,
 *    every index < n; failure -> PG_ERR_INVALID_GRAPH.
 *  *out receives a library-owned handle; free it with pg_graph_free.
 */
pg_status pg_graph_upload(const uint32_t *offsets, const uint32_t *indices, uint32_t n,
                          uint32_t m, uint32_t flags, void *stream, pg_graph **out);

/* Supply the reversed CSR (u->w becomes w->u) instead of building it.
 * Same memory and validation rules as pg_graph_upload. */
pg_status pg_graph_set_transpose(pg_graph *g, const uint32_t *t_offsets,
                                 const uint32_t *t_indices, void *stream);

/* Release every device buffer of g (synchronises g's last stream). */
pg_status pg_graph_free(pg_graph *g);

/* n, m and flags of an uploaded graph (any pointer may be NULL). */
pg_status pg_graph_info(const pg_graph *g, uint32_t *n, uint32_t *m, uint32_t *flags);

/*
 * Single-source BFS (Algorithm 1 with VGC, Sec. 2.1-2.2): dist_out[v] = hop
 * distance from src, 0xFFFFFFFF if v is unreachable.
 *  dist_out: n uint32, device or host memory (host: staged, copied back).
 *  cfg: NULL = defaults.  stats: optional host struct.
 *  Errors: src >= n or NULL pointers -> PG_ERR_INVALID_ARG (nothing run);
 *  pull requested without a transpose on a directed graph -> UNSUPPORTED;
 *  device wait over cfg->timeout_ms -> PG_ERR_TIMEOUT (dist undefined).
 */
pg_status pg_bfs(pg_graph *g, uint32_t src, uint32_t *dist_out, const pg_config *cfg,
                 pg_stats *stats, void *stream);

/*
 * Multi-source reachability (Sec. 2.1, reachability search with VGC), k
 * sources at once as bits of one uint64 per vertex.
 *  sources: host array of k ids (1 <= k <= 64; duplicates allowed).
 *  dir: PG_FWD, PG_BWD or both; both run in one persistent launch.
 *  fwd_out[v] bit j = 1 iff v is reachable from sources[j] (PG_FWD);
 *  bwd_out[v] bit j = 1 iff sources[j] is reachable from v (PG_BWD, needs
 *  the transpose on directed graphs).  Bits >= k are 0.  Outputs are n
 *  uint64, device or host memory; an unused direction's pointer may be NULL.
 */
pg_status pg_reach_multi(pg_graph *g, const uint32_t *sources, uint32_t k, uint32_t dir,
                         uint64_t *fwd_out, uint64_t *bwd_out, const pg_config *cfg,
                         pg_stats *stats, void *stream);

/*
 * Batched BFS from k <= 64 sources in one bit-parallel level-synchronous
 * launch (all sources share each round of Algorithm 1).
 *  dist_out: k*n uint32, source-major (dist_out[j*n + v]), device or host.
 *  cfg: direction, alpha, beta, blocks_per_sm, timeout_ms, max_rounds,
 *    test_stall_block, and hub_degree = edges per chunk of a vertex with at
 *    least 32 edges (0 = 1024; the chunk lists are rebuilt when it changes).
 *  Result equals k independent pg_bfs calls.
 */
pg_status pg_bfs_multi(pg_graph *g, const uint32_t *sources, uint32_t k, uint32_t *dist_out,
                       const pg_config *cfg, pg_stats *stats, void *stream);

/*
 * Strongly connected components (Sec. 2.1: parallel SCC built on
 * reachability searches, each run with vertical granularity control; Sec. 2
 * defines an SCC as a maximal vertex set in which every vertex reaches every
 * other).  Forward-backward over all open parts at once: trimming, one pivot
 * per part, forward and backward searches confined to the part with a
 * tau-hop local queue per warp, split into three parts.  Needs the
 * transpose (undirected graphs have it).
 *  label_out:  n uint32, device or host memory; label_out[v] = the smallest
 *              vertex id of v's SCC (deterministic, independent of cfg).
 *  cfg:        tau (hop window of the local search), threads_per_block,
 *              local_queue, timeout_ms (per wait), seed (pivot priorities)
 *              and test_stall_block are used; NULL = defaults.
 *  stats:      rounds = search rounds summed over iterations, expansions =
 *              vertices expanded, kernel_ms = the whole computation; NULL ok.
 *  iterations: number of pivot iterations (NULL ok).
 * Errors: PG_ERR_UNSUPPORTED without a transpose, PG_ERR_TIMEOUT /
 * PG_ERR_OVERFLOW from the device (output undefined).  Buffers are kept on
 * the graph (about 32 bytes per vertex) until pg_graph_free.
 */
pg_status pg_scc(pg_graph *g, uint32_t *label_out, const pg_config *cfg, pg_stats *stats,
                 uint32_t *iterations, void *stream);

/*
 * Arc weights for pg_sssp: weights[e] (uint32) is the weight of arc e of the
 * forward CSR (m entries, host or device memory, copied).  Replaces earlier
 * weights.  Errors: NULL -> PG_ERR_INVALID_ARG; allocation -> PG_ERR_CUDA.
 */
pg_status pg_graph_set_weights(pg_graph *g, const uint32_t *weights, void *stream);

/*
 * Single-source shortest paths (Sec. 2.2, parallel SSSP on the stepping
 * framework with VGC and frontier bags): dist_out[v] = the smallest sum of
 * arc weights over paths src -> v (uint64), 0xFFFFFFFFFFFFFFFF if v is
 * unreachable.  Needs pg_graph_set_weights.  A round expands the frontier
 * entries below L + delta (L = the frontier's smallest tentative distance;
 * cfg->delta, 0 = 8 x the mean weight) and keeps the others; a warp's local
 * search expands its own improvements below the threshold (up to
 * cfg->tau x 8 per task of 32 entries) and queues the rest.  The result is
 * exact for every delta and tau.
 *  dist_out: n uint64, device or host memory.  cfg: tau, delta,
 *  threads_per_block, blocks_per_sm, local_queue, timeout_ms, max_rounds,
 *  test_stall_block are used; NULL = defaults.  stats: rounds, expansions,
 *  pushes, kernel_ms.
 *  Errors: src >= n, NULL, no weights -> PG_ERR_INVALID_ARG; device wait
 *  over timeout_ms -> PG_ERR_TIMEOUT (dist undefined).
 */
pg_status pg_sssp(pg_graph *g, uint32_t src, uint64_t *dist_out, const pg_config *cfg,
                  pg_stats *stats, void *stream);

/*
 * Traversed-edge count for TEPS: *n_reached = #{v : dist[v] != 0xFFFFFFFF},
 * *m_reached = sum of their out-degrees.  dist: device, n entries.
 */
pg_status pg_count_reached(pg_graph *g, const uint32_t *dist, uint64_t *n_reached,
                           uint64_t *m_reached, void *stream);

/* Install schedule-MLP weights (host, PG_MLP_NPARAMS fp32, packed as above)
 * used by PG_SCHED_LEARNED on this graph.  nfloats must equal PG_MLP_NPARAMS. */
pg_status pg_set_schedule_weights(pg_graph *g, const float *weights, size_t nfloats);

/*
 * Schedule-MLP training kernels (all pointers device, fp32 unless noted).
 *  pg_mlp_forward:  Y[B][8] = network(X[B][5]).
 *  pg_mlp_backward: loss = mean_i (Y[i][act[i]] - target[i])^2 and its
 *                   gradient w.r.t. the packed parameters (grad: 1512,
 *                   overwritten); loss_out: 1 float; act: B uint32 (< 8).
 *  pg_mlp_adam:     one Adam step (Kingma & Ba 2015) with bias correction,
 *                   t >= 1 the step number; params, m, v updated in place.
 */
pg_status pg_mlp_forward(const float *params, const float *X, uint32_t B, float *Y, void *stream);
pg_status pg_mlp_backward(const float *params, const float *X, const uint32_t *act,
                          const float *target, uint32_t B, float *grad, float *loss_out,
                          void *stream);
pg_status pg_mlp_adam(float *params, const float *grad, float *m, float *v, uint32_t count,
                      uint32_t t, float lr, float beta1, float beta2, float eps, void *stream);

/*
 * Autotuner: coordinate descent over timed candidates for the given
 * traversal on g; writes the fastest into *cfg (other fields kept).
 *  kind 0 = pg_bfs from sources[0], 1 = pg_reach_multi (dir) from
 *    sources[0..k): local-search organisation, tau, task chunk, local and
 *    CTA queue sizes, threads per CTA, CTAs per SM and hub_degree (the
 *    out-degree from which a vertex's edges are split across warps);
 *  kind 2 = pg_bfs_multi from sources[0..k): hub_degree (there: edges per
 *    chunk of a vertex with >= 32 edges), alpha (push -> pull threshold) and
 *    CTAs per SM.
 * trials: timed runs per candidate (>= 1).  Output buffers are allocated
 * internally (kind 2: k x n uint32).
 */
pg_status pg_autotune(pg_graph *g, uint32_t kind, const uint32_t *sources, uint32_t k,
                      uint32_t dir, uint32_t trials, pg_config *cfg, void *stream);

/*
 * Single-source BFS that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they call, e.g. inside a framework whose memory pool owns the whole
 * device, or in a latency-bound loop where cudaMalloc's implicit device
 * synchronisation is not allowed.  Same result as pg_graph_upload + pg_bfs.
 *  offsets[n+1], indices[m], dist_out[n]: caller-owned DEVICE memory (the
 *    CSR is validated like pg_graph_upload; invalid -> PG_ERR_INVALID_GRAPH).
 *  n must be 1..PG_NOALLOC_MAX_N (larger -> PG_ERR_INVALID_ARG, nothing run).
 *  cfg: NULL or a fixed push schedule (tau, chunk, launch shape, timeout);
 *    learned/scripted schedules, pull rounds and traces -> PG_ERR_UNSUPPORTED.
 *    High-degree vertices are not split across warps here.
 *  The three buffers must be memory of the CURRENT device (another device's
 *    memory -> PG_ERR_INVALID_ARG); the call runs there.
 *  Scratch lives in a fixed array of PG_NOALLOC_SCRATCH_BYTES compiled into
 *    the library (held by every GPU that loads it until exit) and shared by
 *    all calls on a device: calls that overlap on the GPU race, so serialise
 *    them per device.  The first call on a device looks up the array's
 *    address (cudaGetSymbolAddress); make it before any stream capture.
 *  The call is synchronous (it waits on `stream` for the CSR check and for
 *    its status word, copying both into host memory), so it cannot be
 *    recorded into a CUDA graph.  Calls on different devices do not wait
 *    for each other.
 *  No cudaMalloc, cudaFree or allocating library routine is called.
 */
#define PG_NOALLOC_MAX_N (1u << 20)
#define PG_NOALLOC_SCRATCH_BYTES (13u << 20)
pg_status pg_bfs_noalloc(const uint32_t *offsets, const uint32_t *indices, uint32_t n, uint32_t m,
                         uint32_t src, uint32_t *dist_out, const pg_config *cfg, void *stream);

/*
 * Round-barrier latency probe.  Every round of Algorithm 1 ends with a
 * grid-wide barrier, so a traversal of R rounds takes at least R barrier
 * latencies.  This runs the traversal's persistent launch shape
 * (blocks_per_sm CTAs per SM, 0 = 1; threads_per_block, 0 = 512) through
 * `rounds` (1..2^24) grid barriers with no other work and writes the mean
 * time per barrier in microseconds (CUDA events) to *us_per_barrier.
 * Allocates and frees a 1 KB control block on `stream`; synchronous.
 * Errors: PG_ERR_INVALID_ARG (bad sizes, NULL), PG_ERR_TIMEOUT (a barrier
 * wait exceeded 5 s), PG_ERR_CUDA.
 */
pg_status pg_probe_barrier(uint32_t rounds, uint32_t threads_per_block, uint32_t blocks_per_sm,
                           float *us_per_barrier, void *stream);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char *pg_last_error(void);

/* Library version string. */
const char *pg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PASGAL_GB300_H */

// pg_api.cu -- host side of the C ABI: errors, graph upload (validation,
// transpose), configuration, workspace, and the traversal entry points.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pg_internal.cuh"

// ------------------------------------------------------------------ errors

static thread_local std::string t_err;

pg_status pg_set_error(pg_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

pg_status pg_cuda_error(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear sticky-free errors
    if (e == cudaErrorMemoryAllocation)
        return pg_set_error(PG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return pg_set_error(PG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *pg_last_error(void) { return t_err.c_str(); }
extern "C" const char *pg_version(void) { return "pasgal-gb300 0.1 (sm_103a)"; }

int pg_device_sms(int dev) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

bool pg_is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ config

extern "C" void pg_config_default(pg_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(pg_config);
    c->schedule = PG_SCHED_FIXED;
    c->tau = 16;
    c->chunk = 2;
    c->direction = PG_DIR_PUSH;
    c->alpha = 15;
    c->beta = 18;
    c->test_stall_block = 0xFFFFFFFFu;
}

// ------------------------------------------------------------ graph memory
// A graph's device buffers come from the device's default memory pool in
// stream order (cudaMallocAsync).  The pool keeps up to kPoolKeepBytes of
// freed memory for reuse (set once per device, for this process), so
// uploading and freeing graphs repeatedly costs no driver allocation.  A
// buffer is only freed once the device is idle: pg_graph_free and the
// replacement paths synchronise first.
constexpr uint64_t kPoolKeepBytes = 8ull << 30;
constexpr int kMaxPoolDevices = 64;
static std::mutex g_pool_mu;
static bool g_pool_ready[kMaxPoolDevices];

static void pool_setup(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= kMaxPoolDevices || g_pool_ready[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();  // a device without pools keeps the driver default
    g_pool_ready[dev] = true;
}

static cudaError_t dev_alloc(void *p, size_t bytes, cudaStream_t s) {
    return cudaMallocAsync(reinterpret_cast<void **>(p), bytes, s);
}

// Replace a buffer in use by earlier calls: wait for the device, then free.
static void dev_free_idle(void *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    cudaFreeAsync(p, 0);
}

// Pinned host copies of the control block: a process-wide free list
// (cudaMallocHost is slow enough to show in an upload).
static std::mutex g_pin_mu;
static std::vector<PgCtrl *> g_pin_free;

static PgCtrl *pinned_ctrl_get() {
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_free.empty()) {
            PgCtrl *p = g_pin_free.back();
            g_pin_free.pop_back();
            return p;
        }
    }
    PgCtrl *p = nullptr;
    if (cudaMallocHost(&p, sizeof(PgCtrl)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void pinned_ctrl_put(PgCtrl *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

pg_status pg_resolve_config(pg_graph *g, const pg_config *cfg, PgLaunch *L, cudaStream_t s) {
    pg_config d;
    pg_config_default(&d);
    const pg_config *c = cfg ? cfg : &d;
    if (c->struct_size != sizeof(pg_config))
        return pg_set_error(PG_ERR_INVALID_ARG, "pg_config.struct_size %u != %zu (use pg_config_default)",
                            c->struct_size, sizeof(pg_config));
    memset(L, 0, sizeof(*L));
    L->schedule = c->schedule;
    if (L->schedule > PG_SCHED_SCRIPT) return pg_set_error(PG_ERR_INVALID_ARG, "unknown schedule %u", c->schedule);
    L->tau = c->tau ? c->tau : 16;
    if (L->tau > (1u << 20)) return pg_set_error(PG_ERR_INVALID_ARG, "tau %u too large", L->tau);
    L->direction = c->direction;
    L->alpha = c->alpha ? c->alpha : 15;
    L->beta = c->beta ? c->beta : 18;
    L->blocks = c->blocks_per_sm;
    L->threads = c->threads_per_block ? c->threads_per_block : 512;
    if (L->threads < 64 || L->threads > 512 || (L->threads & 31))
        return pg_set_error(PG_ERR_INVALID_ARG, "threads_per_block %u not in 64..512 / multiple of 32", L->threads);
    L->qcap = c->local_queue ? c->local_queue : 512;
    if (L->qcap < 32 || L->qcap > 4096 || (L->qcap & (L->qcap - 1)))
        return pg_set_error(PG_ERR_INVALID_ARG, "local_queue %u must be a power of two in 32..4096", L->qcap);
    L->chunk = c->chunk ? c->chunk : 2;
    if (L->chunk > 32) return pg_set_error(PG_ERR_INVALID_ARG, "chunk %u > 32", L->chunk);
    L->hub_degree = c->hub_degree ? c->hub_degree : 2048;
    if (L->hub_degree < 32) return pg_set_error(PG_ERR_INVALID_ARG, "hub_degree %u < 32", L->hub_degree);
    if (L->hub_degree < g->hub_degree_alloc) {
        // more vertices qualify as hubs: grow the hub lists (2 bags x 2 directions)
        PgHub *h = nullptr;
        const uint32_t cap = 2 * (g->m / L->hub_degree) + 66;
        PG_CK(dev_alloc(&h, (size_t)2 * cap * sizeof(PgHub), s));
        dev_free_idle(g->d_hubs);
        g->d_hubs = h;
        g->hub_cap = cap;
        g->hub_degree_alloc = L->hub_degree;
    }
    L->timeout_ns = (unsigned long long)(c->timeout_ms ? c->timeout_ms : 5000) * 1000000ull;
    L->vgc = c->vgc_mode;
    if (L->vgc > PG_VGC_BUCKETS) return pg_set_error(PG_ERR_INVALID_ARG, "vgc_mode %u", c->vgc_mode);
    L->cta_queue = c->cta_queue ? c->cta_queue : 2048;
    if (L->cta_queue < 64 || L->cta_queue > 8192)
        return pg_set_error(PG_ERR_INVALID_ARG, "cta_queue %u not in 64..8192", L->cta_queue);
    L->max_rounds = c->max_rounds;
    L->seed = c->seed;
    L->stall_block = c->test_stall_block;
    L->ref_dist = c->ref_dist;
    L->allow_pull = g->has_transpose ? 1u : 0u;
    if (L->schedule == PG_SCHED_SCRIPT) {
        if (!c->script || c->script_len == 0)
            return pg_set_error(PG_ERR_INVALID_ARG, "PG_SCHED_SCRIPT needs script and script_len");
        if (c->script_len > g->script_cap) {
            dev_free_idle(g->d_script);
            g->d_script = nullptr;
            g->script_cap = 0;
            PG_CK(dev_alloc(&g->d_script, c->script_len, s));
            g->script_cap = c->script_len;
        }
        PG_CK(cudaMemcpyAsync(g->d_script, c->script, c->script_len, cudaMemcpyHostToDevice, s));
        PG_CK(cudaStreamSynchronize(s));
        L->script = g->d_script;
        L->script_len = c->script_len;
    }
    if (L->schedule == PG_SCHED_LEARNED) {
        if (!g->has_weights)
            return pg_set_error(PG_ERR_INVALID_ARG, "PG_SCHED_LEARNED: no weights (pg_set_schedule_weights)");
        L->weights = g->d_weights;
    }
    if (c->trace_out && c->trace_cap) {
        if (c->trace_cap > g->trace_cap) {
            dev_free_idle(g->d_trace);
            g->d_trace = nullptr;
            g->trace_cap = 0;
            PG_CK(dev_alloc(&g->d_trace, (size_t)c->trace_cap * sizeof(pg_round_trace), s));
            g->trace_cap = c->trace_cap;
        }
        L->trace = g->d_trace;
        L->trace_cap = c->trace_cap;
    }
    return PG_OK;
}

pg_status pg_stage(pg_graph *g, size_t bytes, void **dev, cudaStream_t s) {
    if (bytes > g->stage_bytes) {
        dev_free_idle(g->d_stage);
        g->d_stage = nullptr;
        g->stage_bytes = 0;
        PG_CK(dev_alloc(&g->d_stage, bytes, s));
        g->stage_bytes = bytes;
    }
    *dev = g->d_stage;
    return PG_OK;
}

// ------------------------------------------------------ upload kernels

__global__ void k_validate(const uint32_t *off, const uint32_t *idx, uint32_t n, uint32_t m,
                           unsigned *bad) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        const uint32_t o = off[v];
        if (v == 0 && o != 0) atomicOr(bad, 1u);
        if (v == n && o != m) atomicOr(bad, 2u);
        if (v < n && off[v + 1] < o) atomicOr(bad, 4u);
    }
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        if (idx[e] >= n) atomicOr(bad, 8u);
}

__global__ void k_count_in(const uint32_t *idx, uint32_t m, uint32_t *cnt) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        atomicAdd(cnt + idx[e], 1u);
}

// Exclusive scan in three launches: per-block scan of 2048 items, scan of
// the block sums (one block, serial over chunks), add-back.
constexpr int kScanItems = 2048;

__global__ void k_scan_blocks(const uint32_t *in, uint32_t *out, uint32_t len, uint32_t *sums) {
    __shared__ uint32_t s[kScanItems];
    const uint32_t base = blockIdx.x * kScanItems;
    for (int i = threadIdx.x; i < kScanItems; i += blockDim.x)
        s[i] = (base + i < len) ? in[base + i] : 0u;
    __syncthreads();
    // Hillis-Steele would be O(n log n); use a two-pass per-thread segment scan.
    const int per = kScanItems / blockDim.x;
    const int t0 = threadIdx.x * per;
    uint32_t acc = 0;
    for (int i = 0; i < per; i++) { uint32_t x = s[t0 + i]; s[t0 + i] = acc; acc += x; }
    __shared__ uint32_t tsum[1024];
    tsum[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0;
        for (int i = 0; i < (int)blockDim.x; i++) { uint32_t x = tsum[i]; tsum[i] = a; a += x; }
        sums[blockIdx.x] = a;
    }
    __syncthreads();
    const uint32_t add = tsum[threadIdx.x];
    for (int i = 0; i < per; i++) s[t0 + i] += add;
    __syncthreads();
    for (int i = threadIdx.x; i < kScanItems; i += blockDim.x)
        if (base + i < len) out[base + i] = s[i];
}

__global__ void k_scan_sums(uint32_t *sums, uint32_t nb) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t a = 0;
        for (uint32_t i = 0; i < nb; i++) { uint32_t x = sums[i]; sums[i] = a; a += x; }
    }
}

__global__ void k_scan_add(uint32_t *out, uint32_t len, const uint32_t *sums) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += sums[i / kScanItems];
}

__global__ void k_scatter_rev(const uint32_t *off, const uint32_t *idx, uint32_t n,
                              uint32_t *cursor, uint32_t *tidx) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        for (uint32_t e = off[u]; e < off[u + 1]; e++) tidx[atomicAdd(cursor + idx[e], 1u)] = u;
}

// Sort each reversed list (short lists: insertion sort by one thread).
__global__ void k_sort_rows(const uint32_t *off, uint32_t *idx, uint32_t n) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t b = off[v], e = off[v + 1];
        if (e - b > 64) continue;  // long rows keep arrival order (order is not needed)
        for (uint32_t i = b + 1; i < e; i++) {
            uint32_t x = idx[i], j = i;
            while (j > b && idx[j - 1] > x) { idx[j] = idx[j - 1]; j--; }
            idx[j] = x;
        }
    }
}

pg_status pg_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t len, cudaStream_t s) {
    const uint32_t nb = (len + kScanItems - 1) / kScanItems;
    uint32_t *sums = nullptr;
    PG_CK(cudaMallocAsync(&sums, (size_t)(nb ? nb : 1) * sizeof(uint32_t), s));
    k_scan_blocks<<<nb, 512, 0, s>>>(in, out, len, sums);
    k_scan_sums<<<1, 32, 0, s>>>(sums, nb);
    k_scan_add<<<(len + 255) / 256, 256, 0, s>>>(out, len, sums);
    PG_CK(cudaGetLastError());
    PG_CK(cudaFreeAsync(sums, s));
    return PG_OK;
}

static pg_status build_transpose(pg_graph *g, cudaStream_t s) {
    const uint32_t n = g->n, m = g->m;
    uint32_t *cnt = nullptr;
    PG_CK(cudaMallocAsync(&cnt, ((size_t)n + 1) * sizeof(uint32_t), s));
    PG_CK(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * sizeof(uint32_t), s));
    const int grid = g->num_sms * 8;
    if (m) k_count_in<<<grid, 256, 0, s>>>(g->d_idx, m, cnt);
    PG_CK(cudaMallocAsync(&g->d_toff, ((size_t)n + 1) * sizeof(uint32_t), s));
    PG_CK(cudaMallocAsync(&g->d_tidx, (size_t)(m ? m : 1) * sizeof(uint32_t), s));
    pg_status st = pg_exclusive_scan(cnt, g->d_toff, n + 1, s);
    if (st) return st;
    PG_CK(cudaMemcpyAsync(cnt, g->d_toff, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    if (m) {
        k_scatter_rev<<<grid, 256, 0, s>>>(g->d_off, g->d_idx, n, cnt, g->d_tidx);
        k_sort_rows<<<grid, 256, 0, s>>>(g->d_toff, g->d_tidx, n);
    }
    PG_CK(cudaGetLastError());
    PG_CK(cudaFreeAsync(cnt, s));
    g->has_transpose = true;
    g->transpose_is_self = false;
    return PG_OK;
}

// Degree statistics: cnt[0..2] = #vertices with degree > 4, > 8, > 16;
// cnt[3] = largest degree.
__global__ void k_deg_stats(const uint32_t *off, uint32_t n, unsigned *cnt) {
    unsigned a = 0, b = 0, c = 0, mx = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t d = off[v + 1] - off[v];
        a += d > 4; b += d > 8; c += d > 16;
        mx = max(mx, d);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
        c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicAdd(cnt, a);
        if (b) atomicAdd(cnt + 1, b);
        if (c) atomicAdd(cnt + 2, c);
        atomicMax(cnt + 3, mx);
    }
}

// Padded rows: row v holds v's neighbours then 0xFFFFFFFF padding, or
// PG_ELL_LONG in every slot when v has more than W neighbours.
__global__ void k_build_ell(const uint32_t *off, const uint32_t *idx, uint32_t n, uint32_t W,
                            uint32_t *ell) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t b = off[v], d = off[v + 1] - b;
        uint32_t *row = ell + (size_t)v * W;
        if (d > W) {
            for (uint32_t j = 0; j < W; j++) row[j] = PG_ELL_LONG;
        } else {
            for (uint32_t j = 0; j < W; j++) row[j] = (j < d) ? idx[b + j] : PG_NONE;
        }
    }
}

// Degree statistics of one direction; builds its padded rows when they fit.
static pg_status build_rows(pg_graph *g, int which, bool allow, cudaStream_t s) {
    const uint32_t *off = which ? g->d_toff : g->d_off;
    const uint32_t *idx = which ? g->d_tidx : g->d_idx;
    unsigned *cnt = nullptr;
    PG_CK(cudaMallocAsync(&cnt, 4 * sizeof(unsigned), s));
    PG_CK(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned), s));
    k_deg_stats<<<g->num_sms * 4, 256, 0, s>>>(off, g->n, cnt);
    unsigned h[4];
    PG_CK(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    PG_CK(cudaFreeAsync(cnt, s));
    g->maxdeg[which] = h[3];
    g->d_ell[which] = nullptr;
    g->ellw[which] = 0;
    if (!allow) return PG_OK;
    const uint64_t tol = g->n / 1000;
    uint32_t W = 0;
    if (h[0] <= tol) W = 4;
    else if (h[1] <= tol) W = 8;
    else if (h[2] <= tol) W = 16;
    if (!W) return PG_OK;
    uint32_t *ell = nullptr;
    if (dev_alloc(&ell, (size_t)g->n * W * sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();  // no room: CSR only
        return PG_OK;
    }
    k_build_ell<<<g->num_sms * 8, 256, 0, s>>>(off, idx, g->n, W, ell);
    PG_CK(cudaGetLastError());
    g->d_ell[which] = ell;
    g->ellw[which] = W;
    return PG_OK;
}

static pg_status copy_in(uint32_t *dst, const uint32_t *src, size_t count, cudaStream_t s) {
    if (count == 0) return PG_OK;
    const cudaMemcpyKind kind = pg_is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PG_CK(cudaMemcpyAsync(dst, src, count * sizeof(uint32_t), kind, s));
    return PG_OK;
}

static pg_status validate(pg_graph *g, const uint32_t *off, const uint32_t *idx, uint32_t n,
                          uint32_t m, cudaStream_t s) {
    unsigned *bad = nullptr;
    PG_CK(cudaMallocAsync(&bad, sizeof(unsigned), s));
    PG_CK(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
    k_validate<<<g->num_sms * 8, 256, 0, s>>>(off, idx, n, m, bad);
    PG_CK(cudaGetLastError());
    unsigned hbad = 0;
    PG_CK(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    PG_CK(cudaFreeAsync(bad, s));
    if (hbad)
        return pg_set_error(PG_ERR_INVALID_GRAPH, "invalid CSR:%s%s%s%s",
                            (hbad & 1) ? " offsets[0]!=0" : "", (hbad & 2) ? " offsets[n]!=m" : "",
                            (hbad & 4) ? " offsets decrease" : "", (hbad & 8) ? " index>=n" : "");
    return PG_OK;
}

static void release(pg_graph *g) {
    if (!g) return;
    cudaDeviceSynchronize();  // no call may still use the buffers
    auto fr = [](void *p) { if (p) cudaFreeAsync(p, 0); };
    if (g->d_ell[1] && g->d_ell[1] != g->d_ell[0]) fr(g->d_ell[1]);
    fr(g->d_ell[0]);
    fr(g->d_off);
    fr(g->d_idx);
    if (!g->transpose_is_self) {
        fr(g->d_toff);
        fr(g->d_tidx);
    }
    fr(g->d_bag);
    fr(g->d_stamp);
    fr(g->d_hubs);
    fr(g->d_ctrl);
    pinned_ctrl_put(g->h_ctrl);
    fr(g->d_stage);
    fr(g->d_trace);
    fr(g->d_script);
    fr(g->d_weights);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    pg_msbfs_release(g);
    pg_scc_release(g);
    pg_sssp_release(g);
    delete g;
}

static pg_status alloc_workspace(pg_graph *g, uint32_t hub_degree, cudaStream_t s) {
    const uint32_t n = g->n;
    g->bag_cap = 2 * n + 64;  // REACH holds forward and backward entries
    PG_CK(dev_alloc(&g->d_bag, (size_t)2 * g->bag_cap * sizeof(uint32_t), s));
    PG_CK(dev_alloc(&g->d_stamp, (size_t)2 * n * sizeof(uint32_t), s));
    PG_CK(cudaMemsetAsync(g->d_stamp, 0, (size_t)2 * n * sizeof(uint32_t), s));
    g->hub_degree_alloc = hub_degree;
    g->hub_cap = 2 * (g->m / hub_degree) + 66;
    PG_CK(dev_alloc(&g->d_hubs, (size_t)2 * g->hub_cap * sizeof(PgHub), s));
    PG_CK(dev_alloc(&g->d_ctrl, sizeof(PgCtrl), s));
    g->h_ctrl = pinned_ctrl_get();
    if (!g->h_ctrl) return pg_set_error(PG_ERR_OOM, "pinned host status buffer");
    g->epoch = 1;
    return PG_OK;
}

extern "C" pg_status pg_graph_upload(const uint32_t *offsets, const uint32_t *indices, uint32_t n,
                                     uint32_t m, uint32_t flags, void *stream, pg_graph **out) {
    if (!out) return pg_set_error(PG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!offsets || (m && !indices)) return pg_set_error(PG_ERR_INVALID_ARG, "NULL CSR pointer");
    if (n == 0 || n >= 0x80000000u) return pg_set_error(PG_ERR_INVALID_ARG, "n=%u out of range 1..2^31-1", n);
    int dev = 0;
    PG_CK(cudaGetDevice(&dev));
    cudaStream_t s = (cudaStream_t)stream;
    pg_graph *g = new pg_graph();
    memset(g, 0, sizeof(*g));
    g->device = dev;
    g->n = n;
    g->m = m;
    g->flags = flags;
    g->num_sms = pg_device_sms(dev);
    pg_status st = PG_OK;
#define PG_TRY(x)                     \
    do {                              \
        st = (x);                     \
        if (st) { release(g); return st; } \
    } while (0)
#define PG_TRYC(call) PG_TRY(((call) == cudaSuccess) ? PG_OK : pg_cuda_error(cudaGetLastError(), #call))
    {
        pool_setup(dev);
        cudaError_t e = dev_alloc(&g->d_off, ((size_t)n + 1) * sizeof(uint32_t), s);
        if (e == cudaSuccess) e = dev_alloc(&g->d_idx, (size_t)(m ? m : 1) * sizeof(uint32_t), s);
        if (e != cudaSuccess) { release(g); return pg_cuda_error(e, "cudaMalloc(graph)"); }
    }
    PG_TRY(copy_in(g->d_off, offsets, (size_t)n + 1, s));
    PG_TRY(copy_in(g->d_idx, indices, m, s));
    if (!(flags & PG_SKIP_VALIDATE)) PG_TRY(validate(g, g->d_off, g->d_idx, n, m, s));
    if (flags & PG_DIRECTED) {
        if (flags & PG_BUILD_TRANSPOSE) PG_TRY(build_transpose(g, s));
    } else {
        g->d_toff = g->d_off;
        g->d_tidx = g->d_idx;
        g->has_transpose = true;
        g->transpose_is_self = true;
    }
    PG_TRY(build_rows(g, 0, (flags & PG_ELL) != 0, s));
    if (g->has_transpose) {
        if (g->transpose_is_self) {
            g->d_ell[1] = g->d_ell[0];
            g->ellw[1] = g->ellw[0];
            g->maxdeg[1] = g->maxdeg[0];
        } else {
            PG_TRY(build_rows(g, 1, (flags & PG_ELL) != 0, s));
        }
    }
    PG_TRY(alloc_workspace(g, 2048, s));
    {
        cudaError_t e = cudaEventCreate(&g->ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev1);
        if (e != cudaSuccess) { release(g); return pg_cuda_error(e, "cudaEventCreate"); }
    }
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { release(g); return pg_cuda_error(e, "upload"); }
    }
#undef PG_TRY
#undef PG_TRYC
    *out = g;
    return PG_OK;
}

extern "C" pg_status pg_graph_set_transpose(pg_graph *g, const uint32_t *t_offsets,
                                            const uint32_t *t_indices, void *stream) {
    if (!g || !t_offsets || (g->m && !t_indices)) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *toff = nullptr, *tidx = nullptr;
    PG_CK(dev_alloc(&toff, ((size_t)g->n + 1) * sizeof(uint32_t), s));
    if (dev_alloc(&tidx, (size_t)(g->m ? g->m : 1) * sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        dev_free_idle(toff);
        return pg_cuda_error(cudaErrorMemoryAllocation, "cudaMallocAsync(transpose)");
    }
    pg_status st = copy_in(toff, t_offsets, (size_t)g->n + 1, s);
    if (!st) st = copy_in(tidx, t_indices, g->m, s);
    if (!st) st = validate(g, toff, tidx, g->n, g->m, s);
    if (st) { dev_free_idle(toff); dev_free_idle(tidx); return st; }
    if (!g->transpose_is_self) { dev_free_idle(g->d_toff); dev_free_idle(g->d_tidx); }
    if (g->d_ell[1] && g->d_ell[1] != g->d_ell[0]) dev_free_idle(g->d_ell[1]);
    pg_msbfs_release(g);  // its in-edge chunk list refers to the old transpose
    g->d_ell[1] = nullptr;
    g->ellw[1] = 0;
    g->d_toff = toff;
    g->d_tidx = tidx;
    g->has_transpose = true;
    g->transpose_is_self = false;
    st = build_rows(g, 1, (g->flags & PG_ELL) != 0, s);
    if (st) return st;
    PG_CK(cudaStreamSynchronize(s));
    return PG_OK;
}

extern "C" pg_status pg_graph_free(pg_graph *g) {
    if (!g) return PG_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    release(g);
    return PG_OK;
}

extern "C" pg_status pg_graph_info(const pg_graph *g, uint32_t *n, uint32_t *m, uint32_t *flags) {
    if (!g) return pg_set_error(PG_ERR_INVALID_ARG, "NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (flags) *flags = g->flags | (g->has_transpose ? PG_BUILD_TRANSPOSE : 0u);
    return PG_OK;
}

extern "C" pg_status pg_set_schedule_weights(pg_graph *g, const float *w, size_t nfloats) {
    if (!g || !w) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (nfloats != PG_MLP_NPARAMS)
        return pg_set_error(PG_ERR_INVALID_ARG, "weights: %zu floats, expected %u", nfloats, PG_MLP_NPARAMS);
    PG_CK(cudaSetDevice(g->device));
    if (!g->d_weights) {
        PG_CK(dev_alloc(&g->d_weights, PG_MLP_NPARAMS * sizeof(float), 0));
        PG_CK(cudaStreamSynchronize(0));
    }
    const cudaMemcpyKind kind = pg_is_device_ptr(w) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PG_CK(cudaMemcpy(g->d_weights, w, PG_MLP_NPARAMS * sizeof(float), kind));
    g->has_weights = true;
    return PG_OK;
}

// ------------------------------------------------------------ traversals

pg_status pg_finish_call(pg_graph *g, const PgLaunch &L, const pg_config *cfg, pg_stats *stats,
                         cudaStream_t s) {
    // status, counters and slots only (the barrier flags are not needed)
    const size_t off = offsetof(PgCtrl, status);
    PG_CK(cudaMemcpyAsync((char *)g->h_ctrl + off, (const char *)g->d_ctrl + off, sizeof(PgCtrl) - off,
                          cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    const PgCtrl &c = *g->h_ctrl;
    // advance the round-tag epoch past every tag this call used
    const uint64_t next = (uint64_t)g->epoch + c.rounds + 2;
    if (next >= 0xF0000000ull) {
        PG_CK(cudaMemset(g->d_stamp, 0, (size_t)2 * g->n * sizeof(uint32_t)));
        g->epoch = 1;
    } else {
        g->epoch = (uint32_t)next;
    }
    if (stats) {
        stats->rounds = c.rounds;
        stats->pull_rounds = c.pull_rounds;
        stats->blocks = L.blocks * (uint32_t)g->num_sms;
        stats->threads = L.threads;
        stats->expansions = c.expansions;
        stats->pushes = c.pushes;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->ev0, g->ev1) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        stats->kernel_ms = ms;
        stats->reserved = 0;
    }
    if (cfg && cfg->trace_out && cfg->trace_cap && L.trace) {
        const uint32_t nrec = c.rounds < cfg->trace_cap ? c.rounds : cfg->trace_cap;
        if (nrec)
            PG_CK(cudaMemcpy(cfg->trace_out, L.trace, (size_t)nrec * sizeof(pg_round_trace),
                             cudaMemcpyDeviceToHost));
    }
    if (c.dbg_site)
        return pg_set_error(PG_ERR_CUDA, "bounds check: site %u saw id 0x%08x (round %u)", c.dbg_site,
                            c.dbg_value, c.dbg_round);
    if (c.status & PG_DEV_TIMEOUT)
        return pg_set_error(PG_ERR_TIMEOUT, "device wait exceeded %llu ms (round %u)",
                            L.timeout_ns / 1000000ull, c.rounds);
    if (c.status & PG_DEV_OVERFLOW)
        return pg_set_error(PG_ERR_OVERFLOW, "frontier capacity or round limit exceeded (round %u)", c.rounds);
    return PG_OK;
}

extern "C" pg_status pg_bfs(pg_graph *g, uint32_t src, uint32_t *dist_out, const pg_config *cfg,
                            pg_stats *stats, void *stream) {
    if (!g || !dist_out) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (src >= g->n) return pg_set_error(PG_ERR_INVALID_ARG, "src %u >= n %u", src, g->n);
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    PgLaunch L;
    pg_status st = pg_resolve_config(g, cfg, &L, s);
    if (st) return st;
    if (L.ref_dist && !L.trace) L.ref_dist = nullptr;
    L.epoch = g->epoch;
    uint32_t *dev = dist_out;
    const bool host_out = !pg_is_device_ptr(dist_out);
    if (host_out) {
        void *p = nullptr;
        st = pg_stage(g, (size_t)g->n * sizeof(uint32_t), &p, s);
        if (st) return st;
        dev = (uint32_t *)p;
    }
    st = pg_launch_traverse(g, L, 0, src, nullptr, 0, 0, dev, nullptr, nullptr, s);
    if (st) return st;
    if (host_out)
        PG_CK(cudaMemcpyAsync(dist_out, dev, (size_t)g->n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return pg_finish_call(g, L, cfg, stats, s);
}

extern "C" pg_status pg_reach_multi(pg_graph *g, const uint32_t *sources, uint32_t k, uint32_t dir,
                                    uint64_t *fwd_out, uint64_t *bwd_out, const pg_config *cfg,
                                    pg_stats *stats, void *stream) {
    if (!g || !sources) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (k == 0 || k > 64) return pg_set_error(PG_ERR_INVALID_ARG, "k=%u not in 1..64", k);
    if (dir == 0 || (dir & ~(PG_FWD | PG_BWD))) return pg_set_error(PG_ERR_INVALID_ARG, "dir=%u", dir);
    if ((dir & PG_FWD) && !fwd_out) return pg_set_error(PG_ERR_INVALID_ARG, "fwd_out is NULL");
    if ((dir & PG_BWD) && !bwd_out) return pg_set_error(PG_ERR_INVALID_ARG, "bwd_out is NULL");
    if ((dir & PG_BWD) && !g->has_transpose)
        return pg_set_error(PG_ERR_UNSUPPORTED, "backward reachability needs the transpose (PG_BUILD_TRANSPOSE)");
    for (uint32_t j = 0; j < k; j++)
        if (sources[j] >= g->n) return pg_set_error(PG_ERR_INVALID_ARG, "sources[%u]=%u >= n", j, sources[j]);
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    PgLaunch L;
    pg_status st = pg_resolve_config(g, cfg, &L, s);
    if (st) return st;
    L.ref_dist = nullptr;
    L.epoch = g->epoch;
    if (L.schedule == PG_SCHED_LEARNED) L.schedule = PG_SCHED_FIXED;
    const size_t bytes = (size_t)g->n * sizeof(uint64_t);
    unsigned long long *f = (unsigned long long *)fwd_out, *b = (unsigned long long *)bwd_out;
    const bool hf = (dir & PG_FWD) && !pg_is_device_ptr(fwd_out);
    const bool hb = (dir & PG_BWD) && !pg_is_device_ptr(bwd_out);
    if (hf || hb) {
        void *p = nullptr;
        st = pg_stage(g, bytes * 2, &p, s);
        if (st) return st;
        if (hf) f = (unsigned long long *)p;
        if (hb) b = (unsigned long long *)((char *)p + bytes);
    }
    st = pg_launch_traverse(g, L, 1, 0, sources, k, dir, nullptr, f, b, s);
    if (st) return st;
    if (hf) PG_CK(cudaMemcpyAsync(fwd_out, f, bytes, cudaMemcpyDeviceToHost, s));
    if (hb) PG_CK(cudaMemcpyAsync(bwd_out, b, bytes, cudaMemcpyDeviceToHost, s));
    return pg_finish_call(g, L, cfg, stats, s);
}

extern "C" pg_status pg_bfs_multi(pg_graph *g, const uint32_t *sources, uint32_t k, uint32_t *dist_out,
                                  const pg_config *cfg, pg_stats *stats, void *stream) {
    if (!g || !sources || !dist_out) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (k == 0 || k > 64) return pg_set_error(PG_ERR_INVALID_ARG, "k=%u not in 1..64", k);
    for (uint32_t j = 0; j < k; j++)
        if (sources[j] >= g->n) return pg_set_error(PG_ERR_INVALID_ARG, "sources[%u]=%u >= n", j, sources[j]);
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    PgLaunch L;
    pg_status st = pg_resolve_config(g, cfg, &L, s);
    if (st) return st;
    const size_t bytes = (size_t)k * g->n * sizeof(uint32_t);
    uint32_t *dev = dist_out;
    const bool host_out = !pg_is_device_ptr(dist_out);
    if (host_out) {
        void *p = nullptr;
        st = pg_stage(g, bytes, &p, s);
        if (st) return st;
        dev = (uint32_t *)p;
    }
    // edges per chunk of a heavy vertex: cfg->hub_degree when given
    const uint32_t clen = cfg ? cfg->hub_degree : 0u;
    if (clen > (1u << 20)) return pg_set_error(PG_ERR_INVALID_ARG, "hub_degree %u too large", clen);
    st = pg_launch_msbfs(g, L, sources, k, clen, dev, s);
    if (st) return st;
    if (host_out) PG_CK(cudaMemcpyAsync(dist_out, dev, bytes, cudaMemcpyDeviceToHost, s));
    return pg_finish_call(g, L, cfg, stats, s);
}

// ---------------------------------------------------------- TEPS count

__global__ void k_count_reached(const uint32_t *off, const uint32_t *dist, uint32_t n,
                                unsigned long long *out) {
    unsigned long long a = 0, b = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] != PG_INF) { a++; b += off[v + 1] - off[v]; }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, a);
        atomicAdd(out + 1, b);
    }
}

extern "C" pg_status pg_count_reached(pg_graph *g, const uint32_t *dist, uint64_t *n_reached,
                                      uint64_t *m_reached, void *stream) {
    if (!g || !dist || !n_reached || !m_reached) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (!pg_is_device_ptr(dist)) return pg_set_error(PG_ERR_INVALID_ARG, "dist must be device memory");
    PG_CK(cudaSetDevice(g->device));
    cudaStream_t s = (cudaStream_t)stream;
    void *p = nullptr;
    pg_status st = pg_stage(g, 16, &p, s);
    if (st) return st;
    PG_CK(cudaMemsetAsync(p, 0, 16, s));
    k_count_reached<<<g->num_sms * 4, 256, 0, s>>>(g->d_off, dist, g->n, (unsigned long long *)p);
    PG_CK(cudaGetLastError());
    unsigned long long h[2];
    PG_CK(cudaMemcpyAsync(h, p, 16, cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    *n_reached = h[0];
    *m_reached = h[1];
    return PG_OK;
}

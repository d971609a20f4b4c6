// pg_noalloc.cu -- single-source BFS that allocates nothing (pg_bfs_noalloc).
//
// Who needs it: callers that may not allocate device memory at call time,
// for example code running inside a framework whose memory pool owns the
// whole device, a real-time loop where cudaMalloc's implicit device
// synchronisation and unbounded latency are not acceptable, or an embedding
// that has already handed out every byte it may use.  pg_graph_upload and
// pg_bfs allocate (graph copy, frontier bags, round tags, control block);
// this entry point instead works on the caller's CSR and output buffers and
// keeps its scratch in a fixed array compiled into the library.
//
// The scratch is one file-scope __device__ array of PG_NOALLOC_SCRATCH_BYTES
// bytes (about 12.6 MB): the control block, two frontier bags of
// PG_NOALLOC_MAX_N + 64 entries and one round tag per vertex.  Every GPU
// that loads the library holds it until the process exits.  All calls on a
// device share it and it keeps the previous call's contents; the control
// block is cleared on every call and the round tags are made unambiguous by
// a per-device tag base (cleared when it would wrap), so stale contents never
// change a result.  Two calls that overlap on the GPU race on the array:
// serialise calls per device (e.g. issue them on one stream).
//
// Host code may not use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress while
// that device is current and keeps it; that first call therefore performs a
// runtime lookup and should be made before any stream capture begins.
//
// Every call is synchronous: it waits on its stream twice (for the CSR
// check and for the status word) and copies both results into host stack
// memory, so no call can be recorded into a CUDA graph.  The caller's three
// buffers must live on the current device (the one whose scratch array is
// used); a buffer on another device is rejected.  Calls on different
// devices take different locks and do not wait for each other.
#include <mutex>

#include "pg_internal.cuh"

namespace {

constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr uint32_t kCap = PG_NOALLOC_MAX_N + 64u;
constexpr size_t kCtrlOff = 0;
constexpr size_t kFlagOff = round_up(sizeof(PgCtrl));
constexpr size_t kBagOff = kFlagOff + kAlign;
constexpr size_t kStampOff = kBagOff + round_up((size_t)2 * kCap * sizeof(uint32_t));
constexpr size_t kScratchBytes = kStampOff + round_up((size_t)PG_NOALLOC_MAX_N * sizeof(uint32_t));
static_assert(kScratchBytes <= PG_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The fixed scratch shared by every call on a device.
static __device__ __align__(256) unsigned char g_bfs_scratch[PG_NOALLOC_SCRATCH_BYTES];

struct DeviceScratch {
    std::mutex mu;                  // serialises the host side of calls on this device
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_bfs_scratch on this device
    uint32_t epoch = 1;             // round-tag base for the next call
};

constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];

// True when p is device (or managed) memory that belongs to device `dev`.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    // managed memory is reachable from every device of the process
    return a.type == cudaMemoryTypeManaged;
}

// CSR checks (same rules as pg_graph_upload); bit flags into *bad.
__global__ void k_noalloc_validate(const uint32_t *off, const uint32_t *idx, uint32_t n, uint32_t m,
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

}  // namespace

extern "C" pg_status pg_bfs_noalloc(const uint32_t *offsets, const uint32_t *indices, uint32_t n,
                                    uint32_t m, uint32_t src, uint32_t *dist_out,
                                    const pg_config *cfg, void *stream) {
    if (!offsets || (m && !indices) || !dist_out)
        return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (n == 0 || n > PG_NOALLOC_MAX_N)
        return pg_set_error(PG_ERR_INVALID_ARG,
                            "pg_bfs_noalloc: n=%u outside 1..%u (the fixed scratch holds at most %u "
                            "vertices; use pg_graph_upload + pg_bfs for larger graphs)",
                            n, PG_NOALLOC_MAX_N, PG_NOALLOC_MAX_N);
    if (src >= n) return pg_set_error(PG_ERR_INVALID_ARG, "src %u >= n %u", src, n);
    int dev = 0;
    PG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return pg_set_error(PG_ERR_UNSUPPORTED, "device %d", dev);
    if (!on_device(offsets, dev) || (m && !on_device(indices, dev)) || !on_device(dist_out, dev))
        return pg_set_error(PG_ERR_INVALID_ARG,
                            "pg_bfs_noalloc: offsets, indices and dist_out must be device memory "
                            "of the current device (%d)", dev);
    pg_config d;
    pg_config_default(&d);
    const pg_config *c = cfg ? cfg : &d;
    if (c->struct_size != sizeof(pg_config))
        return pg_set_error(PG_ERR_INVALID_ARG, "pg_config.struct_size mismatch");
    if (c->schedule != PG_SCHED_FIXED || c->direction != PG_DIR_PUSH || c->trace_out || c->ref_dist)
        return pg_set_error(PG_ERR_UNSUPPORTED,
                            "pg_bfs_noalloc runs the fixed push schedule only (no learned/scripted "
                            "schedules, pull rounds or traces)");
    PgLaunch L;
    memset(&L, 0, sizeof(L));
    L.schedule = PG_SCHED_FIXED;
    L.tau = c->tau ? c->tau : 16;
    L.direction = PG_DIR_PUSH;
    L.alpha = 15;
    L.beta = 18;
    L.blocks = c->blocks_per_sm;
    L.threads = c->threads_per_block ? c->threads_per_block : 512;
    if (L.threads < 64 || L.threads > 512 || (L.threads & 31))
        return pg_set_error(PG_ERR_INVALID_ARG, "threads_per_block %u not in 64..512 / multiple of 32", L.threads);
    L.qcap = c->local_queue ? c->local_queue : 512;
    if (L.qcap < 32 || L.qcap > 4096 || (L.qcap & (L.qcap - 1)))
        return pg_set_error(PG_ERR_INVALID_ARG, "local_queue %u must be a power of two in 32..4096", L.qcap);
    L.chunk = c->chunk ? c->chunk : 2;
    if (L.chunk > 32) return pg_set_error(PG_ERR_INVALID_ARG, "chunk %u > 32", L.chunk);
    if (L.tau > (1u << 20)) return pg_set_error(PG_ERR_INVALID_ARG, "tau %u too large", L.tau);
    L.hub_degree = 0xFFFFFFFFu;  // no hub splitting: it needs graph-sized hub lists
    L.timeout_ns = (unsigned long long)(c->timeout_ms ? c->timeout_ms : 5000) * 1000000ull;
    L.max_rounds = c->max_rounds;
    L.vgc = c->vgc_mode;
    if (L.vgc > PG_VGC_WARP) return pg_set_error(PG_ERR_INVALID_ARG, "vgc_mode %u", c->vgc_mode);
    L.cta_queue = c->cta_queue ? c->cta_queue : 2048;
    if (L.cta_queue < 64 || L.cta_queue > 8192)
        return pg_set_error(PG_ERR_INVALID_ARG, "cta_queue %u not in 64..8192", L.cta_queue);
    L.stall_block = c->test_stall_block;
    L.allow_pull = 0;

    cudaStream_t s = (cudaStream_t)stream;
    DeviceScratch &D = g_dev[dev];
    std::lock_guard<std::mutex> lock(D.mu);
    if (!D.ready) {
        // one-time set-up on this device (it is current): the array's device address
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_bfs_scratch);
        if (e != cudaSuccess) return pg_cuda_error(e, "cudaGetSymbolAddress(g_bfs_scratch)");
        D.base = static_cast<unsigned char *>(p);
        D.epoch = 1;
        D.ready = true;
    }
    PgCtrl *ctrl = reinterpret_cast<PgCtrl *>(D.base + kCtrlOff);
    unsigned *flag = reinterpret_cast<unsigned *>(D.base + kFlagOff);
    uint32_t *bag = reinterpret_cast<uint32_t *>(D.base + kBagOff);
    uint32_t *stamp = reinterpret_cast<uint32_t *>(D.base + kStampOff);

    // validate the caller's CSR
    PG_CK(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
    int sms = pg_device_sms(dev);
    k_noalloc_validate<<<sms * 4, 256, 0, s>>>(offsets, indices, n, m, flag);
    PG_CK(cudaGetLastError());
    unsigned hbad = 0;
    PG_CK(cudaMemcpyAsync(&hbad, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    if (hbad)
        return pg_set_error(PG_ERR_INVALID_GRAPH, "invalid CSR (flags 0x%x)", hbad);

    // round tags: the array keeps the previous call's tags; a fresh base
    // keeps them unambiguous, and they are cleared before the base wraps
    if (D.epoch > 0xF0000000u) {
        PG_CK(cudaMemsetAsync(stamp, 0, (size_t)PG_NOALLOC_MAX_N * sizeof(uint32_t), s));
        D.epoch = 1;
    }
    L.epoch = D.epoch;
    PgRawBfs w;
    w.off = offsets;
    w.idx = indices;
    w.n = n;
    w.m = m;
    w.src = src;
    w.dist = dist_out;
    w.ctrl = ctrl;
    w.bag = bag;
    w.cap = kCap;
    w.stamp = stamp;
    w.device = dev;
    w.num_sms = sms;
    pg_status st = pg_launch_bfs_raw(w, L, s);
    if (st) return st;
    // status and round count back into host stack memory (no pinned buffer)
    PgCtrl h;
    const size_t off = offsetof(PgCtrl, status);
    PG_CK(cudaMemcpyAsync((char *)&h + off, (const char *)ctrl + off, sizeof(PgCtrl) - off,
                          cudaMemcpyDeviceToHost, s));
    PG_CK(cudaStreamSynchronize(s));
    const uint64_t next = (uint64_t)D.epoch + h.rounds + 2;
    D.epoch = next >= 0xF0000000ull ? 0xF0000001u : (uint32_t)next;
    if (h.status & PG_DEV_TIMEOUT)
        return pg_set_error(PG_ERR_TIMEOUT, "device wait exceeded %llu ms (round %u)",
                            L.timeout_ns / 1000000ull, h.rounds);
    if (h.status & PG_DEV_OVERFLOW)
        return pg_set_error(PG_ERR_OVERFLOW, "frontier capacity or round limit exceeded (round %u)",
                            h.rounds);
    return PG_OK;
}

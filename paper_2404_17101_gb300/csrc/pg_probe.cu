// pg_probe.cu -- latency probe for the round barrier (pg_probe_barrier).
//
// A traversal round of Algorithm 1 ends with a grid-wide barrier, so a
// traversal that needs R rounds can never take less than R barrier
// latencies, however little work the rounds hold.  This probe measures that
// term on the device the library runs on: a persistent cooperative kernel of
// the traversal's launch shape that does nothing but `rounds` grid barriers
// (the same bounded barrier primitive the traversal uses), timed with CUDA
// events.  It is a measurement helper: it computes nothing of the path.
#include "pg_internal.cuh"

namespace {

__global__ void __launch_bounds__(512) k_barrier_probe(PgCtrl *ctrl, uint32_t rounds,
                                                       unsigned long long timeout_ns) {
    __shared__ int s_flag;
    unsigned gen = 0;
    for (uint32_t r = 0; r < rounds; r++)
        if (!pg_grid_sync(ctrl, gridDim.x, gen, timeout_ns, &s_flag)) break;
}

}  // namespace

extern "C" pg_status pg_probe_barrier(uint32_t rounds, uint32_t threads_per_block,
                                      uint32_t blocks_per_sm, float *us_per_barrier, void *stream) {
    if (!us_per_barrier) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (rounds == 0 || rounds > (1u << 24))
        return pg_set_error(PG_ERR_INVALID_ARG, "rounds %u not in 1..2^24", rounds);
    const uint32_t threads = threads_per_block ? threads_per_block : 512u;
    if (threads < 32 || threads > 512 || (threads & 31))
        return pg_set_error(PG_ERR_INVALID_ARG, "threads_per_block %u not in 32..512 / multiple of 32",
                            threads);
    int dev = 0;
    PG_CK(cudaGetDevice(&dev));
    int per_sm = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_probe, (int)threads, 0));
    if (per_sm < 1) return pg_set_error(PG_ERR_CUDA, "barrier probe does not fit an SM");
    const uint32_t bps = blocks_per_sm ? min((uint32_t)per_sm, blocks_per_sm) : 1u;
    const uint32_t grid = bps * (uint32_t)pg_device_sms(dev);
    cudaStream_t s = (cudaStream_t)stream;
    PgCtrl *ctrl = nullptr;
    PG_CK(cudaMallocAsync(&ctrl, sizeof(PgCtrl), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pg_status st = PG_OK;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    unsigned status = 0;
    const unsigned long long timeout_ns = 5000ull * 1000000ull;
    if (ce == cudaSuccess) ce = cudaMemsetAsync(ctrl, 0, sizeof(PgCtrl), s);
    void *args[] = {(void *)&ctrl, (void *)&rounds, (void *)&timeout_ns};
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
    if (ce == cudaSuccess)
        ce = cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(grid), dim3(threads), args,
                                         0, s);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(&status, &ctrl->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce != cudaSuccess) st = pg_cuda_error(ce, "barrier probe");
    else if (status & PG_DEV_TIMEOUT) st = pg_set_error(PG_ERR_TIMEOUT, "barrier probe timed out");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(ctrl, s);
    if (st == PG_OK) *us_per_barrier = ms * 1000.f / (float)rounds;
    return st;
}

// pg_mlp.cu -- training kernels of the schedule network (5 -> 32 -> 32 -> 8,
// ReLU, fp32).  The network is not in the paper: it learns, per round, the
// choice the paper leaves as a tunable constant (tau, Sec. 2.1) together
// with the direction-optimisation switch (Sec. 2.2).
//
// These are GEMV-sized FMA loops; no tensor cores are involved (a batch of
// a few thousand 5-float rows is far too small to feed them).
//   forward:  one thread per row, weights staged in shared memory
//   backward: rows pass (activations and deltas, component-major) then one
//             thread per parameter summing its rows in a fixed order, so
//             the gradient is deterministic; loss summed by one block
//   adam:     element-wise update with host-computed bias corrections
#include <cmath>

#include "pg_internal.cuh"

namespace {

constexpr int kIn = 5, kH = 32, kA = 8;
constexpr int oW1 = 0, ob1 = 160, oW2 = 192, ob2 = 1216, oW3 = 1248, ob3 = 1504, kP = 1512;

__device__ __forceinline__ void load_w(float *s, const float *P) {
    for (int i = threadIdx.x; i < kP; i += blockDim.x) s[i] = P[i];
    __syncthreads();
}

__global__ void k_forward(const float *P, const float *X, uint32_t B, float *Y) {
    __shared__ float w[kP];
    load_w(w, P);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        float x[kIn], h1[kH], h2[kH];
#pragma unroll
        for (int c = 0; c < kIn; c++) x[c] = X[(size_t)i * kIn + c];
#pragma unroll
        for (int j = 0; j < kH; j++) {
            float z = w[ob1 + j];
#pragma unroll
            for (int c = 0; c < kIn; c++) z = fmaf(w[oW1 + j * kIn + c], x[c], z);
            h1[j] = fmaxf(z, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kH; j++) {
            float z = w[ob2 + j];
#pragma unroll
            for (int c = 0; c < kH; c++) z = fmaf(w[oW2 + j * kH + c], h1[c], z);
            h2[j] = fmaxf(z, 0.f);
        }
#pragma unroll
        for (int a = 0; a < kA; a++) {
            float z = w[ob3 + a];
#pragma unroll
            for (int c = 0; c < kH; c++) z = fmaf(w[oW3 + a * kH + c], h2[c], z);
            Y[(size_t)i * kA + a] = z;
        }
    }
}

// Row pass of the backward: stores X^T, h1, h2, dz1, dz2 component-major
// (component c of row i at [c * B + i]), dy and the squared error per row.
__global__ void k_rows(const float *P, const float *X, const uint32_t *act, const float *tgt,
                       uint32_t B, float *H1, float *H2, float *DZ1, float *DZ2, float *DY,
                       float *SQ) {
    __shared__ float w[kP];
    load_w(w, P);
    const float invB = 1.0f / (float)B;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        float x[kIn], z1[kH], h1[kH], z2[kH], h2[kH];
#pragma unroll
        for (int c = 0; c < kIn; c++) x[c] = X[(size_t)i * kIn + c];
#pragma unroll
        for (int j = 0; j < kH; j++) {
            float z = w[ob1 + j];
#pragma unroll
            for (int c = 0; c < kIn; c++) z = fmaf(w[oW1 + j * kIn + c], x[c], z);
            z1[j] = z;
            h1[j] = fmaxf(z, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kH; j++) {
            float z = w[ob2 + j];
#pragma unroll
            for (int c = 0; c < kH; c++) z = fmaf(w[oW2 + j * kH + c], h1[c], z);
            z2[j] = z;
            h2[j] = fmaxf(z, 0.f);
        }
        const uint32_t a = min(act[i], (uint32_t)(kA - 1));
        float y = w[ob3 + a];
#pragma unroll
        for (int c = 0; c < kH; c++) y = fmaf(w[oW3 + a * kH + c], h2[c], y);
        const float err = y - tgt[i];
        const float dy = 2.0f * err * invB;
        DY[i] = dy;
        SQ[i] = err * err;
        float dz2[kH];
#pragma unroll
        for (int j = 0; j < kH; j++) {
            dz2[j] = (z2[j] > 0.f) ? w[oW3 + a * kH + j] * dy : 0.f;
            DZ2[(size_t)j * B + i] = dz2[j];
            H1[(size_t)j * B + i] = h1[j];
            H2[(size_t)j * B + i] = h2[j];
        }
#pragma unroll
        for (int c = 0; c < kH; c++) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < kH; j++) s = fmaf(w[oW2 + j * kH + c], dz2[j], s);
            DZ1[(size_t)c * B + i] = (z1[c] > 0.f) ? s : 0.f;
        }
    }
}

// One thread per parameter; rows summed in index order.
__global__ void k_grad(const float *X, const uint32_t *act, uint32_t B, const float *H1,
                       const float *H2, const float *DZ1, const float *DZ2, const float *DY,
                       const float *SQ, float *G, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kP) return;
    float s = 0.f;
    if (p == kP) {
        for (uint32_t i = 0; i < B; i++) s += SQ[i];
        *loss = s / (float)B;
        return;
    }
    if (p < ob1) {
        const int j = p / kIn, c = p % kIn;
        for (uint32_t i = 0; i < B; i++) s = fmaf(DZ1[(size_t)j * B + i], X[(size_t)i * kIn + c], s);
    } else if (p < oW2) {
        const int j = p - ob1;
        for (uint32_t i = 0; i < B; i++) s += DZ1[(size_t)j * B + i];
    } else if (p < ob2) {
        const int j = (p - oW2) / kH, c = (p - oW2) % kH;
        for (uint32_t i = 0; i < B; i++) s = fmaf(DZ2[(size_t)j * B + i], H1[(size_t)c * B + i], s);
    } else if (p < oW3) {
        const int j = p - ob2;
        for (uint32_t i = 0; i < B; i++) s += DZ2[(size_t)j * B + i];
    } else if (p < ob3) {
        const uint32_t a = (uint32_t)((p - oW3) / kH);
        const int c = (p - oW3) % kH;
        for (uint32_t i = 0; i < B; i++)
            if (min(act[i], (uint32_t)(kA - 1)) == a) s = fmaf(DY[i], H2[(size_t)c * B + i], s);
    } else {
        const uint32_t a = (uint32_t)(p - ob3);
        for (uint32_t i = 0; i < B; i++)
            if (min(act[i], (uint32_t)(kA - 1)) == a) s += DY[i];
    }
    G[p] = s;
}

__global__ void k_adam(float *P, const float *G, float *M, float *V, uint32_t count, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

}  // namespace

extern "C" pg_status pg_mlp_forward(const float *params, const float *X, uint32_t B, float *Y,
                                    void *stream) {
    if (!params || !X || !Y) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (B == 0) return PG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_forward<<<(B + 127) / 128, 128, 0, s>>>(params, X, B, Y);
    PG_CK(cudaGetLastError());
    return PG_OK;
}

extern "C" pg_status pg_mlp_backward(const float *params, const float *X, const uint32_t *act,
                                     const float *target, uint32_t B, float *grad, float *loss_out,
                                     void *stream) {
    if (!params || !X || !act || !target || !grad || !loss_out)
        return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (B == 0) return pg_set_error(PG_ERR_INVALID_ARG, "B = 0");
    cudaStream_t s = (cudaStream_t)stream;
    float *buf = nullptr;
    const size_t per = (size_t)B;
    PG_CK(cudaMallocAsync(&buf, (4 * kH + 2) * per * sizeof(float), s));
    float *H1 = buf, *H2 = H1 + kH * per, *DZ1 = H2 + kH * per, *DZ2 = DZ1 + kH * per,
          *DY = DZ2 + kH * per, *SQ = DY + per;
    k_rows<<<(B + 127) / 128, 128, 0, s>>>(params, X, act, target, B, H1, H2, DZ1, DZ2, DY, SQ);
    k_grad<<<(kP + 1 + 127) / 128, 128, 0, s>>>(X, act, B, H1, H2, DZ1, DZ2, DY, SQ, grad, loss_out);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return pg_cuda_error(e, "mlp backward");
    return PG_OK;
}

extern "C" pg_status pg_mlp_adam(float *params, const float *grad, float *m, float *v,
                                 uint32_t count, uint32_t t, float lr, float beta1, float beta2,
                                 float eps, void *stream) {
    if (!params || !grad || !m || !v) return pg_set_error(PG_ERR_INVALID_ARG, "NULL argument");
    if (t == 0) return pg_set_error(PG_ERR_INVALID_ARG, "Adam step t must be >= 1");
    if (count == 0) return PG_OK;
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, (double)t));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, (double)t));
    k_adam<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, count, lr, beta1,
                                                                  beta2, eps, (float)c1, (float)c2);
    PG_CK(cudaGetLastError());
    return PG_OK;
}

// FP32 throughput probe: the measured peak that the roofline of the
// interior-point solve (an FP32 FMA-bound kernel) is reported against.
//
// Every lane runs 8 independent FMA chains, as scalar FFMA or as packed
// FFMA2 (two FMAs per instruction, fma.rn.f32x2), on a persistent grid of
// 8 blocks of 256 threads per SM; the work is fixed, the time is taken
// with CUDA events on the caller's stream around the second of two
// launches.  flops = 2 per FMA.
#include <cuda_runtime.h>

#include "linmin.h"

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int BLOCKS_PER_SM = 8;
constexpr int ITERS = 1 << 14;

__global__ void __launch_bounds__(THREADS) ffma_probe_kernel(float *out, float m, float a)
{
    float v[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) v[c] = fmaf(v[c], m, a);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) ffma2_probe_kernel(float *out, float m, float a)
{
    float2 v[CHAINS];
    const float2 mm = make_float2(m, m), aa = make_float2(a, a);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) v[c] = make_float2(threadIdx.x * 1e-3f + c, 0.5f * c);
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) v[c] = __ffma2_rn(v[c], mm, aa);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += v[c].x + v[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" linmin_status linmin_fp32_peak(double *tflops_ffma, double *tflops_ffma2,
                                          void *cuda_stream)
{
    if (!tflops_ffma || !tflops_ffma2) return LINMIN_ERR_INVALID;
    *tflops_ffma = *tflops_ffma2 = 0.0;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LINMIN_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = nsm * BLOCKS_PER_SM;
    float *out = nullptr;
    if (cudaMallocAsync(&out, sizeof(float) * blocks * THREADS, st) != cudaSuccess)
        return LINMIN_ERR_OOM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    linmin_status rc = LINMIN_OK;
    double res[2] = {0.0, 0.0};
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = LINMIN_ERR_CUDA;
    } else {
        for (int k = 0; k < 2 && rc == LINMIN_OK; ++k) {
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {      // the first launch warms up
                cudaEventRecord(e0, st);
                if (k == 0) ffma_probe_kernel<<<blocks, THREADS, 0, st>>>(out, 0.9999f, 0.5f);
                else ffma2_probe_kernel<<<blocks, THREADS, 0, st>>>(out, 0.9999f, 0.5f);
                cudaEventRecord(e1, st);
            }
            if (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
                rc = LINMIN_ERR_CUDA;
                break;
            }
            const double fmas = (double)blocks * THREADS * CHAINS * ITERS * (k == 0 ? 1 : 2);
            res[k] = 2.0 * fmas / (ms * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        rc = LINMIN_ERR_CUDA;
    *tflops_ffma = res[0];
    *tflops_ffma2 = res[1];
    return rc;
}

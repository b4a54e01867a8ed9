// Per-bucket launcher of the interior-point kernels (instantiated in
// ipm_b<NS>x<G>_<mode>.cu, one translation unit per bucket and mode).
#pragma once
#include "ipm.cuh"

namespace lm {

template <int NS, int G, bool ACC, bool BATCH = false>
cudaError_t launch_ipm_mode(const IpmArgs &a, cudaStream_t st)
{
    using C = IpmCfg<NS, G>;
    const long long n = BATCH ? (long long)a.total : a.N;
    if (n <= 0) return cudaSuccess;
    auto kern = ipm_kernel<NS, G, ACC, BATCH>;
    const size_t smem = C::smem_bytes(ACC);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    // persistent grid: one wave of resident blocks, capped by the pixel count
    const long long groups_per_block = (long long)C::WARPS * C::GPW;
    long long blocks = (long long)nsm * per_sm;
    const long long need = (n + groups_per_block - 1) / groups_per_block;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, C::THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

#define LM_DECLARE_BUCKET(NS, G)                                                          \
    extern template cudaError_t launch_ipm_mode<NS, G, false>(const IpmArgs &, cudaStream_t); \
    extern template cudaError_t launch_ipm_mode<NS, G, true>(const IpmArgs &, cudaStream_t);  \
    extern template cudaError_t launch_ipm_mode<NS, G, false, true>(const IpmArgs &, cudaStream_t);

LM_DECLARE_BUCKET(2, 4)
LM_DECLARE_BUCKET(4, 4)
LM_DECLARE_BUCKET(4, 8)
LM_DECLARE_BUCKET(9, 4)
LM_DECLARE_BUCKET(5, 8)
LM_DECLARE_BUCKET(3, 16)
LM_DECLARE_BUCKET(4, 16)
LM_DECLARE_BUCKET(2, 8)
LM_DECLARE_BUCKET(8, 4)
LM_DECLARE_BUCKET(6, 8)

}  // namespace lm

// Interior-point kernel, NS = 2 slots of G = 8 lanes per pixel (P <= 16),
// float32 residual phase (single cube and batched).
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<2, 8, false>(const IpmArgs &, cudaStream_t);
template cudaError_t launch_ipm_mode<2, 8, false, true>(const IpmArgs &, cudaStream_t);
}

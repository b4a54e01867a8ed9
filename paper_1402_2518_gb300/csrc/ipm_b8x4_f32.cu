// Interior-point kernel, NS = 8 slots of G = 4 lanes per pixel (P <= 32),
// float32 residual phase (single cube and batched).
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<8, 4, false>(const IpmArgs &, cudaStream_t);
template cudaError_t launch_ipm_mode<8, 4, false, true>(const IpmArgs &, cudaStream_t);
}

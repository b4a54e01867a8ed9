// Interior-point kernel for P <= 32 (NS = 4 slots, G = 8 lanes per pixel),
// float32 residual phase (single cube and batched).
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<4, 8, false>(const IpmArgs &, cudaStream_t);
template cudaError_t launch_ipm_mode<4, 8, false, true>(const IpmArgs &, cudaStream_t);
}

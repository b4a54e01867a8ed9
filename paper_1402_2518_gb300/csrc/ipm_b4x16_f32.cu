// Interior-point kernel for P <= 64 (NS = 4 slots, G = 16 lanes per pixel),
// float32 residual phase (single cube and batched).
#include "ipm_launch.cuh"
namespace lm {
template cudaError_t launch_ipm_mode<4, 16, false>(const IpmArgs &, cudaStream_t);
template cudaError_t launch_ipm_mode<4, 16, false, true>(const IpmArgs &, cudaStream_t);
}
